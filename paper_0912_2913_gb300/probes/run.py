"""Compile and run the GB300 throughput probes: python -m paper_0912_2913_gb300.probes.run

FP64 and conversion rates bound the FP64 path and shaped the FP32 recovery;
the bulk-copy rates explain the TMA-staged kernel's behaviour.
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    exe = os.path.join(tempfile.gettempdir(), f"gb300_probes_{os.getpid()}")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "gb300_probes.cu")])
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
        return r.returncode
    finally:
        os.remove(exe)


if __name__ == "__main__":
    sys.exit(main())
