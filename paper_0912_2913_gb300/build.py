"""Build librlb.so in-tree with nvcc for sm_103a (GB300).

Each .cu file compiles in its own nvcc process (in parallel); the objects are
linked into ``paper_0912_2913_gb300/_build/librlb_<hash>.so``.  A rebuild
happens only when a source file changed (content hash in the library's file
name).  ``build(bounds=True)`` makes the bounds-checking debug library
``librlb_bounds_<hash>.so`` (``-DRLB_CHECK_BOUNDS``: every state-buffer index
of the step, adjoint and general-EOS kernels is range-checked and counted,
``rlb_debug_bounds_violations`` reads the count); the release library is
unaffected by it.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["rlb_forward.cu", "rlb_stream.cu", "rlb_adjoint.cu", "rlb_eos.cu", "rlb_f64df.cu", "rlb_api.cu"]
HEADERS = ["rlb_internal.h", "rlb_device.cuh", "rlb_collide.cuh", "rlb_tma.cuh", "rlb_dfloat.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit a*b+c contraction, so every kernel computes exactly
# the operations its source writes (fused ones are explicit fma/fmaf calls) and
# results do not depend on launch variant or register allocation.
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-Xcompiler",
              "-fvisibility=hidden", "--expt-relaxed-constexpr"]
# The adjoint kernels are held to the oracle within a tolerance rather than
# bit for bit across launch variants, so contraction is allowed there for speed.
FMAD_SOURCES = {"rlb_adjoint.cu"}


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librlb")
    return cand


def _digest() -> str:
    h = hashlib.sha1()
    for name in SOURCES + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(INCLUDE, "rlb.h"), "rb") as fh:
        h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + sorted(FMAD_SOURCES)).encode())
    return h.hexdigest()[:12]


def unit_digest(source: str) -> str:
    """Digest of what one translation unit is compiled from (the .cu file,
    the shared headers and the flags): the kernels it defines change only if
    this does."""
    h = hashlib.sha1()
    for name in [source] + HEADERS:
        with open(os.path.join(CSRC, name), "rb") as fh:
            h.update(fh.read())
    flags = ARCH + NVCC_FLAGS + (["-fmad=true"] if source in FMAD_SOURCES else [])
    h.update(" ".join(flags).encode())
    return h.hexdigest()[:12]


def _prefix(bounds: bool) -> str:
    return "librlb_bounds_" if bounds else "librlb_"


def library_path(bounds: bool = False) -> str:
    return os.path.join(BUILD, f"{_prefix(bounds)}{_digest()}.so")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, bounds: bool = False) -> str:
    """Compile (if needed) and return the path of librlb_<hash>.so (of the
    bounds-checking librlb_bounds_<hash>.so with ``bounds=True``)."""
    so = library_path(bounds)
    if os.path.exists(so) and not force and not ptxas_info:
        return so
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    tag = _digest()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(src):
        obj = os.path.join(BUILD, f"{os.path.splitext(src)[0]}_{'b' if bounds else ''}{tag}.o")
        flags = list(NVCC_FLAGS) + (["-DRLB_CHECK_BOUNDS"] if bounds else [])
        if src in FMAD_SOURCES:
            flags[flags.index("-fmad=false")] = "-fmad=true"
        cmd = [nvcc, *ARCH, *flags, *extra, "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose or ptxas_info:
        for _, log in results:
            sys.stdout.write(log)
    tmp = so + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    for o, _ in results:
        os.remove(o)
    # drop libraries of superseded sources (of the same kind)
    for f in os.listdir(BUILD):
        if (f.startswith(_prefix(bounds)) and f.endswith(".so") and f[len(_prefix(bounds)):-3].isalnum()
                and os.path.join(BUILD, f) != so):
            try:
                os.remove(os.path.join(BUILD, f))
            except OSError:
                pass
    return so


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds="--bounds" in sys.argv))
