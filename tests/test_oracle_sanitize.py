"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer:
a C driver (tests/sanitize/oracle_driver.c) runs init, steps, macro output
and the adjoint entry points on small lattices of every boundary kind, with
solid cells and both equations of state.  CPU only; skipped when gcc cannot
build sanitized binaries."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    exe = str(tmp_path / "oracle_asan")
    cmd = [gcc, "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-ffp-contract=off", "-std=c11", "-o", exe,
           os.path.join(ROOT, "oracle", "rlb_oracle.c"), os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"),
           "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("sanitized build unavailable: " + r.stderr.strip().splitlines()[-1][:200])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr
    assert "ok" in r.stdout
