"""The C ABI from plain C: tests/c_consumer/rlb_c_consumer.c is compiled
as strict C99 (-pedantic -Werror) against include/rlb.h, linked to the built
librlb and run; it makes host-side calls only (sizes, parameter validation,
status strings), so it needs no GPU.  CPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_plain_c_program_uses_the_library(tmp_path):
    if os.environ.get("RLB_LIBRARY_VARIANT", "release") != "release":
        pytest.skip("the bounds build is loaded")
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_0912_2913_gb300 import build

    lib = build.build()
    exe = str(tmp_path / "rlb_c_consumer")
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_consumer", "rlb_c_consumer.c"), "-o", exe, lib,
           f"-Wl,-rpath,{os.path.dirname(lib)}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
