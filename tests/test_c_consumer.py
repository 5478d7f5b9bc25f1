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


def test_plain_c_program_under_asan_and_ubsan(tmp_path):
    """The same program against a build of the library whose host code is
    compiled with AddressSanitizer and UndefinedBehaviorSanitizer (the
    parameter checks, size arithmetic, error strings and the create/destroy
    paths it reaches): it runs clean.  The device code is compiled to PTX only
    (no GPU is used).  CPU."""
    if os.environ.get("RLB_LIBRARY_VARIANT", "release") != "release":
        pytest.skip("the bounds build is loaded")
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    from concurrent.futures import ThreadPoolExecutor

    from paper_0912_2913_gb300 import build as B

    nvcc = B._nvcc()
    san = []
    for f in ("-fsanitize=address", "-fsanitize=undefined", "-fno-omit-frame-pointer",
              "-fno-sanitize-recover=undefined"):
        san += ["-Xcompiler", f]  # one flag each: nvcc splits -Xcompiler values at commas
    arch = ["-gencode", "arch=compute_103a,code=compute_103a"]

    def compile_one(src):
        obj = str(tmp_path / (os.path.splitext(src)[0] + ".o"))
        flags = list(B.NVCC_FLAGS)
        if src in B.FMAD_SOURCES:
            flags[flags.index("-fmad=false")] = "-fmad=true"
        r = subprocess.run([nvcc, *arch, *flags, *san, "-I", B.INCLUDE, "-c",
                            os.path.join(B.CSRC, src), "-o", obj], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        return obj

    with ThreadPoolExecutor(max_workers=len(B.SOURCES)) as ex:
        objs = list(ex.map(compile_one, B.SOURCES))
    lib = str(tmp_path / "librlb_asan.so")
    r = subprocess.run([nvcc, *arch, "-shared", "-o", lib, *objs, "-lcudart", *san],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    exe = str(tmp_path / "rlb_c_consumer_asan")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsanitize=address,undefined",
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c_consumer", "rlb_c_consumer.c"), "-o", exe, lib,
                        f"-Wl,-rpath,{tmp_path}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:protect_shadow_gap=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr[-4000:]
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-4000:]
