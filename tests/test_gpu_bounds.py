"""The bounds-checking debug build of librlb (``-DRLB_CHECK_BOUNDS``): every
state-buffer index of the step, adjoint and general-EOS kernels is range
checked on the device.  The parity cases (all forward launch variants, all
adjoint kernels, the autograd path, the general EOS; small, ragged and
solid-cell lattices) run through it in a process of their own and meet no
out-of-range index, and still agree with the oracle.  The checker itself
counts an index outside [0, n) and passes one inside it."""
import json
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_parity_cases_meet_no_out_of_range_index():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_0912_2913_gb300 import build

    build.build(bounds=True)
    env = dict(os.environ, RLB_LIBRARY_VARIANT="bounds")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_driver.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"].startswith("librlb_bounds_")
    assert out["groups"] == {"forward": 0, "adjoint": 0, "autograd": 0, "general_eos": 0}
    e = out["errors"]
    assert e["forward_fp64"] <= 1e-10 and e["forward_fp32"] <= 1e-4
    assert e["adjoint_fp64"] <= 1e-11 and e["adjoint_fp32"] <= 1e-4
    assert e["general_eos"] <= 1e-10
    # [index, checked index, violations counted since the last read]
    assert out["selftest"] == [[5, 5, 0], [10, 0, 1], [-1, 0, 1]]
