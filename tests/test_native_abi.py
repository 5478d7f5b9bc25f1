"""CPU checks of the C ABI library: it builds, loads, exports every symbol
include/rlb.h declares, and validates parameters (no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_0912_2913_gb300 import _native as N
    from paper_0912_2913_gb300 import build

    build.build()
    N.load()
    return N


def declared_symbols():
    with open(os.path.join(ROOT, "include", "rlb.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"RLB_API\s+[\w\s\*]+?\b(rlb_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    from paper_0912_2913_gb300 import _native as N

    assert declared_symbols() == sorted(N.EXPORTS)


def test_library_exports_every_declared_symbol(native):
    L = native.load()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_parameter_validation(native):
    N = native
    ok = N.make_params(16, 8, 4, 0.8)
    S, elem, nbytes = N.rlb_state_layout(ok)
    assert S % 64 == 0 and S >= 16 * 8 * 4 and elem == 8 and nbytes == 38 * S * 8
    p32 = N.make_params(200, 100, 100, 0.8, prec=N.RLB_FP32_DEV, xbc=N.RLB_BC_INFLOW_OUTFLOW, n_ref=0.3, eps_ref=0.1)
    S, elem, nbytes = N.rlb_state_layout(p32)
    assert elem == 4 and nbytes == 38 * S * 4
    assert N.rlb_workspace_bytes(p32) >= 2 * nbytes
    bad = [
        N.make_params(0, 1, 1, 0.8),
        N.make_params(4, 4, 4, 0.5),  # tau must be > 1/2
        N.make_params(4, 4, 4, 0.8, c_l=0.0),
        N.make_params(2, 4, 4, 0.8, xbc=N.RLB_BC_OUTFLOW_BOTH),  # ghost planes need nx >= 3
        N.make_params(4, 4, 4, 0.8, xbc=N.RLB_BC_INFLOW_OUTFLOW, beta_in=(1.0, 0.0, 0.0)),
        N.make_params(4, 4, 4, 0.8, prec=N.RLB_FP32_DEV, n_ref=0.0),
        N.make_params(2048, 2048, 1024, 0.8),  # N >= 2^31
        N.make_params(4, 4, 4, 0.8, prec=N.RLB_FP32_DEV, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=5 / 3),  # FP64 only
        N.make_params(4, 4, 4, 0.8, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=1.0),  # 1 < Gamma <= 2
        N.make_params(4, 4, 4, 0.8, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=2.5),
        N.make_params(4, 4, 4, 0.8, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=1.5, eos_mass=-1.0),
        N.make_params(4, 4, 2, 0.8, zbc=N.RLB_ZBC_HALO),  # a z slab needs nz >= 3
        N.make_params(4, 4, 4, 0.8, zbc=2),
        N.make_params(4, 4, 4, 0.8, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=5 / 3, zbc=N.RLB_ZBC_HALO),
        N.make_params(2145386497, 1, 1, 0.8),  # N > 2^31 - 2^21
    ]
    for p in bad:
        with pytest.raises(N.RLBError) as ei:
            N.rlb_state_layout(p)
        assert ei.value.status == N.RLB_ERR_ARG
    p = N.make_params(4, 4, 4, 0.8)
    p.eos = 2
    with pytest.raises(N.RLBError):
        N.rlb_workspace_bytes(p)
    N.rlb_state_layout(N.make_params(4, 4, 4, 0.8, eos=N.RLB_EOS_GAMMA_LAW, eos_gamma=5 / 3, eos_mass=0.5))
    N.rlb_state_layout(N.make_params(4, 4, 3, 0.8, zbc=N.RLB_ZBC_HALO))
    N.rlb_state_layout(N.make_params(2145386496, 1, 1, 0.8))  # N = 2^31 - 2^21
    p = N.make_params(4, 4, 4, 0.8)
    p.reserved = 1
    with pytest.raises(N.RLBError):
        N.rlb_state_layout(p)
    assert N.rlb_status_str(N.RLB_ERR_UNPHYSICAL) == "RLB_ERR_UNPHYSICAL"


def test_product_does_not_import_the_oracle():
    """The product package never imports the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_0912_2913_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "rlb_oracle" not in src, f


def test_allocation_failure_is_reported(native, monkeypatch):
    """A failing workspace allocation (injected on the host, before any CUDA
    call) comes back as RLB_ERR_OOM with its message; nothing is created."""
    N = native
    monkeypatch.setenv("RLB_INJECT_ALLOC_FAILURE", "1")
    with pytest.raises(N.RLBError) as ei:
        N.rlb_create(N.make_params(16, 8, 4, 0.8), None, None, 0)
    assert ei.value.status == N.RLB_ERR_OOM
    assert "injected allocation failure" in N.rlb_last_error(None)


def test_release_library_refuses_the_bounds_debug_calls(native):
    """The bounds counters exist only in the -DRLB_CHECK_BOUNDS build; the
    release library answers RLB_ERR_STATE without touching the GPU."""
    N = native
    if os.environ.get("RLB_LIBRARY_VARIANT", "release") != "release":
        pytest.skip("the bounds build is loaded")
    for call in (N.rlb_debug_bounds_violations, lambda: N.rlb_debug_bounds_selftest(1, 2)):
        with pytest.raises(N.RLBError) as ei:
            call()
        assert ei.value.status == N.RLB_ERR_STATE
        assert "RLB_CHECK_BOUNDS" in N.rlb_last_error(None)


def test_host_buffers_are_refused_where_device_buffers_are_expected(native):
    """The binding refuses host memory (numpy arrays, CPU tensors) for the
    device arguments, and CUDA tensors for host-side outputs, before any
    library call: no kernel is ever handed a host address."""
    import numpy as np
    import torch

    N = native
    host_np = np.zeros(64)
    host_t = torch.zeros(64, dtype=torch.float64)
    for bad in (host_np, host_t):
        with pytest.raises(ValueError, match="device buffer"):
            N.rlb_step_into(None, bad, bad)
        with pytest.raises(ValueError, match="device buffer"):
            N.rlb_adjoint_step(None, bad, bad, bad, bad, bad)
        with pytest.raises(ValueError, match="device buffer"):
            N.rlb_macro(None, bad, None, None, None, N.RLB_HOST)
        with pytest.raises(ValueError, match="device buffer"):
            N.rlb_init_fields(None, bad, bad, bad, None, N.RLB_DEVICE)
        with pytest.raises(ValueError, match="device buffer"):
            N.rlb_create(N.make_params(8, 4, 4, 0.8), None, bad, 1 << 20)
    assert N._dptr(None) is None and N._dptr(1234) == 1234
    assert N._wptr(host_np, N.RLB_HOST) == host_np.ctypes.data
    assert N._wptr(host_t, N.RLB_HOST) == host_t.data_ptr()
