"""rlb_adjoint_step_noalloc (the allocation-free adjoint step) against
rlb_adjoint_step, through the C ABI: two calls in a row of each on the same
inputs, lambda_t and both accumulated sums compared after every call (the
two entry points run the same kernels on the same grids, so bit for bit).

Kept in its own file, collected last, so that it also runs after everything
else has used the library in this process."""
import numpy as np
import pytest
import torch

from tests._helpers import tiny_workload

pytestmark = pytest.mark.gpu

# FP64 to 1e-10, FP32 deviations to 1e-4 (relative to the largest |value|),
# the tolerances of the adjoint parity tests.
TOL = {"fp64": 1e-10, "fp32": 1e-4}

CASES = [
    # ragged: fewer cells than one persistent grid, inflow/outflow, solids
    dict(nx=37, ny=9, nz=5, xbc=1, solid=((12, 4, 2), (13, 4, 2), (12, 5, 2))),
    # more cells than the persistent grid covers in one sweep (grid-stride)
    dict(nx=160, ny=48, nz=40, xbc=0, solid=((80, 20, 20), (81, 20, 20))),
    dict(nx=130, ny=33, nz=29, xbc=2, solid=()),
]
IDS = ["ragged_inflow", "periodic_strided", "outflow_both"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@pytest.fixture(scope="module", autouse=True)
def _setup_call(_need_gpu):
    """The entry point's documented set-up: its first call on the device (here
    on a small FP64 periodic lattice) takes the scratch array's address and
    loads every kernel it launches.  After it, no call of any precision or x
    boundary may change the device's free memory."""
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as N

    w = tiny_workload(6, 5, 4, 0, seed=2)
    sim = RLB.from_workload(w, "fp64", device="cuda:0").init_fields(w.n, w.eps, w.beta)
    s = sim.state()
    li, lo = torch.zeros_like(s), torch.zeros_like(s)
    acc = torch.zeros(4, dtype=torch.float64, device="cuda")
    N.rlb_adjoint_step_noalloc(sim.ctx, s, li, lo, acc[0:1], acc[1:4])
    sim.sync()
    sim.close()


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_noalloc_adjoint_step_matches_adjoint_step(case, prec):
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as N

    w = tiny_workload(case["nx"], case["ny"], case["nz"], case["xbc"], seed=11, solid_cells=case["solid"])
    sim = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid)
    sim.step(3)
    state = sim.state().clone()
    fluid = torch.from_numpy(np.ones((w.nz, w.ny, w.nx), bool) if w.solid is None else w.solid == 0).cuda()
    g = torch.Generator(device="cpu").manual_seed(3)
    shp = (w.nz, w.ny, w.nx)
    dn = (torch.randn(shp, generator=g, dtype=torch.float64).cuda()) * fluid
    de = (torch.randn(shp, generator=g, dtype=torch.float64).cuda()) * fluid
    db = (torch.randn((3,) + shp, generator=g, dtype=torch.float64).cuda()) * fluid
    lam = sim.new_state()
    sim.adjoint_macro(state, dn, de, db, lam)

    acc_a = torch.zeros(4, dtype=torch.float64, device="cuda")
    acc_b = torch.zeros(4, dtype=torch.float64, device="cuda")
    la_in, la_out = lam.clone(), torch.zeros_like(lam)
    lb_in, lb_out = lam.clone(), torch.zeros_like(lam)
    n = sim.N  # planes hold N cells, then padding that no kernel touches
    for call in range(2):
        N.rlb_adjoint_step(sim.ctx, state, la_in, la_out, acc_a[0:1], acc_a[1:4])
        torch.cuda.synchronize()
        # after the set-up call, no call allocates: also not the first one of
        # this precision and x boundary (no kernel is loaded on demand)
        free_before = torch.cuda.mem_get_info()[0]
        N.rlb_adjoint_step_noalloc(sim.ctx, state, lb_in, lb_out, acc_b[0:1], acc_b[1:4])
        sim.sync()
        assert torch.cuda.mem_get_info()[0] == free_before, f"device memory changed across call {call + 1}"
        assert torch.isfinite(lb_out[:, :n]).all()
        assert _rel(lb_out[:, :n], la_out[:, :n]) <= TOL[prec], f"lambda_t differs after call {call + 1}"
        assert abs(acc_b[0].item() - acc_a[0].item()) <= TOL[prec] * max(abs(acc_a[0].item()), 1e-30)
        if case["xbc"] == 1:
            assert acc_a[1:4].abs().max().item() > 0
            assert _rel(acc_b[1:4], acc_a[1:4]) <= TOL[prec]
        else:
            assert acc_b[1:4].abs().max().item() == 0
        ints = torch.int64 if prec == "fp64" else torch.int32
        assert torch.equal(lb_out[:, :n].contiguous().view(ints), la_out[:, :n].contiguous().view(ints))
        assert torch.equal(acc_b.view(torch.int64), acc_a.view(torch.int64))
        la_in, la_out = la_out, la_in
        lb_in, lb_out = lb_out, lb_in
    st = N.rlb_stats(sim.ctx)
    assert st["steps"] == 3
    sim.close()
