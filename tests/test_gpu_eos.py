"""The general equation of state on the GPU (FP64; an ideal gas with rest
mass, P = (Gamma - 1)(eps - n m), Eqs. equil1/equil2a/equil2b with a Newton
recovery): parity with the oracle (fields to 1e-10, populations to 1e-11,
counters exact), the reduction to the eps = 3P kernels at Gamma = 4/3, m = 0,
and the refusals (FP32 storage, discrete adjoint)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests._helpers import gpu_run, oracle_run, rel_errors, tiny_workload

pytestmark = pytest.mark.gpu

CASES = [
    dict(nx=5, ny=4, nz=3, xbc=0, solid=(), eos=(5 / 3, 0.0), c_l=2.0),
    dict(nx=9, ny=5, nz=4, xbc=1, solid=((4, 2, 1), (5, 2, 1)), eos=(1.2, 0.3), c_l=1.0),
    dict(nx=37, ny=11, nz=5, xbc=1, solid=((10, 5, 2), (11, 5, 2)), eos=(1.2, 0.3), c_l=1.0),
    dict(nx=12, ny=1, nz=1, xbc=2, solid=(), eos=(1.25, 0.0), c_l=1.0),
]
IDS = ["periodic_c2", "inflow_solid", "ragged", "outflow_both"]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _eos_workload(case, seed=3):
    w = tiny_workload(case["nx"], case["ny"], case["nz"], case["xbc"], seed=seed, c_l=case["c_l"],
                      solid_cells=case["solid"])
    w.eos, (w.eos_gamma, w.eos_mass) = 1, case["eos"]
    return w


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_general_eos_parity(case):
    w = _eos_workload(case)
    steps = 40
    stats = oracle.Stats()
    ref, st_ref = oracle_run(w, steps, stats)
    got, sim = gpu_run(w, steps, "fp64")
    assert max(rel_errors(got, ref, w.solid)) <= 1e-10
    s = sim.stats()
    assert s["n_unphysical"] == stats.n_unphysical == 0
    assert s["n_nonpositive_eq"] == stats.n_nonpositive_eq
    cells = sim.state_to_cells(sim.state()).cpu().numpy()
    fluid = np.ones(cells.shape[:3], bool) if w.solid is None else w.solid == 0
    d = np.abs(cells - st_ref)[fluid]
    assert np.max(d / np.maximum(np.abs(st_ref[fluid]), 1e-300)) < 1e-11
    sim.close()


def test_general_eos_shock_tube_and_sphere():
    """A 1:4 pressure jump in a Gamma = 1.2, m = 0.3 gas (1600 cells, 1000
    steps) and the reduced sphere (60 x 30 x 30, 200 steps, Gamma = 1.2,
    m = 0.3) against the oracle."""
    tube = W.shock_tube_1d(steps=1000, eps_r=0.25, n_r=0.5)
    tube.eos, tube.eos_gamma, tube.eos_mass = 1, 1.2, 0.3
    sph = W.sphere_3d(nx=60, ny=30, nz=30, steps=200)
    sph.eos, sph.eos_gamma, sph.eos_mass = 1, 1.2, 0.3
    for w in (tube, sph):
        stats = oracle.Stats()
        ref, _ = oracle_run(w, w.steps, stats)
        got, sim = gpu_run(w, w.steps, "fp64")
        assert stats.n_unphysical == 0 and sim.stats()["n_unphysical"] == 0
        assert max(rel_errors(got, ref, w.solid)) <= 1e-10
        sim.close()


def test_gamma_four_thirds_massless_is_the_eps3p_scheme():
    """The general kernels at Gamma = 4/3, m = 0 against the eps = 3P kernels
    on the same lattice: 50 steps agree to 1e-12."""
    w = tiny_workload(37, 11, 5, 1, seed=9, solid_cells=((10, 5, 2),))
    a, sa = gpu_run(w, 50, "fp64")
    w.eos, w.eos_gamma, w.eos_mass = 1, 4.0 / 3.0, 0.0
    b, sb = gpu_run(w, 50, "fp64")
    assert max(rel_errors(b, a, w.solid)) <= 1e-12
    sa.close()
    sb.close()


def test_general_eos_refusals():
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as N

    with pytest.raises(N.RLBError) as ei:
        RLB(8, 4, 4, 0.8, precision="fp32", eos="gamma_law", eos_gamma=1.5)
    assert ei.value.status == N.RLB_ERR_ARG
    w = _eos_workload(CASES[0])
    got, sim = gpu_run(w, 2, "fp64")
    lam = sim.new_state()
    acc = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(N.RLBError) as ei:
        sim.adjoint_step(sim.state(), lam, sim.new_state(), acc[0:1], acc[1:4])
    assert ei.value.status == N.RLB_ERR_ARG
    sim.close()
