"""The FP64 step with its arithmetic in compensated binary32 pairs
(RLB_F64_ARITH=df; binary64 storage, binary64 recovery root): held to the
oracle at the FP64 tolerance 1e-10 on the forward parity cases and to the
all-FP64 GPU step closely, through the C ABI."""
import numpy as np
import pytest
import torch

import workloads as W
from tests._helpers import gpu_run, oracle_run, rel_errors, tiny_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _df_run(w, steps, monkeypatch):
    monkeypatch.setenv("RLB_F64_ARITH", "df")
    got, sim = gpu_run(w, steps, "fp64")
    st = sim.stats()
    sim.close()
    monkeypatch.delenv("RLB_F64_ARITH")
    return got, st


CASES = [
    ("periodic", lambda: tiny_workload(9, 7, 5, 0, seed=41), 40),
    ("solid", lambda: tiny_workload(10, 8, 6, 0, seed=42, solid_cells=((4, 3, 2), (5, 3, 2))), 40),
    ("inflow_ragged", lambda: tiny_workload(37, 11, 5, 1, seed=43, solid_cells=((12, 4, 2), (13, 4, 2))), 60),
    ("outflow_both", lambda: tiny_workload(20, 3, 4, 2, seed=44), 60),
    ("sphere_60", lambda: W.sphere_3d(nx=60, ny=30, nz=30), 500),
    ("shock_tube", lambda: W.shock_tube_1d(), 2000),
]


@pytest.mark.parametrize("name,make,steps", CASES, ids=[c[0] for c in CASES])
def test_f64df_matches_the_oracle(name, make, steps, monkeypatch):
    w = make()
    ostats = __import__("oracle").Stats()
    ref, _ = oracle_run(w, steps, ostats)
    got, st = _df_run(w, steps, monkeypatch)
    assert st["n_unphysical"] == ostats.n_unphysical
    assert max(rel_errors(got, ref, w.solid)) <= 1e-10
    plain, sim = gpu_run(w, steps, "fp64")
    sim.close()
    assert max(rel_errors(got, plain, w.solid)) <= 1e-11


def test_f64df_strong_shock_at_c_l_10(monkeypatch):
    """The 1:16 strong shock at c_l = 10, tau = 0.52, 4000 steps (the case
    that amplifies rounding most)."""
    w = W.riemann_tube(1 / 3, 1 / 48, 1 / 3, 1 / 6, cells=1598, tau=0.52, c_l=10.0, steps=4000)
    ref, _ = oracle_run(w, w.steps)
    got, st = _df_run(w, w.steps, monkeypatch)
    assert st["n_unphysical"] == 0
    assert max(rel_errors(got, ref)) <= 1e-10
