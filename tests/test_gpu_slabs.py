"""The z-slab decomposition on one GPU (rlb_halo_exchange between slab
contexts) against the whole lattice: the slabs run the same kernels on the
same values, so after any number of steps their planes equal the whole
lattice's bit for bit; and the oracle's whole-lattice run within the parity
tolerances."""
import numpy as np
import pytest
import torch

import workloads as W
from tests._helpers import gpu_run, oracle_run, rel_errors, tiny_workload

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def _same(a, b):
    return all(np.array_equal(x, y, equal_nan=True) for x, y in zip(a, b))


CASES = [
    ("periodic_2", lambda: tiny_workload(12, 7, 9, 0, seed=31), dict(nslabs=2)),
    ("periodic_ragged_3", lambda: tiny_workload(12, 7, 9, 0, seed=32), dict(bounds=[(0, 1), (1, 6), (6, 9)])),
    ("periodic_single", lambda: tiny_workload(10, 6, 5, 0, seed=33), dict(nslabs=1)),
    ("sphere_inflow_4", lambda: W.sphere_3d(nx=60, ny=30, nz=30), dict(nslabs=4)),
    ("outflow_both_3", lambda: tiny_workload(16, 5, 8, 2, seed=34, solid_cells=((6, 2, 3), (7, 2, 4))),
     dict(nslabs=3)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name,make,split", CASES, ids=[c[0] for c in CASES])
def test_slabs_equal_the_whole_lattice(name, make, split, prec):
    from paper_0912_2913_gb300.slabs import SlabLattice

    w = make()
    T = 25
    whole, sim = gpu_run(w, T, prec)
    st_whole = sim.stats()
    sim.close()
    lat = SlabLattice.from_workload(w, prec, device="cuda:0", **split)
    lat.init_fields(w.n, w.eps, w.beta, w.solid).step(T)
    n, e, b, ok = lat.macro()
    st = lat.stats()
    lat.close()
    assert _same((n, e, b), whole), "slab lattice differs from the whole lattice"
    assert st["n_unphysical"] == st_whole["n_unphysical"]
    assert st["n_nonpositive_eq"] == st_whole["n_nonpositive_eq"]
    ref, _ = oracle_run(w, T)
    assert max(rel_errors((n, e, b), ref, w.solid)) <= TOL[prec]


def test_slabs_on_two_streams():
    """Slabs on different streams: the exchange orders itself after the
    work already queued on either stream and before later work there."""
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as Nat
    from paper_0912_2913_gb300.slabs import slab_planes, split_z

    w = tiny_workload(20, 9, 14, 0, seed=35)
    whole, sim = gpu_run(w, 30, "fp64")
    sim.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    slabs = []
    for (z0, z1), s in zip(split_z(w.nz, 2), streams):
        zz = slab_planes(z0, z1, w.nz)
        r = RLB(w.nx, w.ny, z1 - z0 + 2, w.tau, c_l=w.c_l, precision="fp64", device="cuda:0", stream=s, zbc="halo")
        r.init_fields(np.ascontiguousarray(w.n[zz]), np.ascontiguousarray(w.eps[zz]),
                      np.ascontiguousarray(w.beta[:, zz]))
        slabs.append(r)
    for _ in range(30):
        for r in slabs:
            r.step(1)
        Nat.rlb_halo_exchange(slabs[0].ctx, slabs[1].ctx)
        Nat.rlb_halo_exchange(slabs[1].ctx, slabs[0].ctx)
    parts = [r.macro(where="host") for r in slabs]
    got = (np.concatenate([p[0][1:-1] for p in parts]), np.concatenate([p[1][1:-1] for p in parts]),
           np.concatenate([p[2][:, 1:-1] for p in parts], 1))
    for r in slabs:
        r.close()
    assert _same(got, whole)


def test_halo_contexts_refuse_the_adjoint_and_mismatched_slabs():
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as Nat

    w = tiny_workload(8, 5, 6, 0, seed=36)
    a = RLB(8, 5, 5, 0.8, precision="fp64", device="cuda:0", zbc="halo").init_fields(
        w.n[:5], w.eps[:5], w.beta[:, :5])
    b = RLB(9, 5, 5, 0.8, precision="fp64", device="cuda:0", zbc="halo")
    c = RLB(8, 5, 5, 0.8, precision="fp32", device="cuda:0", zbc="halo")
    s = a.state()
    acc = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(Nat.RLBError):
        a.adjoint_step(s, torch.zeros_like(s), torch.zeros_like(s), acc[0:1], acc[1:4])
    for other in (b, c):
        with pytest.raises(Nat.RLBError):
            Nat.rlb_halo_exchange(a.ctx, other.ctx)
    for r in (a, b, c):
        r.close()
