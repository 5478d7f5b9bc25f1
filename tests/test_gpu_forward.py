"""Parity of the CUDA forward path (through the C ABI) with the FP64 oracle.

FP64 path: max relative error of n, eps, beta <= 1e-10; FP32 deviation path:
<= 1e-4, after the stated step counts.  Population-level comparisons on tiny
grids, statistics counters compared exactly.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from tests._helpers import gpu_run, light_cone_cells, light_cone_oracle, oracle_run, rel_errors, tiny_workload

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-4}
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

TINY = [
    dict(nx=1, ny=1, nz=1, xbc=0, solid=()),
    dict(nx=2, ny=3, nz=4, xbc=0, solid=()),
    dict(nx=3, ny=3, nz=3, xbc=0, solid=((1, 1, 1),)),
    dict(nx=5, ny=4, nz=3, xbc=0, solid=((2, 1, 1), (3, 1, 1))),
    dict(nx=7, ny=5, nz=3, xbc=1, solid=((3, 2, 1),)),
    dict(nx=3, ny=2, nz=2, xbc=1, solid=()),
    dict(nx=9, ny=1, nz=1, xbc=2, solid=()),
    dict(nx=37, ny=11, nz=5, xbc=0, solid=((10, 5, 2), (11, 5, 2), (10, 6, 2))),  # spans blocks, ragged tail
]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", TINY, ids=[f"{c['nx']}x{c['ny']}x{c['nz']}_bc{c['xbc']}" for c in TINY])
def test_tiny_grids_populations_and_stats(case, prec):
    w = tiny_workload(case["nx"], case["ny"], case["nz"], case["xbc"], seed=7, solid_cells=case["solid"])
    steps = 12
    stats = oracle.Stats()
    ref, st_ref = oracle_run(w, steps, stats)
    got, sim = gpu_run(w, steps, prec)
    en, ee, eb = rel_errors(got, ref, w.solid)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    s = sim.stats()
    assert s["steps"] == steps
    assert s["n_unphysical"] == stats.n_unphysical == 0
    assert s["n_nonpositive_eq"] == stats.n_nonpositive_eq
    if prec == "fp64":
        # population-level parity (oracle layout is cell-major)
        cells = sim.state_to_cells(sim.state()).cpu().numpy()
        fluid = np.ones(cells.shape[:3], bool) if w.solid is None else w.solid == 0
        d = np.abs(cells - st_ref)[fluid]
        assert np.max(d / np.maximum(np.abs(st_ref[fluid]), 1e-300)) < 1e-11
        if w.solid is not None:
            marker = cells[w.solid == 1]
            assert np.all(np.isnan(marker))
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shock_tube_1600_2000_steps(prec):
    """The 1D shock tube: 1600 x 1 x 1, tau 0.9, 2000 steps, outflow ghosts."""
    w = W.shock_tube_1d()
    stats = oracle.Stats()
    ref, _ = oracle_run(w, w.steps, stats)
    got, sim = gpu_run(w, w.steps, prec)
    en, ee, eb = rel_errors(got, ref)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    s = sim.stats()
    assert s["n_unphysical"] == stats.n_unphysical
    if prec == "fp64":
        assert s["n_nonpositive_eq"] == stats.n_nonpositive_eq
    else:  # binary32 populations shift beta in the last bits; the count may differ near the bound
        assert abs(s["n_nonpositive_eq"] - stats.n_nonpositive_eq) <= 1e-4 * stats.n_nonpositive_eq
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_reduced_500_steps(prec):
    """The sphere workload at 60 x 30 x 30 (sphere scaled with the box), 500 steps."""
    w = W.sphere_3d(nx=60, ny=30, nz=30)
    ref, _ = oracle_run(w, 500)
    got, sim = gpu_run(w, 500, prec)
    en, ee, eb = rel_errors(got, ref, w.solid)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_full_size_short(prec):
    """Full 200 x 100 x 100 sphere lattice, 10 steps, every cell compared."""
    w = W.sphere_3d()
    stats = oracle.Stats()
    ref, _ = oracle_run(w, 10, stats)
    got, sim = gpu_run(w, 10, prec)
    en, ee, eb = rel_errors(got, ref, w.solid)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    s = sim.stats()
    if prec == "fp64":
        assert s["n_nonpositive_eq"] == stats.n_nonpositive_eq
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_full_size_5000_steps_sampled(prec):
    """Full-size sphere run to 5000 steps against the stored oracle samples."""
    path = os.path.join(GOLDEN, "sphere_fp64_5000.json")
    if not os.path.exists(path):
        pytest.skip("sampled oracle reference not generated")
    with open(path) as fh:
        g = json.load(fh)
    w = W.sphere_3d(steps=g["steps"])
    got, sim = gpu_run(w, g["steps"], prec)
    cells = np.array(g["cells"])
    n = got[0].reshape(-1)[cells]
    e = got[1].reshape(-1)[cells]
    b = np.stack([got[2][a].reshape(-1)[cells] for a in range(3)])
    ref = (np.array(g["n"]), np.array(g["eps"]), np.array(g["beta"]))
    en, ee, eb = rel_errors((n, e, b), ref)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    s = sim.stats()
    assert s["n_unphysical"] == g["stats"]["n_unphysical"]
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sphere_as_written_breaks_down_identically(prec):
    """The sphere with the 10:1 energy jump against the inflow (interior eps =
    0.1) leaves the scheme's range: oracle and GPU agree on the fields before
    the breakdown and flag the same first unphysical update (FP64).  After it
    the fields are non-finite and the counts are not comparable."""
    w = W.sphere_3d(nx=60, ny=30, nz=30, eps_int=0.1)
    before = 10
    ref, _ = oracle_run(w, before)
    got, sim = gpu_run(w, before, prec)
    en, ee, eb = rel_errors(got, ref, w.solid)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    sim.close()
    stats = oracle.Stats()
    ref, _ = oracle_run(w, 60, stats)
    got, sim = gpu_run(w, 60, prec)
    s = sim.stats()
    assert stats.first_bad >= 0 and s["first_bad"] >= 0 and s["n_unphysical"] > 0
    if prec == "fp64":
        assert s["first_bad"] == stats.first_bad
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_random_box_64(prec):
    """Periodic box with the Gaussian-random-field recipe (sigma = 8) at 64^3, 200 steps."""
    w = W.random_box(L=64, steps=200)
    ref, _ = oracle_run(w, 200)
    got, sim = gpu_run(w, 200, prec)
    en, ee, eb = rel_errors(got, ref)
    assert max(en, ee, eb) <= TOL[prec], (en, ee, eb)
    sim.close()


@pytest.mark.slow
def test_random_box_512_fp32_against_fp64_subsample():
    """The 512^3 periodic box (tau 0.7, 1000 steps): the FP32 deviation path
    against the FP64 GPU path on the 64^3 lattice of points with x, y, z = 0
    (mod 8), within the FP32 bound.  The reference is the FP64 GPU run (held
    to the oracle at 1e-10 by the other tests, in full at 64^3 with the same
    field recipe); the FP64 oracle itself would need about two hours of host
    time at 512^3."""
    from paper_0912_2913_gb300 import RLB

    w = W.random_box(L=512, steps=1000)
    e_vel = torch.tensor(oracle.lattice()[0], dtype=torch.float64, device="cuda:0")

    def totals(sim):
        """Lattice totals of n gamma, T^00 and T^0i (planes summed in float64;
        FP32 deviations summed as stored: the reference is uniform)."""
        st = sim.state()[:, :sim.N]
        per_plane = torch.stack([st[q].double().sum() for q in range(38)])
        return torch.cat([per_plane[:19].sum()[None], per_plane[19:].sum()[None],
                          w.c_l * (per_plane[19:, None] * e_vel).sum(0)]).cpu().numpy()

    def run(prec):
        sim = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta)
        t0 = totals(sim)
        sim.step(1000)
        t1 = totals(sim)
        n, e, b, _ = sim.macro()
        out = tuple(a[..., ::8, ::8, ::8].double().cpu().numpy() for a in (n, e, b))
        st = sim.stats()
        sim.close()
        del sim, n, e, b
        torch.cuda.empty_cache()
        return out, st, t0, t1

    ref, st64, a0, a1 = run("fp64")
    got, st32, b0, b1 = run("fp32")
    assert ref[0].shape == (64, 64, 64)
    assert st64["n_unphysical"] == 0 and st32["n_unphysical"] == 0
    en, ee, eb = rel_errors(got, ref)
    assert max(en, ee, eb) <= TOL["fp32"], (en, ee, eb)
    # at full size: number, energy and momentum totals conserved over 1000
    # steps: FP64 to round-off of the sums; the FP32 deviations drift by their
    # binary32 rounding, measured 1.3e-6 of the totals of the full populations
    # after 1000 steps (about 1e-9 per step): bound 1e-5
    scale = np.abs(a0[:2]).max()
    assert np.all(np.abs(a1 - a0) <= 1e-12 * scale), (a0, a1)
    assert np.all(np.abs(b1 - b0) <= 1e-5 * scale), (b0, b1)


@pytest.mark.slow
def test_random_box_512_against_the_oracle_on_light_cones():
    """At full size, against the oracle itself: 12 steps of the 512^3 box on
    the GPU (FP64 and FP32, contexts made as the benchmark makes them) and,
    at 48 seeded cells (the eight corners among them), the oracle's values
    computed on each cell's 25^3 neighbourhood alone, which equal the
    whole-lattice oracle bit for bit (tests/test_light_cone.py)."""
    from paper_0912_2913_gb300 import RLB

    k = 12
    w = W.random_box(L=512, steps=k)
    cells = light_cone_cells(w, 48, seed=512)
    ref = light_cone_oracle(w, k, cells)
    zs, ys, xs = (torch.tensor(c, dtype=torch.long, device="cuda:0") for c in zip(*cells))
    for prec in ("fp64", "fp32"):
        sim = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta)
        sim.step(k)
        n, e, b, ok = sim.macro()
        got = (n[zs, ys, xs].cpu().numpy(), e[zs, ys, xs].cpu().numpy(), b[:, zs, ys, xs].cpu().numpy())
        st = sim.stats()
        sim.close()
        del sim, n, e, b
        torch.cuda.empty_cache()
        assert ok and st["n_unphysical"] == 0
        en, ee, eb = rel_errors(got, ref)
        assert max(en, ee, eb) <= TOL[prec], (prec, en, ee, eb)


def test_tachyon_lattice_speed():
    """c_l = 10 (numerical tachyons) with beta up to 0.6 in a periodic box."""
    w = tiny_workload(16, 8, 6, 0, seed=3, c_l=10.0, bmax=0.6)
    for prec in ("fp64", "fp32"):
        stats = oracle.Stats()
        ref, _ = oracle_run(w, 50, stats)
        got, sim = gpu_run(w, 50, prec)
        en, ee, eb = rel_errors(got, ref)
        assert max(en, ee, eb) <= TOL[prec], (prec, en, ee, eb)
        sim.close()


@pytest.mark.parametrize("shape", [(60, 30, 30, 1), (64, 16, 12, 0), (200, 100, 100, 1), (16, 5, 7, 2)])
def test_tma_staged_step_equals_plain_step(shape, monkeypatch):
    """The TMA-staged FP32 step and the launch variants of the one-cell-per-
    thread FP32 step do the same arithmetic: states agree bit for bit after
    several steps (tiles that wrap in y, ghost planes, solid cells)."""
    nx, ny, nz, xbc = shape
    if xbc == 1:
        w = W.sphere_3d(nx=nx, ny=ny, nz=nz)
    else:
        w = tiny_workload(nx, ny, nz, xbc, seed=13)
    from paper_0912_2913_gb300 import RLB

    states = []
    for tma, var, minb in (("1", "0", "2"), ("1", "0", "3"), ("0", "0", "2"), ("0", "1", "2"), ("0", "2", "2"),
                           ("0", "3", "2"), ("0", "4", "2"), ("0", "5", "2"), ("0", "6", "2"), ("0", "7", "2"),
                           ("0", "8", "2")):
        monkeypatch.setenv("RLB_TMA", tma)
        monkeypatch.setenv("RLB_F32_VARIANT", var)
        monkeypatch.setenv("RLB_TMA_MINB", minb)
        sim = RLB.from_workload(w, "fp32", device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid).step(7)
        torch.cuda.synchronize()
        states.append((sim.state()[:, :sim.N].clone(), sim.stats()))
        sim.close()
    for st, stats in states[1:]:
        assert torch.equal(states[0][0].view(torch.int32), st.view(torch.int32))
        assert states[0][1] == stats


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cuda_graph_of_steps_matches_stream_steps(prec):
    """rlb_step captured in a CUDA graph (an even number of steps, so the
    ping-pong buffers return to their places) and replayed gives the state of
    the same number of steps issued on the stream, bit for bit."""
    from paper_0912_2913_gb300 import RLB

    w = W.shock_tube_1d()
    ref = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta)
    ref.step(2).step(200)
    s = torch.cuda.Stream()
    sim = RLB.from_workload(w, prec, device="cuda:0", stream=s).init_fields(w.n, w.eps, w.beta)
    sim.step(2)  # the first FP32 step times its launch variants: not in a capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        sim.step(100)
    with torch.cuda.stream(s):
        g.replay()
        g.replay()
    torch.cuda.synchronize()
    a, b = ref.state()[:, :w.N].clone(), sim.state()[:, :w.N].clone()
    iv = torch.int64 if prec == "fp64" else torch.int32
    assert torch.equal(a.view(iv), b.view(iv))
    ref.close()
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_file_resume(prec, tmp_path):
    """save() after 20 steps, load() into a fresh context and 15 more steps
    give the state of 35 uninterrupted steps, bit for bit; a file written with
    other parameters is refused."""
    from paper_0912_2913_gb300 import RLB

    w = W.sphere_3d(nx=40, ny=20, nz=18)
    a = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid).step(20)
    path = str(tmp_path / "state.rlb")
    a.save(path)
    a.step(15)
    b = RLB.from_workload(w, prec, device="cuda:0").load(path).step(15)
    iv = torch.int64 if prec == "fp64" else torch.int32
    assert torch.equal(a.state()[:, :a.N].view(iv), b.state()[:, :b.N].view(iv))
    w2 = W.sphere_3d(nx=40, ny=20, nz=18, tau=0.9)
    c = RLB.from_workload(w2, prec, device="cuda:0")
    with pytest.raises(ValueError):
        c.load(path)
    for s in (a, b, c):
        s.close()


def test_step_into_matches_step():
    w = tiny_workload(12, 6, 5, 1, seed=5, solid_cells=((5, 3, 2),))
    from paper_0912_2913_gb300 import RLB

    sim = RLB.from_workload(w, "fp64", device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid)
    a = sim.state().clone()
    b = torch.full_like(a, float("nan"))
    sim.step_into(a, b)
    sim.step(1)
    torch.cuda.synchronize()
    # bitwise (the solid markers are NaN payloads)
    assert torch.equal(sim.state()[:, :sim.N].view(torch.int64), b[:, :sim.N].view(torch.int64))
    sim.close()


def test_device_and_host_init_agree():
    w = W.sphere_3d(nx=30, ny=16, nz=14)
    from paper_0912_2913_gb300 import RLB

    s1 = RLB.from_workload(w, "fp32", device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid)
    dev = lambda a, dt=torch.float64: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0", dt)
    s2 = RLB.from_workload(w, "fp32", device="cuda:0").init_fields(dev(w.n), dev(w.eps), dev(w.beta),
                                                                   dev(w.solid, torch.uint8))
    torch.cuda.synchronize()
    x1, x2 = s1.state()[:, :s1.N], s2.state()[:, :s2.N]
    assert torch.equal(x1.isnan(), x2.isnan())
    assert torch.equal(torch.nan_to_num(x1), torch.nan_to_num(x2))
    s1.close()
    s2.close()


def test_errors_are_status_codes():
    from paper_0912_2913_gb300 import RLB, RLBError
    from paper_0912_2913_gb300 import _native as N

    w = W.sphere_3d(nx=30, ny=16, nz=14)
    bad = w.solid.copy()
    bad[7, 8, 1] = 1  # solid next to the inflow ghost plane
    sim = RLB.from_workload(w, "fp64", device="cuda:0")
    with pytest.raises(RLBError) as ei:
        sim.init_fields(w.n, w.eps, w.beta, bad)
    assert ei.value.status == N.RLB_ERR_ARG
    with pytest.raises(RLBError) as ei:
        N.rlb_step(sim.ctx, 1)  # not initialised
    assert ei.value.status == N.RLB_ERR_STATE
    dev_bad = torch.from_numpy(bad).to("cuda:0")
    with pytest.raises(RLBError):
        sim.init_fields(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w.n, w.eps, w.beta)), dev_bad)
    sim.init_fields(w.n, w.eps, w.beta, w.solid).step(2)
    assert sim.stats()["steps"] == 2
    before = sim.state().clone()
    sim.step(0)  # an empty step request is a no-op
    assert sim.stats()["steps"] == 2 and torch.equal(before.view(torch.int64), sim.state().view(torch.int64))
    with pytest.raises(RLBError) as ei:
        N.rlb_step(sim.ctx, -1)
    assert ei.value.status == N.RLB_ERR_ARG
    st = sim.new_state()
    with pytest.raises(RLBError) as ei:
        N.rlb_step_into(sim.ctx, st, st)  # src and dst must differ
    assert ei.value.status == N.RLB_ERR_ARG
    with pytest.raises(RLBError) as ei:
        N.rlb_step(None, 1)
    assert ei.value.status == N.RLB_ERR_ARG
    assert sim.stats()["steps"] == 2  # the refused calls changed nothing
    sim.close()


def test_unphysical_cells_are_counted_not_fatal():
    """A state with T^00 < 0 somewhere: the run continues, the cells are
    counted and rlb_macro reports RLB_ERR_UNPHYSICAL."""
    w = tiny_workload(6, 4, 3, 0, seed=9)
    from paper_0912_2913_gb300 import RLB

    sim = RLB.from_workload(w, "fp64", device="cuda:0").init_fields(w.n, w.eps, w.beta)
    st = sim.state()
    st[19 + 0, 5] = -50.0  # T^00 < 0 in one cell
    sim.step(1)
    n, e, b, ok = sim.macro()
    s = sim.stats()
    assert s["n_unphysical"] >= 1 and s["first_bad"] >= 0
    assert not ok
    p = oracle.Params(**w.params())
    ref = oracle.init(p, w.n, w.eps, w.beta)
    ref.reshape(-1, 38)[5, 19 + 0] = -50.0
    os_ = oracle.Stats()
    oracle.run(p, ref, 1, stats=os_)
    assert s["n_unphysical"] == os_.n_unphysical and s["first_bad"] == os_.first_bad
    sim.close()


@pytest.mark.parametrize("scale", [1e-30, 1e30])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fields_scaled_far_outside_binary32_squares(scale, prec):
    """The scheme is homogeneous of degree one in (f, g): scaling n and eps by
    s scales every population, n and eps by s and leaves beta unchanged.  At
    s = 1e-30 and 1e+30 the recovery's discriminant (~ s^2) lies far outside
    the binary32 range that the FP64 path's Newton seeds come from; the shock
    tube, 300 steps, still matches the oracle on the same scaled inputs (FP64
    1e-10, FP32 1e-4) and the unscaled GPU run divided by s."""
    w = W.shock_tube_1d(steps=300)
    ws = W.Workload(**{**w.__dict__, "n": w.n * scale, "eps": w.eps * scale})
    ref, _ = oracle_run(ws, 300)
    got, sim = gpu_run(ws, 300, prec)
    st = sim.stats()
    sim.close()
    assert st["n_unphysical"] == 0
    assert max(rel_errors(got, ref)) <= TOL[prec]
    base, sim = gpu_run(w, 300, prec)
    sim.close()
    n, e, b = got
    n0, e0, b0 = base
    tol = 1e-11 if prec == "fp64" else TOL[prec]
    assert max(rel_errors((n / scale, e / scale, b), (n0, e0, b0))) <= tol


@pytest.mark.parametrize("name,make", [
    ("shock_tube", lambda: W.shock_tube_1d()),
    ("inflow_solid", lambda: tiny_workload(37, 9, 5, 1, seed=41, solid_cells=((12, 4, 2), (13, 4, 2), (12, 5, 2)))),
    ("outflow_both_nx3", lambda: tiny_workload(3, 4, 5, 2, seed=42)),
    ("periodic_ragged", lambda: tiny_workload(13, 7, 11, 0, seed=43)),
    ("sphere_60", lambda: W.sphere_3d(nx=60, ny=30, nz=30)),
], ids=lambda v: v if isinstance(v, str) else "")
def test_fp64_split_step_equals_the_one_thread_step(name, make, monkeypatch):
    """The FP64 step with eight lanes per cell (k_step_f64_split, the small
    lattices' kernel) does the one-thread kernel's arithmetic term for term
    (the moments summed in the same tree), so both give the same values and
    statistics; RLB_F64_SPLIT forces either kernel on any lattice."""
    w = make()
    runs = []
    for force in ("0", "1"):
        monkeypatch.setenv("RLB_F64_SPLIT", force)
        (n, e, b), sim = gpu_run(w, 40, "fp64")
        state = sim.state()[:, :sim.N].clone()
        runs.append(((n, e, b), state, sim.stats()))
        sim.close()
    (m0, s0, st0), (m1, s1, st1) = runs
    for a, c in zip(m0, m1):
        assert np.array_equal(a, c, equal_nan=True)
    assert torch.equal(s0.isnan(), s1.isnan())
    assert torch.equal(torch.nan_to_num(s0), torch.nan_to_num(s1))
    assert st0 == st1
