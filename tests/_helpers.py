"""Helpers shared by the test files: error metrics and oracle/GPU runners."""
import numpy as np

import oracle
import workloads as W


def rel_errors(gpu, ref, solid=None):
    """Max relative error of n and eps and the scaled max error of beta:
    |beta_gpu - beta_ref|_inf / max(max |beta_ref|, 1e-3) (beta passes
    through zero).  Solid cells are excluded."""
    n, e, b = gpu
    n0, e0, b0 = ref
    m = np.ones(n0.shape, bool) if solid is None else (solid == 0)
    en = float(np.max(np.abs(n - n0)[m] / np.abs(n0)[m]))
    ee = float(np.max(np.abs(e - e0)[m] / np.abs(e0)[m]))
    bs = max(float(np.max(np.abs(b0[:, m]))), 1e-3)
    eb = float(np.max(np.abs(b - b0)[:, m]) / bs)
    return en, ee, eb


def oracle_run(w, steps, stats=None):
    p = oracle.Params(**w.params())
    st = oracle.init(p, w.n, w.eps, w.beta, w.solid)
    if steps:
        oracle.run(p, st, steps, solid=w.solid, stats=stats)
    n, e, b, bad = oracle.macro(p, st, w.solid)
    return (n, e, b), st


def gpu_run(w, steps, precision, device="cuda:0", **kw):
    from paper_0912_2913_gb300 import RLB

    sim = RLB.from_workload(w, precision, device=device, **kw)
    sim.init_fields(w.n, w.eps, w.beta, w.solid)
    if steps:
        sim.step(steps)
    n, e, b, ok = sim.macro(where="host")
    return (n, e, b), sim


def tiny_workload(nx, ny, nz, xbc, seed, tau=0.8, c_l=1.0, solid_cells=(), beta_in=(0.3, 0.05, -0.02), bmax=0.3):
    n, eps, beta = W.smooth_random_fields(nx, ny, nz, seed, bmax=bmax)
    solid = None
    if solid_cells:
        solid = np.zeros((nz, ny, nx), np.uint8)
        for (x, y, z) in solid_cells:
            solid[z, y, x] = 1
    return W.Workload("tiny", nx, ny, nz, tau, c_l, xbc, 0, n, eps, beta, solid, n_in=0.9, eps_in=1.2,
                      beta_in=beta_in)


def light_cone_cells(w, m, seed):
    """m seeded (z, y, x) cells of a lattice, the eight corners first (their
    neighbourhoods wrap across every periodic face)."""
    rng = np.random.default_rng(seed)
    corners = [(z, y, x) for z in (0, w.nz - 1) for y in (0, w.ny - 1) for x in (0, w.nx - 1)]
    rest = [(int(rng.integers(w.nz)), int(rng.integers(w.ny)), int(rng.integers(w.nx)))
            for _ in range(max(0, m - len(corners)))]
    return corners + rest


def light_cone_oracle(w, steps, cells):
    """Oracle n, eps (m values) and beta (3, m) after `steps` steps at the
    given (z, y, x) cells of a periodic lattice without solid cells, each
    computed on the (2 steps + 1)^3 neighbourhood of the cell (periodic wrap)
    alone.  After k steps a cell depends only on the cells within k cells of
    it along each axis, because every D3Q19 velocity moves at most one cell
    per axis per step; the values that wrap across the neighbourhood's own
    faces reach the centre only after k + 1 steps."""
    assert w.xbc == 0 and w.solid is None
    k = int(steps)
    r = np.arange(-k, k + 1)
    side = 2 * k + 1
    p = oracle.Params(**{**w.params(), "nx": side, "ny": side, "nz": side})
    out_n, out_e, out_b = [], [], []
    for (z, y, x) in cells:
        iz, iy, ix = (z + r) % w.nz, (y + r) % w.ny, (x + r) % w.nx
        sub = lambda a: np.ascontiguousarray(a[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]])
        st = oracle.init(p, sub(w.n), sub(w.eps), sub(w.beta))
        if k:
            oracle.run(p, st, k)
        n, e, b, _ = oracle.macro(p, st)
        out_n.append(n[k, k, k])
        out_e.append(e[k, k, k])
        out_b.append(b[:, k, k, k])
    return np.array(out_n), np.array(out_e), np.array(out_b).T
