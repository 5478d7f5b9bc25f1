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
