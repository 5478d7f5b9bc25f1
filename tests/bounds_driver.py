"""The parity cases run through the bounds-checking debug build of librlb.

Run as a program of its own by ``tests/test_gpu_bounds.py`` with
``RLB_LIBRARY_VARIANT=bounds`` in the environment (the variant is chosen when
the library loads, so it cannot share a process with the release library).
Every forward launch variant, the adjoint kernels, the general-EOS kernels
and the autograd path run on small lattices (periodic, solid cells, inflow,
outflow at both ends, a ragged 37 x 9 x 5 lattice, the reduced sphere); after
each group the driver reads the count of out-of-range state indices.  It
prints one JSON line: the counts per group, the parity errors against the
oracle, and the checker's own self-test.
"""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402
from tests._helpers import gpu_run, oracle_run, rel_errors, tiny_workload  # noqa: E402

CASES = [(5, 4, 3, 0, ()), (6, 5, 4, 0, ((3, 2, 2),)), (9, 5, 4, 1, ((4, 2, 1), (5, 2, 1))), (8, 1, 1, 2, ()),
         (37, 9, 5, 1, ((12, 4, 2), (13, 4, 2), (12, 5, 2)))]
# (RLB_TMA, RLB_F32_VARIANT): the TMA-staged step only on lattices whose rows
# it takes (nx a multiple of 4), as in its own parity test
F32_VARIANTS = [("0", v) for v in "012345"]
TMA_SHAPES = {(16, 5, 7), (60, 30, 30)}


def _set_env(**kw):
    for k, v in kw.items():
        os.environ[k] = v


def forward(out):
    from paper_0912_2913_gb300 import _native as N

    works = [tiny_workload(nx, ny, nz, xbc, seed=5, solid_cells=s) for nx, ny, nz, xbc, s in CASES]
    works += [tiny_workload(16, 5, 7, 2, seed=13), W.sphere_3d(nx=60, ny=30, nz=30)]
    steps = 7
    e64, e32 = [], []
    for w in works:
        ref, _ = oracle_run(w, steps)
        got, sim = gpu_run(w, steps, "fp64")
        sim.close()
        e64.append(max(rel_errors(got, ref, w.solid)))
        variants = F32_VARIANTS + ([("1", "0")] if (w.nx, w.ny, w.nz) in TMA_SHAPES else [])
        for tma, var in variants:
            _set_env(RLB_TMA=tma, RLB_F32_VARIANT=var)
            got, sim = gpu_run(w, steps, "fp32")
            sim.close()
            e32.append(max(rel_errors(got, ref, w.solid)))
        _set_env(RLB_TMA="0", RLB_F32_VARIANT="0")
    out["groups"]["forward"] = N.rlb_debug_bounds_violations()
    out["errors"]["forward_fp64"] = max(e64)
    out["errors"]["forward_fp32"] = max(e32)


def _adjoint_inputs(w, sim, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    fluid = torch.from_numpy(np.ones((w.nz, w.ny, w.nx), bool) if w.solid is None else w.solid == 0).cuda()
    shp = (w.nz, w.ny, w.nx)
    dn = torch.randn(shp, generator=g, dtype=torch.float64).cuda() * fluid
    de = torch.randn(shp, generator=g, dtype=torch.float64).cuda() * fluid
    db = torch.randn((3,) + shp, generator=g, dtype=torch.float64).cuda() * fluid
    return dn, de, db


def adjoint(out):
    """Every adjoint kernel (both precisions; FP32: one cell per thread,
    persistent, shared-memory staged with lambda copied by the block or per
    thread; the
    allocation-free step; macro and field adjoints); the parity of the
    adjoint step with the oracle's taped adjoint."""
    from paper_0912_2913_gb300 import RLB
    from paper_0912_2913_gb300 import _native as N

    worst = {"fp64": 0.0, "fp32": 0.0}
    for k, (nx, ny, nz, xbc, s) in enumerate(CASES + [(70, 40, 33, 1, ((30, 20, 16), (31, 20, 16)))]):
        w = tiny_workload(nx, ny, nz, xbc, seed=12, solid_cells=s)
        p = oracle.Params(**w.params())
        for prec in ("fp64", "fp32"):
            modes = ("0", "1", "2", "2p") if prec == "fp32" else ("0",)
            for mode in modes:
                _set_env(RLB_ADJ_PIPE=mode[0], RLB_ADJ_COOP="0" if mode == "2p" else "1")
                sim = RLB.from_workload(w, prec, device="cuda:0").init_fields(w.n, w.eps, w.beta, w.solid)
                sim.step(3)
                state = sim.state().clone()
                dn, de, db = _adjoint_inputs(w, sim, seed=k)
                lam = sim.new_state()
                sim.adjoint_macro(state, dn, de, db, lam)
                # lambda of solid cells set to zero on both sides
                fluid = (np.ones((w.nz, w.ny, w.nx), bool) if w.solid is None else w.solid == 0)[..., None, None]
                li = np.where(fluid, sim.state_to_cells(lam).double().cpu().numpy(), 0.0)
                lam = sim.cells_to_state(torch.from_numpy(li).cuda())
                lo = torch.zeros_like(lam)
                acc = torch.zeros(4, dtype=torch.float64, device="cuda")
                sim.adjoint_step(state, lam, lo, acc[0:1], acc[1:4])
                lo2 = torch.zeros_like(lam)
                N.rlb_adjoint_step_noalloc(sim.ctx, state, lam, lo2, acc[0:1], acc[1:4])
                sim.sync()
                # the same step by the oracle, on the fluid state and lambda the
                # GPU holds (solid cells: the oracle's own initial values)
                st = sim.state_to_cells(state).double().cpu().numpy()
                if prec == "fp32":
                    fr, gr = oracle.equilibrium(sim.params.n_ref, sim.params.eps_ref, np.zeros(3), w.c_l)
                    st = st + np.stack([fr, gr])
                st = np.where(fluid, st, oracle.init(p, w.n, w.eps, w.beta, w.solid))
                ref_out, _, _ = oracle.adjoint_step(p, st, li, w.solid)
                scale = max(np.max(np.abs(np.where(fluid, ref_out, 0.0))), 1e-300)
                for res in (lo, lo2):
                    got = sim.state_to_cells(res).double().cpu().numpy()
                    d = np.where(fluid, np.abs(got - ref_out), 0.0)
                    worst[prec] = max(worst[prec], float(np.max(d)) / scale)
                lam0 = sim.new_state()
                lam0.copy_(lo)
                shp = (w.nz, w.ny, w.nx)
                f64 = dict(dtype=torch.float64, device="cuda")
                cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
                sim.adjoint_fields(cu(w.n), cu(w.eps), cu(w.beta), lam0, torch.empty(shp, **f64),
                                   torch.empty(shp, **f64), torch.empty((3,) + shp, **f64), torch.zeros(3, **f64))
                sim.sync()
                sim.close()
    _set_env(RLB_ADJ_PIPE="2", RLB_ADJ_COOP="1")
    out["groups"]["adjoint"] = N.rlb_debug_bounds_violations()
    out["errors"]["adjoint_fp64"] = worst["fp64"]
    out["errors"]["adjoint_fp32"] = worst["fp32"]


def autograd(out):
    """rlb_run forward and backward (checkpointed) on a ragged inflow lattice."""
    from paper_0912_2913_gb300 import RunSpec, rlb_run
    from paper_0912_2913_gb300 import _native as N

    w = tiny_workload(37, 9, 5, 1, seed=21, solid_cells=((12, 4, 2),))
    for prec in ("fp64", "fp32"):
        spec = RunSpec.from_workload(w, prec, steps=12, checkpoint_every=4)
        tau = torch.tensor(w.tau, dtype=torch.float64, device="cuda", requires_grad=True)
        bi = torch.tensor(w.beta_in, dtype=torch.float64, device="cuda", requires_grad=True)
        n0, e0, b0 = (torch.from_numpy(np.ascontiguousarray(a)).cuda().requires_grad_(True)
                      for a in (w.n, w.eps, w.beta))
        n, e, b = rlb_run(tau, bi, n0, e0, b0, spec)
        (e * e).sum().backward()
        assert torch.isfinite(tau.grad) and torch.isfinite(e0.grad).all()
    torch.cuda.synchronize()
    out["groups"]["autograd"] = N.rlb_debug_bounds_violations()


def general_eos(out):
    from paper_0912_2913_gb300 import _native as N

    worst = 0.0
    for (nx, ny, nz, xbc, s), eos in zip(CASES, [(5 / 3, 0.0), (1.2, 0.3), (1.2, 0.3), (1.25, 0.0), (1.2, 0.3)]):
        w = tiny_workload(nx, ny, nz, xbc, seed=3, c_l=2.0 if eos[1] == 0.0 and xbc == 0 else 1.0, solid_cells=s)
        w.eos, (w.eos_gamma, w.eos_mass) = 1, eos
        ref, _ = oracle_run(w, 20)
        got, sim = gpu_run(w, 20, "fp64")
        sim.close()
        worst = max(worst, max(rel_errors(got, ref, w.solid)))
    out["groups"]["general_eos"] = N.rlb_debug_bounds_violations()
    out["errors"]["general_eos"] = worst


def selftest(out):
    """The checker on three indices: inside, one past the end, negative."""
    from paper_0912_2913_gb300 import _native as N

    r = []
    for i in (5, 10, -1):
        checked = N.rlb_debug_bounds_selftest(i, 10)
        r.append([i, checked, N.rlb_debug_bounds_violations()])
    out["selftest"] = r


def main():
    assert os.environ.get("RLB_LIBRARY_VARIANT") == "bounds"
    from paper_0912_2913_gb300 import _native as N

    out = {"library": os.path.basename(N.library_path()), "groups": {}, "errors": {}}
    N.rlb_debug_bounds_violations()  # starts the count at zero
    forward(out)
    adjoint(out)
    autograd(out)
    general_eos(out)
    selftest(out)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
