"""Gradients of RLB runs: a ``torch.autograd.Function`` over the C ABI adjoint.

``rlb_run`` maps (tau, beta_in, n0, eps0, beta0) to the macroscopic fields
(n, eps, beta) after T steps.  Its backward pass is the discrete adjoint of
the whole run, computed by librlb's adjoint kernels with sqrt(T)
checkpointing:

* forward: the state is saved every K steps (K = ceil(sqrt(T)) by default);
* backward: lambda_T = (d macro / d A_T)^T (dL/dn, dL/deps, dL/dbeta)
  (rlb_adjoint_macro); then, segment by segment from the last, the K states
  of the segment are recomputed from its checkpoint into a tape
  (rlb_step_into) and the adjoint steps run backwards through them
  (rlb_adjoint_step), accumulating dL/dtau and dL/dbeta_in on the device;
  finally rlb_adjoint_fields maps lambda_0 to the initial fields.

Memory: ceil(T/K) checkpoints + K+1 tape states + 2 adjoint states, each one
state of the context's layout.  Python only sequences the calls; every
arithmetic step runs in the library's kernels.
"""
from __future__ import annotations

import math

import torch

from .rlb import RLB


class RunSpec:
    """Everything about a run that is not differentiated."""

    def __init__(self, nx, ny, nz, steps, c_l=1.0, precision="fp64", xbc="periodic", n_in=1.0, eps_in=1.0,
                 solid=None, n_ref=1.0, eps_ref=1.0, checkpoint_every=None, device="cuda:0"):
        self.nx, self.ny, self.nz, self.steps = int(nx), int(ny), int(nz), int(steps)
        self.c_l, self.precision, self.xbc = float(c_l), precision, xbc
        self.n_in, self.eps_in = float(n_in), float(eps_in)
        self.solid = solid
        self.n_ref, self.eps_ref = float(n_ref), float(eps_ref)
        self.K = int(checkpoint_every) if checkpoint_every else max(1, math.ceil(math.sqrt(max(self.steps, 1))))
        self.device = torch.device(device)
        self.last_sim = None

    @classmethod
    def from_workload(cls, w, precision="fp64", steps=None, checkpoint_every=None, device="cuda:0", **kw):
        import numpy as np

        m = np.ones(w.eps.shape, bool) if w.solid is None else (w.solid == 0)
        n_ref = kw.pop("n_ref", RLB.reference_value(np.append(w.n[m], w.n_in)))
        eps_ref = kw.pop("eps_ref", RLB.reference_value(np.append(w.eps[m], w.eps_in)))
        xbc = {0: "periodic", 1: "inflow_outflow", 2: "outflow_both"}[w.xbc]
        solid = None if w.solid is None else torch.from_numpy(np.ascontiguousarray(w.solid)).to(device)
        return cls(w.nx, w.ny, w.nz, w.steps if steps is None else steps, w.c_l, precision, xbc, w.n_in, w.eps_in,
                   solid, n_ref, eps_ref, checkpoint_every, device)


class _RLBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, beta_in, n0, eps0, beta0, spec: RunSpec):
        sim = RLB(spec.nx, spec.ny, spec.nz, float(tau), spec.c_l, spec.precision, spec.xbc, spec.n_in, spec.eps_in,
                  tuple(float(v) for v in beta_in.detach().cpu().tolist()), spec.n_ref, spec.eps_ref,
                  device=spec.device)
        n0c, e0c, b0c = (t.detach().to(spec.device, torch.float64).contiguous() for t in (n0, eps0, beta0))
        sim.init_fields(n0c, e0c, b0c, spec.solid)
        T, K = spec.steps, spec.K
        checkpoints = []
        for t0 in range(0, T, K):
            checkpoints.append(sim.state().clone())
            sim.step(min(K, T - t0))
        n, e, b, ok = sim.macro()
        spec.last_sim = sim
        ctx.sim, ctx.spec, ctx.checkpoints = sim, spec, checkpoints
        ctx.fields0 = (n0c, e0c, b0c)
        return n, e, b

    @staticmethod
    def backward(ctx, gn, ge, gb):
        sim, spec = ctx.sim, ctx.spec
        dev = spec.device
        T, K = spec.steps, spec.K
        z = lambda g, shp: torch.zeros(shp, dtype=torch.float64, device=dev) if g is None else \
            g.to(dev, torch.float64).contiguous()
        shp = (spec.nz, spec.ny, spec.nx)
        gn, ge, gb = z(gn, shp), z(ge, shp), z(gb, (3,) + shp)
        # NaN at solid cells in the outputs: their gradients are not defined, use 0
        if spec.solid is not None:
            m = spec.solid.to(torch.bool)
            gn, ge = gn.masked_fill(m, 0.0), ge.masked_fill(m, 0.0)
            gb = gb.masked_fill(m.unsqueeze(0), 0.0)
        lam = sim.new_state()
        lam2 = sim.new_state()
        sim.adjoint_macro(sim.state(), gn, ge, gb, lam)
        acc = torch.zeros(4, dtype=torch.float64, device=dev)
        tape = [sim.new_state() for _ in range(min(K, T) + 1)]
        starts = list(range(0, T, K))
        for s_idx in range(len(starts) - 1, -1, -1):
            t0 = starts[s_idx]
            L = min(K, T - t0)
            tape[0].copy_(ctx.checkpoints[s_idx])
            for j in range(L):
                sim.step_into(tape[j], tape[j + 1])
            for j in range(L - 1, -1, -1):
                sim.adjoint_step(tape[j], lam, lam2, acc[0:1], acc[1:4])
                lam, lam2 = lam2, lam
        n0, e0, b0 = ctx.fields0
        dn0 = torch.empty_like(n0)
        de0 = torch.empty_like(e0)
        db0 = torch.empty_like(b0)
        sim.adjoint_fields(n0, e0, b0, lam, dn0, de0, db0, acc[1:4])
        dtau = acc[0].to(torch.float64)
        dbeta_in = acc[1:4].clone()
        return dtau, dbeta_in, dn0, de0, db0, None


def rlb_run(tau, beta_in, n0, eps0, beta0, spec: RunSpec):
    """Macroscopic fields (n, eps, beta) after spec.steps steps; differentiable
    with respect to tau (0-dim tensor), beta_in (3-vector, inflow velocity of
    the inflow/outflow boundary) and the initial fields n0, eps0 (nz, ny, nx)
    and beta0 (3, nz, ny, nx)."""
    return _RLBRun.apply(tau, beta_in, n0, eps0, beta0, spec)
