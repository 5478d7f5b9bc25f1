"""Gradients of RLB runs: a ``torch.autograd.Function`` over the C ABI adjoint.

``rlb_run`` maps (tau, beta_in, n0, eps0, beta0) to the macroscopic fields
(n, eps, beta) after T steps.  Its backward pass is the discrete adjoint of
the whole run, computed by librlb's adjoint kernels with sqrt(T)
checkpointing:

* forward: the state is saved every K steps (K = ceil(sqrt(T)) by default);
* backward: lambda_T = (d macro / d A_T)^T (dL/dn, dL/deps, dL/dbeta)
  (rlb_adjoint_macro); then, segment by segment from the last, the states
  inside the segment are recomputed from its checkpoint into a tape
  (rlb_step_into) and the adjoint steps run backwards through them
  (rlb_adjoint_step), accumulating dL/dtau and dL/dbeta_in on the device;
  finally rlb_adjoint_fields maps lambda_0 to the initial fields.

Memory: ceil(T/K) checkpoints + K-1 tape states + 2 adjoint states, each one
state of the context's layout; every state but the checkpoints is recomputed
once (T - ceil(T/K) forward steps in the backward pass).

With ``RunSpec(store_budget_bytes=B)`` the run trades device memory for
recomputation: the last P states of the run are kept as the forward pass
writes them (rlb_step_into_counted into their own buffers, no copies) and
need no recomputation; the first H = T - P steps are checkpointed as above.
P is the largest tail for which the tail, the head's checkpoints and tape and
the adjoint pair fit in B (``CheckpointPlan``).  The adjoint steps see the
same states either way, so the gradients are the same bit for bit.

Python only sequences the calls; every arithmetic step runs in the library's
kernels.
"""
from __future__ import annotations

import math

import torch

from .rlb import RLB


class CheckpointPlan:
    """Which states of a T-step run the backward pass holds and which it
    recomputes.  States s_0 .. s_{T-1} (s_t = the state before step t) are
    needed by the adjoint steps; the head s_0 .. s_{H-1} is checkpointed every
    K steps (segments (t0, L)) and recomputed segment by segment, the tail
    s_H .. s_{T-1} (P = T - H states) is kept from the forward pass.

    max_states: how many states may be held at once (None: no tail, the plain
    checkpointed run).  K: the checkpoint interval of the head (default
    ceil(sqrt(H))).  Raises ValueError when even the plain checkpointed run
    does not fit."""

    ADJOINT_STATES = 2  # lambda_{t+1} and lambda_t

    def __init__(self, T: int, max_states: int | None = None, K: int | None = None):
        self.T = int(T)
        if self.T < 0:
            raise ValueError("T must be >= 0")
        self.K_fixed = int(K) if K else None
        if max_states is None:
            self._set(self.T)
            return
        for H in range(0, self.T + 1):
            if self.held(H) <= max_states:
                self._set(H)
                return
        raise ValueError(f"{max_states} states do not hold a {self.T}-step checkpointed run "
                         f"(it needs {self.held(self.T)})")

    def _k(self, H: int) -> int:
        if H <= 0:
            return 0
        return self.K_fixed or max(1, math.ceil(math.sqrt(H)))

    def held(self, H: int) -> int:
        """States held at once when the head has H states."""
        K = self._k(H)
        nseg = -(-H // K) if H else 0
        return (self.T - H) + nseg + max(K - 1, 0) + self.ADJOINT_STATES

    def _set(self, H: int):
        self.H, self.P, self.K = H, self.T - H, self._k(H)
        self.segments = [(t0, min(self.K, H - t0)) for t0 in range(0, H, self.K)] if H else []
        self.states_held = self.held(H)
        # forward steps the backward pass runs: every head state that is not a checkpoint
        self.recomputed_steps = sum(L - 1 for _, L in self.segments)


class RunSpec:
    """Everything about a run that is not differentiated.  store_budget_bytes:
    device memory the run may hold in states for its backward pass (None:
    plain sqrt(T) checkpointing)."""

    def __init__(self, nx, ny, nz, steps, c_l=1.0, precision="fp64", xbc="periodic", n_in=1.0, eps_in=1.0,
                 solid=None, n_ref=1.0, eps_ref=1.0, checkpoint_every=None, device="cuda:0",
                 store_budget_bytes=None):
        self.nx, self.ny, self.nz, self.steps = int(nx), int(ny), int(nz), int(steps)
        self.c_l, self.precision, self.xbc = float(c_l), precision, xbc
        self.n_in, self.eps_in = float(n_in), float(eps_in)
        self.solid = solid
        self.n_ref, self.eps_ref = float(n_ref), float(eps_ref)
        self.checkpoint_every = int(checkpoint_every) if checkpoint_every else None
        self.K = self.checkpoint_every or max(1, math.ceil(math.sqrt(max(self.steps, 1))))
        self.store_budget_bytes = store_budget_bytes
        self.device = torch.device(device)
        self.last_sim = None
        self.last_plan = None

    def plan(self, state_bytes: int) -> CheckpointPlan:
        max_states = None if self.store_budget_bytes is None else int(self.store_budget_bytes // state_bytes)
        return CheckpointPlan(self.steps, max_states, self.checkpoint_every)

    @classmethod
    def from_workload(cls, w, precision="fp64", steps=None, checkpoint_every=None, device="cuda:0",
                      store_budget_bytes=None, **kw):
        import numpy as np

        m = np.ones(w.eps.shape, bool) if w.solid is None else (w.solid == 0)
        n_ref = kw.pop("n_ref", RLB.reference_value(np.append(w.n[m], w.n_in)))
        eps_ref = kw.pop("eps_ref", RLB.reference_value(np.append(w.eps[m], w.eps_in)))
        xbc = {0: "periodic", 1: "inflow_outflow", 2: "outflow_both"}[w.xbc]
        solid = None if w.solid is None else torch.from_numpy(np.ascontiguousarray(w.solid)).to(device)
        return cls(w.nx, w.ny, w.nz, w.steps if steps is None else steps, w.c_l, precision, xbc, w.n_in, w.eps_in,
                   solid, n_ref, eps_ref, checkpoint_every, device, store_budget_bytes)


def forward_states(sim, plan: CheckpointPlan):
    """The forward pass of a checkpointed run on the context's state: T steps,
    keeping the head's checkpoints (clones of s_{t0}) and the tail s_H ..
    s_{T-1} (s_H a clone, the others written by counted steps into their own
    buffers); the context ends on s_T with every step in its statistics."""
    checkpoints = []
    for t0, L in plan.segments:
        checkpoints.append(sim.state().clone())
        sim.step(L)
    tail = []
    if plan.P:
        tail.append(sim.state().clone())  # s_H
        for _ in range(plan.P - 1):
            nxt = sim.new_state()
            sim.step_into(tail[-1], nxt, counted=True)
            tail.append(nxt)
        sim.load_state(tail[-1])  # s_{T-1} into the context; its last step gives s_T
        sim.step(1)
    return checkpoints, tail


def backward_states(sim, plan: CheckpointPlan, checkpoints, tail, lam, lam2, acc):
    """The adjoint steps t = T-1 .. 0 from lambda_T (in lam): the stored
    tail first, then the head segment by segment from the last, its states
    s_{t0+1} .. s_{t0+L-1} recomputed from the checkpoint s_{t0} into a tape.
    dL/dtau and dL/dbeta_in accumulate in acc; returns lambda_0."""
    for st in reversed(tail):
        sim.adjoint_step(st, lam, lam2, acc[0:1], acc[1:4])
        lam, lam2 = lam2, lam
    tape = [sim.new_state() for _ in range(max(plan.K - 1, 0))]
    for s_idx in range(len(plan.segments) - 1, -1, -1):
        t0, L = plan.segments[s_idx]
        seg = [checkpoints[s_idx]] + tape[:L - 1]
        for j in range(L - 1):
            sim.step_into(seg[j], seg[j + 1])
        for j in range(L - 1, -1, -1):
            sim.adjoint_step(seg[j], lam, lam2, acc[0:1], acc[1:4])
            lam, lam2 = lam2, lam
    return lam


class _RLBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, beta_in, n0, eps0, beta0, spec: RunSpec):
        sim = RLB(spec.nx, spec.ny, spec.nz, float(tau), spec.c_l, spec.precision, spec.xbc, spec.n_in, spec.eps_in,
                  tuple(float(v) for v in beta_in.detach().cpu().tolist()), spec.n_ref, spec.eps_ref,
                  device=spec.device)
        try:
            plan = spec.plan(sim.state_bytes)
        except ValueError:
            sim.close()
            raise
        n0c, e0c, b0c = (t.detach().to(spec.device, torch.float64).contiguous() for t in (n0, eps0, beta0))
        sim.init_fields(n0c, e0c, b0c, spec.solid)
        checkpoints, tail = forward_states(sim, plan)
        n, e, b, ok = sim.macro()
        spec.last_sim, spec.last_plan = sim, plan
        ctx.sim, ctx.spec, ctx.plan, ctx.checkpoints, ctx.tail = sim, spec, plan, checkpoints, tail
        ctx.fields0 = (n0c, e0c, b0c)
        return n, e, b

    @staticmethod
    def backward(ctx, gn, ge, gb):
        sim, spec = ctx.sim, ctx.spec
        dev = spec.device
        plan = ctx.plan
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
        lam = backward_states(sim, plan, ctx.checkpoints, ctx.tail, lam, lam2, acc)
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
