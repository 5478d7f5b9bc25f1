"""The backward-pass schedule of rlb_run (CheckpointPlan, forward_states,
backward_states), run on a stand-in for the library whose 'states' are
buffers holding the time index t of the state they represent: every adjoint
step sees exactly s_t, in the order t = T-1 .. 0; the context ends on s_T
with T steps counted; the states held at once are those the plan counts and
never exceed the budget; the stored tail is the largest that fits; the
recomputed forward steps are counted right.  CPU."""
import math

import pytest
import torch

from paper_0912_2913_gb300.autograd import CheckpointPlan, RunSpec, backward_states, forward_states


class FakeSim:
    def __init__(self):
        self.cur = torch.zeros(1)
        self.steps = 0
        self.forward_steps = 0
        self.seen = []
        self.buffers = 0

    def state(self):
        return self.cur

    def new_state(self):
        self.buffers += 1
        return torch.full((1,), -1.0)

    def step(self, n):
        self.cur = self.cur + n
        self.steps += n

    def step_into(self, src, dst, counted=False):
        assert src.data_ptr() != dst.data_ptr() and float(src) >= 0
        dst.copy_(src + 1)
        self.forward_steps += 1
        self.steps += 1 if counted else 0

    def load_state(self, src):
        self.cur = src.clone()

    def adjoint_step(self, state, lam, lam_out, a, b):
        self.seen.append(int(state))
        lam_out.copy_(lam - 1)


def _run(plan):
    sim = FakeSim()
    checkpoints, tail = forward_states(sim, plan)
    assert sim.steps == plan.T and int(sim.state()) == plan.T
    assert [int(c) for c in checkpoints] == [t0 for t0, _ in plan.segments]
    assert [int(s) for s in tail] == list(range(plan.H, plan.T))
    fwd = sim.forward_steps
    lam, lam2 = torch.full((1,), float(plan.T)), torch.zeros(1)
    lam0 = backward_states(sim, plan, checkpoints, tail, lam, lam2, torch.zeros(4))
    assert int(lam0) == 0  # T adjoint steps, each lambda_{t+1} -> lambda_t
    held = len(checkpoints) + len(tail) + (sim.buffers - (len(tail) - 1 if tail else 0)) + CheckpointPlan.ADJOINT_STATES
    return sim.seen, sim.forward_steps - fwd, held


@pytest.mark.parametrize("T,max_states,K", [(0, None, None), (1, None, None), (7, None, None), (100, None, None),
                                            (2000, None, 45), (100, 30, None), (100, 200, None), (17, 10, None),
                                            (2000, 657, None), (1000, 657, 20), (5, 6, None), (5, 7, None)])
def test_every_adjoint_step_sees_its_own_state(T, max_states, K):
    plan = CheckpointPlan(T, max_states, K)
    seen, recomputed, held = _run(plan)
    assert seen == list(range(T - 1, -1, -1))
    assert recomputed == plan.recomputed_steps
    assert held == plan.states_held
    if max_states is not None:
        assert held <= max_states
        if plan.H > 0:  # the tail is the largest that fits
            assert plan.held(plan.H - 1) > max_states


def test_plain_plan_is_sqrt_checkpointing():
    p = CheckpointPlan(2000, None, 45)
    assert (p.H, p.P, p.K, len(p.segments)) == (2000, 0, 45, 45)
    assert p.recomputed_steps == 2000 - 45  # every state but the checkpoints, once
    assert p.states_held == 45 + 44 + 2
    assert CheckpointPlan(2000).K == math.ceil(math.sqrt(2000))


def test_budget_trades_memory_for_recomputation():
    prev = CheckpointPlan(2000, None).recomputed_steps
    for m in (100, 300, 657, 1500, 2002):
        p = CheckpointPlan(2000, m)
        assert p.recomputed_steps < prev
        prev = p.recomputed_steps
    full = CheckpointPlan(2000, 2002)
    assert (full.H, full.P, full.recomputed_steps) == (0, 2000, 0)
    with pytest.raises(ValueError):
        CheckpointPlan(2000, 50)  # below what sqrt(T) checkpointing needs
    with pytest.raises(ValueError):
        CheckpointPlan(17, 9)


def test_runspec_plan_from_bytes():
    spec = RunSpec(8, 4, 4, 100, store_budget_bytes=40 * 1000)
    p = spec.plan(1000)
    assert p.states_held <= 40 and p.P > 0
    assert RunSpec(8, 4, 4, 100).plan(1000).P == 0


def test_schedule_sweep():
    """Every (T, budget, K) with T < 40: either the plan is refused because
    the plain checkpointed run does not fit, or every adjoint step sees its
    own state, the held states are those counted and within the budget, and
    no smaller head fits."""
    for T in range(0, 40):
        for K in (None, 1, 2, 3, 7):
            for max_states in [None] + list(range(2, T + 4)):
                try:
                    plan = CheckpointPlan(T, max_states, K)
                except ValueError:
                    assert max_states is not None
                    assert all(CheckpointPlan(T, None, K).held(H) > max_states for H in range(T + 1))
                    continue
                seen, recomputed, held = _run(plan)
                assert seen == list(range(T - 1, -1, -1)), (T, K, max_states)
                assert recomputed == plan.recomputed_steps and held == plan.states_held
                assert plan.H + plan.P == T
                if max_states is not None:
                    assert held <= max_states
                    assert all(plan.held(H) > max_states for H in range(plan.H))
