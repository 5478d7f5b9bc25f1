"""Pins of the oracle's x boundary planes (the inflow ghost plane held at the
equilibrium of the inflow state, the outflow copy x = nx-1 <- x = nx-2, and
outflow copies at both ends).  The paper does not state boundary conditions;
these tests fix the reading against the lattice definition itself:

* a uniform state equal to the inflow state is a fixed point of an
  inflow/outflow lattice, and a uniform drifting state is one of an
  outflow-both lattice;
* the inflow ghost plane carries exactly N^mu and T^{0 mu} of the inflow
  state (written from their definitions);
* over a step, the change of the interior totals of n gamma and T^00 is the
  flux of populations through the two x faces of the interior (streaming
  moves each population one cell, the collision conserves both sums);
* five steps agree with an independent numpy transcription with explicit
  ghost planes (tests/_numpy_rlb.py) to 1e-14.

Each of these fails for a plausible slip in the oracle's boundary code: a copy
from nx-3 instead of nx-2, a skipped ghost rewrite, swapped components of
beta_in, a wrapped x neighbour."""
import math

import numpy as np
import pytest

from tests import _numpy_rlb as NR

BETA_IN = (0.3, 0.1, -0.05)


def _uniform(orc, p, n, eps, beta):
    shape = (p.nz, p.ny, p.nx)
    b = np.empty((3,) + shape)
    for a in range(3):
        b[a] = beta[a]
    return orc.init(p, np.full(shape, n), np.full(shape, eps), b)


def _random_state(orc, p, rng, c_l, jitter=0.01):
    shape = (p.nz, p.ny, p.nx)
    n0 = rng.uniform(0.5, 1.5, size=shape)
    e0 = rng.uniform(0.5, 1.5, size=shape)
    b0 = rng.uniform(-0.2, 0.2, size=(3,) + shape) / c_l
    a = orc.init(p, n0, e0, b0)
    return a * (1.0 + jitter * rng.uniform(-1, 1, size=a.shape))


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_inflow_state_is_a_fixed_point(orc, c_l):
    """Every cell (ghosts included) at the equilibrium of the inflow state:
    nothing changes on an inflow/outflow lattice over ten steps."""
    p = orc.Params(nx=7, ny=3, nz=4, tau=0.8, c_l=c_l, xbc=orc.XBC_INFLOW_OUTFLOW, n_in=0.7, eps_in=1.3,
                   beta_in=BETA_IN)
    a = _uniform(orc, p, 0.7, 1.3, BETA_IN)
    ref = a.copy()
    orc.run(p, a, 10)
    assert np.max(np.abs(a - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_drifting_uniform_state_is_a_fixed_point_outflow_both(orc, c_l):
    p = orc.Params(nx=6, ny=4, nz=3, tau=0.7, c_l=c_l, xbc=orc.XBC_OUTFLOW_BOTH)
    a = _uniform(orc, p, 0.4, 2.0, (-0.25, 0.05, 0.1))
    ref = a.copy()
    orc.run(p, a, 10)
    assert np.max(np.abs(a - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_inflow_ghost_carries_the_inflow_moments(orc, c_l):
    """N^0 = n gamma, T^00 = (eps + P) gamma^2 - P and T^0i = (eps + P) gamma^2
    beta_i (P = eps/3) of the inflow state, at every cell of the x = 0 plane
    after init and after steps of a lattice whose interior differs from it."""
    n_in, eps_in = 0.7, 1.3
    p = orc.Params(nx=7, ny=3, nz=4, tau=0.8, c_l=c_l, xbc=orc.XBC_INFLOW_OUTFLOW, n_in=n_in, eps_in=eps_in,
                   beta_in=BETA_IN)
    a = _random_state(orc, p, np.random.default_rng(11), c_l, jitter=0.0)
    b = np.array(BETA_IN)
    gam2 = 1 / (1 - b @ b)
    P = eps_in / 3
    want = np.array([n_in * math.sqrt(gam2), (eps_in + P) * gam2 - P, *((eps_in + P) * gam2 * b)])
    e = NR.E19
    for t in range(4):
        ghost = a[:, :, 0]
        f, g = ghost[..., 0, :], ghost[..., 1, :]
        got = np.concatenate([f.sum(-1)[..., None], g.sum(-1)[..., None], c_l * g @ e], axis=-1)
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want)), t
        a = orc.step(p, a, step_index=t)


@pytest.mark.parametrize("xbc", ["inflow_outflow", "outflow_both"])
@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_interior_totals_change_by_the_face_fluxes(orc, xbc, c_l):
    """With ghost planes at x = 0 and x = nx-1, the interior cells 1..nx-2
    gain, per step, the populations moving in from the ghost planes and lose
    those moving out into them.  The collision conserves sum f and sum g of
    every cell, so for s in (f, g):

      sum_int out_s - sum_int in_s
        = sum_{e_x=+1} [A(0) - A(nx-2)] + sum_{e_x=-1} [A(nx-1) - A(1)]

    (sums over y, z and the velocities named).  A(0) and A(nx-1) are the
    ghost contents before the step; by the boundary rule they are the inflow
    equilibrium (or a copy of x = 1) and a copy of x = nx-2."""
    kind = orc.XBC_INFLOW_OUTFLOW if xbc == "inflow_outflow" else orc.XBC_OUTFLOW_BOTH
    p = orc.Params(nx=9, ny=3, nz=4, tau=0.75, c_l=c_l, xbc=kind, n_in=0.9, eps_in=1.4, beta_in=BETA_IN)
    rng = np.random.default_rng(5 + kind)
    a = _random_state(orc, p, rng, c_l)
    # ghosts as the boundary rule leaves them after a step
    a = orc.step(p, a, step_index=0)
    ex = NR.E19[:, 0]
    pos, neg = ex > 0, ex < 0
    for t in range(1, 6):
        out = orc.step(p, a, step_index=t)
        for s in (0, 1):
            before = a[:, :, 1:-1, s, :].sum()
            after = out[:, :, 1:-1, s, :].sum()
            flux = (a[:, :, 0, s, pos].sum() - a[:, :, -2, s, pos].sum()
                    + a[:, :, -1, s, neg].sum() - a[:, :, 1, s, neg].sum())
            scale = np.abs(a[:, :, :, s, :]).sum()
            assert abs((after - before) - flux) <= 1e-14 * scale, (t, s, after - before, flux)
        # the boundary rule, from the interior after the step
        assert np.array_equal(out[:, :, -1], out[:, :, -2])
        if kind == orc.XBC_OUTFLOW_BOTH:
            assert np.array_equal(out[:, :, 0], out[:, :, 1])
        else:
            assert np.array_equal(out[:, :, 0], a[:, :, 0])
        a = out


@pytest.mark.parametrize("xbc", ["inflow_outflow", "outflow_both"])
@pytest.mark.parametrize("c_l", [1.0, 10.0])
@pytest.mark.parametrize("shape", [(7, 3, 4), (4, 2, 3), (3, 1, 1)])
def test_brute_force_numpy_step_with_ghost_planes(orc, xbc, c_l, shape):
    """Five oracle steps against the numpy transcription with explicit ghost
    planes, populations off equilibrium everywhere (ghosts included), to
    1e-14 of the largest population."""
    kind = orc.XBC_INFLOW_OUTFLOW if xbc == "inflow_outflow" else orc.XBC_OUTFLOW_BOTH
    nx, ny, nz = shape
    inflow = (0.8, 1.2, BETA_IN)
    p = orc.Params(nx=nx, ny=ny, nz=nz, tau=0.8, c_l=c_l, xbc=kind, n_in=inflow[0], eps_in=inflow[1],
                   beta_in=inflow[2])
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz + 7 * kind)
    a = _random_state(orc, p, rng, c_l)
    b = a.copy()
    for t in range(5):
        a = orc.step(p, a, step_index=t)
        b = NR.step(b, 0.8, c_l, xbc=kind, inflow=inflow)
        for s in (0, 1):
            err = np.max(np.abs(a[..., s, :] - b[..., s, :])) / np.max(np.abs(b[..., s, :]))
            assert err <= 1e-14, (t, s, err)


def test_numpy_ghost_transcription_detects_a_shifted_copy(orc):
    """The comparison above is sharp enough to see the slips it guards
    against: a copy from nx-3, or a ghost plane left as it was, changes the
    state by far more than 1e-14 within two steps."""
    p = orc.Params(nx=7, ny=3, nz=4, tau=0.8, c_l=1.0, xbc=orc.XBC_INFLOW_OUTFLOW, n_in=0.8, eps_in=1.2,
                   beta_in=BETA_IN)
    a0 = _random_state(orc, p, np.random.default_rng(3), 1.0)
    good = NR.step(NR.step(a0, 0.8, 1.0, xbc=1, inflow=(0.8, 1.2, BETA_IN)), 0.8, 1.0, xbc=1,
                   inflow=(0.8, 1.2, BETA_IN))

    def shifted(h):
        out = NR.collide(NR.stream(h), 0.8, 1.0)
        out[:, :, -1] = out[:, :, -3]
        fi, gi = NR.equilibria(0.8, 1.2, np.array(BETA_IN), 1.0)
        out[:, :, 0, 0], out[:, :, 0, 1] = fi, gi
        return out

    def stale(h):
        out = NR.collide(NR.stream(h), 0.8, 1.0)
        out[:, :, -1] = out[:, :, -2]
        out[:, :, 0] = h[:, :, 0]
        return out

    def swapped(h):
        return NR.step(h, 0.8, 1.0, xbc=1, inflow=(0.8, 1.2, (BETA_IN[1], BETA_IN[0], BETA_IN[2])))

    for bad in (shifted, stale, swapped):
        wrong = bad(bad(a0))
        assert np.max(np.abs(wrong - good)) > 1e-8 * np.max(np.abs(good)), bad.__name__
