"""Pins of the oracle's general equation of state (an ideal gas with rest
mass, P = (Gamma - 1)(eps - n m), with the equilibria of Eqs. equil1,
equil2a, equil2b and a Newton recovery): the energy-momentum tensor written
from its definition with a general P, the recovery round trip, the
reduction to the eps = 3P scheme at Gamma = 4/3, m = 0, conservation, and
the relativistic ideal-gas sound speed c_s^2 = Gamma P / (eps + P).  CPU."""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(20091216)
EOS_CASES = [(4.0 / 3.0, 0.0), (5.0 / 3.0, 0.0), (5.0 / 3.0, 0.7), (1.2, 0.3)]


def t_munu_general(n, eps, P, beta):
    """T^{mu nu} = P eta^{mu nu} + (eps + P) u^mu u^nu, N^mu = n u^mu."""
    beta = np.asarray(beta, float)
    gam = 1.0 / math.sqrt(1.0 - beta @ beta)
    u = np.concatenate([[gam], gam * beta])
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    return P * eta + (eps + P) * np.outer(u, u), n * u


def random_gas_state(rng, gamma_ad, mass, bmax=0.9):
    n = rng.uniform(0.2, 3.0)
    P = rng.uniform(0.02, 3.0)
    eps = n * mass + P / (gamma_ad - 1.0)  # the EOS solved for eps
    d = rng.normal(size=3)
    beta = d / np.linalg.norm(d) * rng.uniform(0.0, bmax)
    return n, eps, P, beta


@pytest.mark.parametrize("c_l", [1.0, 10.0])
@pytest.mark.parametrize("gamma_ad,mass", EOS_CASES)
def test_general_equilibria_match_energy_momentum_tensor(orc, gamma_ad, mass, c_l):
    e, w, _ = orc.lattice()
    c = c_l * e
    for _ in range(100):
        n, eps, P, beta = random_gas_state(RNG, gamma_ad, mass)
        assert orc.eos_pressure(gamma_ad, mass, n, eps) == pytest.approx(P, rel=1e-12)
        f, g = orc.equilibrium_general(n, eps, P, beta, c_l)
        T, N = t_munu_general(n, eps, P, beta)
        scale = abs(T).max()
        assert abs(f.sum() - N[0]) <= 1e-14 * N[0]
        assert np.allclose(f @ c, N[1:], rtol=0, atol=1e-14 * N[0])
        assert abs(g.sum() - T[0, 0]) <= 4e-14 * scale
        assert np.allclose(g @ c, T[0, 1:], rtol=0, atol=4e-14 * scale)
        assert np.allclose(np.einsum("i,ia,ib->ab", g, c, c), T[1:, 1:], rtol=0, atol=1e-13 * scale * c_l)


@pytest.mark.parametrize("gamma_ad,mass", EOS_CASES)
def test_general_recovery_round_trip(orc, gamma_ad, mass):
    for _ in range(300):
        n, eps, P, beta = random_gas_state(RNG, gamma_ad, mass, bmax=0.95)
        T, N = t_munu_general(n, eps, P, beta)
        nn, ee, pp, bb, bad, iters = orc.recover_general(np.array([N[0], T[0, 0], *T[0, 1:]]), 1.0, gamma_ad, mass)
        assert not bad and iters < 40
        assert abs(nn - n) <= 1e-12 * n and abs(ee - eps) <= 1e-12 * eps and abs(pp - P) <= 1e-11 * P
        assert np.allclose(bb, beta, rtol=0, atol=1e-13)


def test_general_recovery_flags_unphysical(orc):
    # |T^0i| > T^00: no fluid state has these moments
    *_, bad, _ = orc.recover_general(np.array([1.0, 1.0, 2.0, 0.0, 0.0]), 1.0, 5.0 / 3.0, 0.5)
    assert bad
    *_, bad, _ = orc.recover_general(np.array([-1.0, 1.0, 0.1, 0.0, 0.0]), 1.0, 5.0 / 3.0, 0.5)
    assert bad


def _fields(p, rng, bmax=0.05, gamma_ad=5.0 / 3.0, mass=0.5, P_range=(0.08, 0.12)):
    """Cell-by-cell random fields (n within 10 %, P in P_range)."""
    shape = (p.nz, p.ny, p.nx)
    n = rng.uniform(0.9, 1.1, size=shape)
    P = rng.uniform(*P_range, size=shape)
    eps = n * mass + P / (gamma_ad - 1.0)
    beta = rng.uniform(-bmax, bmax, size=(3,) + shape)
    return n, eps, beta


def test_general_eos_reduces_to_the_ultrarelativistic_scheme(orc):
    """Gamma = 4/3, m = 0 is eps = 3P: ten steps of the general path equal the
    eps = 3P path to 1e-13 (the recoveries differ only in rounding)."""
    for xbc, solid in ((orc.XBC_PERIODIC, None), (orc.XBC_INFLOW_OUTFLOW, (2, 3, 4))):
        common = dict(nx=9, ny=6, nz=5, tau=0.8, c_l=1.0, xbc=xbc, n_in=1.1, eps_in=1.2, beta_in=(0.3, 0.0, 0.05))
        p3 = orc.Params(**common)
        pg = orc.Params(**common, eos=orc.EOS_GAMMA_LAW, eos_gamma=4.0 / 3.0, eos_mass=0.0)
        s = None
        if solid is not None:
            s = np.zeros((5, 6, 9), np.uint8)
            s[solid[2], solid[1], solid[0]] = 1
        n, eps, beta = _fields(p3, RNG, bmax=0.2, gamma_ad=4.0 / 3.0, mass=0.0, P_range=(0.3, 0.5))
        a = orc.init(p3, n, eps, beta, s)
        b = orc.init(pg, n, eps, beta, s)
        assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
        orc.run(p3, a, 10, solid=s)
        orc.run(pg, b, 10, solid=s)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("gamma_ad,mass,c_l", [(5.0 / 3.0, 0.0, 2.0), (1.2, 0.3, 1.0)])
def test_general_eos_conservation_periodic(orc, gamma_ad, mass, c_l):
    """Totals of n gamma, T^00 and T^0i stay constant to round-off (sound
    speeds 0.82 at c_l = 2 and 0.41 at c_l = 1)."""
    p = orc.Params(nx=8, ny=6, nz=5, tau=0.7, c_l=c_l, eos=orc.EOS_GAMMA_LAW, eos_gamma=gamma_ad, eos_mass=mass)
    n, eps, beta = _fields(p, RNG, bmax=0.2, gamma_ad=gamma_ad, mass=mass, P_range=(0.24, 0.36))
    a = orc.init(p, n, eps, beta)
    tot = lambda s: np.array([s[..., 0, :].sum(), s[..., 1, :].sum(),
                              *(np.einsum("zyxi,ia->a", s[..., 1, :], c_l * orc.lattice()[0]))])
    t0 = tot(a)
    st = orc.Stats()
    orc.run(p, a, 60, stats=st)
    assert st.n_unphysical == 0
    t1 = tot(a)
    assert np.all(np.abs(t1 - t0) <= 1e-12 * np.abs(t0[:2]).max())


@pytest.mark.parametrize("gamma_ad,mass,P0", [(1.25, 0.0, 0.25), (1.2, 0.3, 0.3)])
def test_general_eos_sound_speed(orc, gamma_ad, mass, P0):
    """Relativistic ideal gas: c_s^2 = Gamma P / (eps + P) (Gamma - 1 without
    rest mass).  A small standing pressure wave (isentropic: n follows
    P^(1/Gamma)) of wavenumber k oscillates with omega = c_s k per step at
    c_l = 1; its first node in time lies at pi / (2 omega)."""
    L, A = 128, 1e-5
    p = orc.Params(nx=L, ny=1, nz=1, tau=0.52, c_l=1.0, eos=orc.EOS_GAMMA_LAW, eos_gamma=gamma_ad,
                   eos_mass=mass)
    x = np.arange(L)
    k = 2 * np.pi / L
    n0 = 1.0
    Px = P0 * (1.0 + A * np.cos(k * x))
    nx_ = n0 * (Px / P0) ** (1.0 / gamma_ad)
    eps = nx_ * mass + Px / (gamma_ad - 1.0)
    a = orc.init(p, nx_[None, None, :], eps[None, None, :], np.zeros((3, 1, 1, L)))
    eps0 = n0 * mass + P0 / (gamma_ad - 1.0)
    cs = math.sqrt(gamma_ad * P0 / (eps0 + P0))
    omega = cs * k
    t_node = math.pi / (2 * omega)
    prev_t, prev_a = 0, A
    step = max(1, int(t_node / 40))
    t = 0
    while True:
        orc.run(p, a, step)
        t += step
        _, e_, _, _ = orc.macro(p, a)
        amp = 2.0 / L * np.sum((e_[0, 0] - eps0) * np.cos(k * x)) / (P0 / (gamma_ad - 1.0) * 1.0)
        if amp <= 0.0:
            tz = prev_t + (t - prev_t) * prev_a / (prev_a - amp)
            break
        prev_t, prev_a = t, amp
        assert t < 3 * t_node
    assert abs(tz / t_node - 1.0) < 0.01, (tz, t_node)


def test_oracle_adjoint_refuses_the_general_eos(orc):
    p = orc.Params(nx=3, ny=2, nz=2, tau=0.8, eos=orc.EOS_GAMMA_LAW, eos_gamma=5.0 / 3.0, eos_mass=0.5)
    st = np.ones((2, 2, 3, 2, 19))
    with pytest.raises(ValueError):
        orc.adjoint_step(p, st, st)
