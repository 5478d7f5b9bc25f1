"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
energy-momentum tensor written from its definition, closed forms, invariants,
the exact ideal Riemann solution, transport coefficients, and finite
differences.  All run on the CPU in seconds.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import riemann
from tests import _numpy_rlb as NR

RNG = np.random.default_rng(20091215)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def t_munu(n, eps, beta):
    """T^{mu nu} = P eta^{mu nu} + (eps + P) u^mu u^nu and N^mu = n u^mu with
    u^mu = (gamma, gamma beta), eta = diag(-1, 1, 1, 1), P = eps/3."""
    beta = np.asarray(beta, float)
    gam = 1.0 / math.sqrt(1.0 - beta @ beta)
    u = np.concatenate([[gam], gam * beta])
    P = eps / 3.0
    eta = np.diag([-1.0, 1.0, 1.0, 1.0])
    return P * eta + (eps + P) * np.outer(u, u), n * u


def random_state(rng, bmax=0.8):
    n = rng.uniform(0.1, 3.0)
    eps = rng.uniform(0.05, 5.0)
    d = rng.normal(size=3)
    beta = d / np.linalg.norm(d) * rng.uniform(0.0, bmax)
    return n, eps, beta


# --------------------------------------------------------------------------- lattice
def test_d3q19_table_isotropy(orc):
    e, w, opp = orc.lattice()
    assert e.shape == (19, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    speeds = (e * e).sum(1)
    assert sorted(set(speeds.tolist())) == [0, 1, 2]  # 0, c_l, sqrt(2) c_l (Fig. 2 caption)
    assert np.allclose(w[speeds == 0], 1 / 3) and np.allclose(w[speeds == 1], 1 / 18)
    assert np.allclose(w[speeds == 2], 1 / 36)
    assert (speeds == 1).sum() == 6 and (speeds == 2).sum() == 12
    for i in range(19):
        assert np.all(e[opp[i]] == -e[i])
    I = np.eye(3)
    assert np.allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, e, e), I / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(four, iso, atol=1e-16)


# --------------------------------------------------------------------------- equilibria
@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_equilibria_match_energy_momentum_tensor(orc, c_l):
    """The moment matching the scheme is built on: zeroth, first and second
    moments of f^eq, g^eq equal N^mu and T^{mu nu} for any (n, eps, beta)."""
    e, w, _ = orc.lattice()
    c = c_l * e
    for _ in range(200):
        n, eps, beta = random_state(RNG, 0.95)
        f, g = orc.equilibrium(n, eps, beta, c_l)
        T, N = t_munu(n, eps, beta)
        scale = abs(T).max()
        assert abs(f.sum() - N[0]) <= 1e-14 * N[0]
        assert np.allclose(f @ c, N[1:], rtol=0, atol=1e-14 * N[0])
        assert abs(g.sum() - T[0, 0]) <= 2e-14 * scale
        assert np.allclose(g @ c, T[0, 1:], rtol=0, atol=2e-14 * scale)
        assert np.allclose(np.einsum("i,ia,ib->ab", g, c, c), T[1:, 1:], rtol=0, atol=5e-14 * scale * c_l)


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_rest_equilibrium(orc, c_l):
    """beta = 0: f_i = w_i n, g_i = w_i eps / c_l^2 (i > 0), g_0 = w_0 eps (3 - 2/c_l^2)."""
    _, w, _ = orc.lattice()
    n, eps = 0.7, 2.3
    f, g = orc.equilibrium(n, eps, np.zeros(3), c_l)
    assert np.allclose(f, w * n, rtol=1e-15, atol=0)
    assert np.allclose(g[1:], w[1:] * eps / c_l**2, rtol=1e-14, atol=0)
    assert abs(g[0] - w[0] * eps * (3 - 2 / c_l**2)) <= 1e-14 * eps


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_recovery_roundtrip(orc, c_l):
    """recover(moments(eq(n, eps, beta))) = (n, eps, beta), and recovery from
    T^{0 mu}, N^0 written from their definitions gives the same fields."""
    for _ in range(300):
        n, eps, beta = random_state(RNG, 0.97)
        f, g = orc.equilibrium(n, eps, beta, c_l)
        m = orc.moments(np.concatenate([f, g]), c_l)
        nn, ee, bb, bad = orc.recover(m, c_l)
        assert not bad
        assert abs(nn - n) <= 1e-12 * n and abs(ee - eps) <= 1e-12 * eps
        assert np.allclose(bb, beta, rtol=0, atol=1e-13)
        T, N = t_munu(n, eps, beta)
        nn, ee, bb, bad = orc.recover(np.array([N[0], T[0, 0], *T[0, 1:]]), c_l)
        assert abs(nn - n) <= 1e-12 * n and abs(ee - eps) <= 1e-12 * eps
        assert np.allclose(bb, beta, rtol=0, atol=1e-13)


def test_recovery_flags_unphysical(orc):
    assert orc.recover(np.array([1.0, 1.0, 1.2, 0.0, 0.0]), 1.0)[3]  # 4E^2 < 3M^2
    assert orc.recover(np.array([-1.0, 1.0, 0.0, 0.0, 0.0]), 1.0)[3]  # sum f <= 0
    assert orc.recover(np.array([1.0, -1.0, 0.0, 0.0, 0.0]), 1.0)[3]  # E <= 0
    assert not orc.recover(np.array([1.0, 1.0, 0.3, 0.1, 0.0]), 1.0)[3]


def test_positivity_flag_matches_equilibrium_signs(orc):
    """The diagnostic fires when some f_i^eq or g_i^eq is <= 0 (the positivity
    condition stated for the tachyon runs); checked against the signs of the
    FP64 equilibria away from a thin band around the threshold."""
    checked = 0
    for c_l in (1.0, 10.0):
        for _ in range(3000):
            n, eps, beta = random_state(RNG, 0.99 if c_l == 10.0 else 0.7)
            f, g = orc.equilibrium(n, eps, beta, c_l)
            lo = min((f / (n * 1.0)).min(), (g / eps).min())
            if abs(lo) < 1e-5:
                continue
            assert orc.positivity_flag(beta, c_l) == bool(lo <= 0.0)
            checked += 1
    assert checked > 5000
    # the paper's bound |c_i . u| < c_l^2/3 along an axis
    assert not orc.positivity_flag(np.array([0.33, 0, 0]), 1.0)
    assert orc.positivity_flag(np.array([0.34, 0, 0]), 1.0)


# --------------------------------------------------------------------------- streaming
def _uniform(orc, p, n=1.0, eps=1.0, beta=(0.0, 0.0, 0.0), solid=None):
    b = np.zeros((3, p.nz, p.ny, p.nx))
    for a in range(3):
        b[a] = beta[a]
    return orc.init(p, np.full((p.nz, p.ny, p.nx), n), np.full((p.nz, p.ny, p.nx), eps), b, solid)


def test_streaming_moves_population_along_its_velocity(orc):
    """Eq. (lbe1): f_i leaves x and arrives at x + c_i dt.  With 1/tau ~ 0 the
    step is pure streaming; a marked population must land one cell along e_i
    (periodic wrap in every direction)."""
    e, _, _ = orc.lattice()
    p = orc.Params(nx=5, ny=4, nz=3, tau=1e12, c_l=1.0)
    for i in range(1, 19):
        for s in (0, 1):
            a = _uniform(orc, p)
            x0, y0, z0 = 0, 3, 1  # on the wrap edge in x and y
            a[z0, y0, x0, s, i] += 1e-3
            out = orc.step(p, a)
            ref = _uniform(orc, p)
            d = out - ref
            xt, yt, zt = (x0 + e[i, 0]) % 5, (y0 + e[i, 1]) % 4, (z0 + e[i, 2]) % 3
            assert abs(d[zt, yt, xt, s, i] - 1e-3) < 1e-12
            d[zt, yt, xt, s, i] = 0.0
            assert abs(d).max() < 1e-12


def test_bounce_back_reverses_population(orc):
    e, _, opp = orc.lattice()
    p = orc.Params(nx=6, ny=5, nz=4, tau=1e12, c_l=1.0)
    solid = np.zeros((4, 5, 6), np.uint8)
    xs, ys, zs = 3, 2, 2
    solid[zs, ys, xs] = 1
    for i in range(1, 19):
        a = _uniform(orc, p, solid=solid)
        # a population at x_s - e_i moving along e_i would enter the solid cell
        x, y, z = xs - e[i, 0], ys - e[i, 1], zs - e[i, 2]
        a[z, y, x, 1, i] += 1e-3
        out = orc.step(p, a, solid=solid)
        d = out - _uniform(orc, p, solid=solid)
        assert abs(d[z, y, x, 1, opp[i]] - 1e-3) < 1e-12
        d[z, y, x, 1, opp[i]] = 0.0
        assert abs(d).max() < 1e-12


# --------------------------------------------------------------------------- invariants
def _smooth_fields(p, rng, amp_eps=0.3, bmax=0.3):
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 6)
    eps = 1.0 + amp_eps * np.sin(2 * np.pi * x / p.nx + ph[0]) * np.cos(2 * np.pi * y / p.ny + ph[1])
    n = eps**0.75 * (1.0 + 0.1 * np.cos(2 * np.pi * z / p.nz + ph[2]))
    beta = np.stack([bmax * np.sin(2 * np.pi * y / p.ny + ph[3]), bmax * np.sin(2 * np.pi * z / p.nz + ph[4]),
                     bmax * np.sin(2 * np.pi * x / p.nx + ph[5])]) / math.sqrt(3)
    return n, eps, beta


def _totals(orc, p, state, solid=None):
    e, _, _ = orc.lattice()
    s = state.reshape(-1, 2, 19)
    if solid is not None:
        s = s[solid.reshape(-1) == 0]
    f, g = s[:, 0, :], s[:, 1, :]
    return np.array([f.sum(), g.sum(), *(g @ (p.c_l * e)).sum(0)])


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (3, 3, 3), (5, 2, 3)])
@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_brute_force_numpy_step(orc, shape, c_l):
    """Tiny periodic grids: five oracle steps against the numpy transcription
    of tests/_numpy_rlb.py (np.roll streaming), agreement to 1e-14 of the largest population."""
    e, w, _ = orc.lattice()
    assert np.array_equal(e, NR.E19) and np.allclose(w, NR.W19, rtol=0, atol=1e-17)
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    n0 = rng.uniform(0.5, 1.5, size=(nz, ny, nx))
    e0 = rng.uniform(0.5, 1.5, size=(nz, ny, nx))
    b0 = rng.uniform(-0.2, 0.2, size=(3, nz, ny, nx)) / c_l
    p = orc.Params(nx=nx, ny=ny, nz=nz, tau=0.8, c_l=c_l)
    a = orc.init(p, n0, e0, b0)
    a *= 1.0 + 0.01 * rng.uniform(-1, 1, size=a.shape)  # off equilibrium
    b = a.copy()
    for t in range(5):
        a = orc.step(p, a, step_index=t)
        b = NR.step(b, 0.8, c_l)
        for s in (0, 1):
            err = np.max(np.abs(a[..., s, :] - b[..., s, :])) / np.max(np.abs(b[..., s, :]))
            assert err <= 1e-14, (t, s, err)


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_conservation_periodic(orc, c_l):
    """Streaming is a permutation and the collision conserves n gamma, T^00 and
    T^0i in each cell, so the lattice totals are constant to round-off."""
    p = orc.Params(nx=8, ny=6, nz=5, tau=0.7, c_l=c_l)
    n, eps, beta = _smooth_fields(p, RNG, bmax=0.6 if c_l > 1 else 0.2)
    a = orc.init(p, n, eps, beta)
    t0 = _totals(orc, p, a)
    orc.run(p, a, 60)
    t1 = _totals(orc, p, a)
    scale = np.abs(t0[:2]).max()
    assert np.all(np.abs(t1 - t0) <= 1e-12 * scale)


def test_conservation_with_bounce_back(orc):
    """With solid cells, number and energy stay conserved (momentum is not)."""
    p = orc.Params(nx=9, ny=7, nz=6, tau=0.8, c_l=1.0)
    solid = np.zeros((6, 7, 9), np.uint8)
    solid[2:4, 3:5, 4:6] = 1
    n, eps, beta = _smooth_fields(p, RNG)
    a = orc.init(p, n, eps, beta, solid)
    t0 = _totals(orc, p, a, solid)
    orc.run(p, a, 50, solid=solid)
    t1 = _totals(orc, p, a, solid)
    assert abs(t1[0] - t0[0]) <= 1e-12 * abs(t0[0])
    assert abs(t1[1] - t0[1]) <= 1e-12 * abs(t0[1])


def test_uniform_state_is_fixed_point(orc):
    p = orc.Params(nx=4, ny=3, nz=2, tau=0.9, c_l=1.0)
    a = _uniform(orc, p, n=0.4, eps=1.3, beta=(0.1, -0.05, 0.02))
    ref = a.copy()
    orc.run(p, a, 20)
    assert np.allclose(a, ref, rtol=1e-13, atol=0)


def test_tau_one_gives_equilibrium_of_gathered(orc):
    """tau = 1: out = eq(h), so the next macro fields equal the recovery of h."""
    e, _, _ = orc.lattice()
    p = orc.Params(nx=4, ny=4, nz=4, tau=1.0, c_l=1.0)
    n, eps, beta = _smooth_fields(p, RNG)
    a = orc.init(p, n, eps, beta)
    a += 1e-4 * RNG.normal(size=a.shape)
    out = orc.step(p, a)
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (3, 3, 1)]:
        h = np.zeros((2, 19))
        for i in range(19):
            h[:, i] = a[(z - e[i, 2]) % 4, (y - e[i, 1]) % 4, (x - e[i, 0]) % 4, :, i]
        nn, ee, bb, _ = orc.recover(orc.moments(h.reshape(-1), 1.0), 1.0)
        f, g = orc.equilibrium(nn, ee, bb, 1.0)
        assert np.allclose(out[z, y, x, 0], f, rtol=1e-13, atol=1e-15)
        assert np.allclose(out[z, y, x, 1], g, rtol=1e-13, atol=1e-15)


def test_thread_count_does_not_change_bits(orc):
    p = orc.Params(nx=7, ny=5, nz=6, tau=0.75, c_l=1.0)
    n, eps, beta = _smooth_fields(p, RNG)
    a1 = orc.init(p, n, eps, beta)
    a2 = a1.copy()
    orc.set_threads(1)
    orc.run(p, a1, 10)
    orc.set_threads(4)
    orc.run(p, a2, 10)
    orc.set_threads(0)
    assert np.array_equal(a1, a2)


# --------------------------------------------------------------------------- transport
@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_shear_wave_decay_matches_viscosity(orc, c_l):
    """eta = (4/9) gamma^2 eps (tau - dt/2) c_l^2 over the inertia (4/3) eps
    gives a kinematic viscosity (tau - 1/2)/3 in cells^2 per step: a small
    shear wave beta_y = A sin(kx) decays as exp(-nu k^2 t)."""
    L, tau, A = 64, 0.8, 1e-4
    p = orc.Params(nx=L, ny=1, nz=1, tau=tau, c_l=c_l)
    x = np.arange(L)
    k = 2 * np.pi / L
    beta = np.zeros((3, 1, 1, L))
    beta[1, 0, 0] = A * np.sin(k * x)
    a = orc.init(p, np.ones((1, 1, L)), np.ones((1, 1, L)), beta)
    amps = {}
    t = 0
    for t_next in (100, 400):
        orc.run(p, a, t_next - t)
        t = t_next
        _, _, b, _ = orc.macro(p, a)
        amps[t] = 2.0 / L * np.sum(b[1, 0, 0] * np.sin(k * x))
    rate = math.log(amps[100] / amps[400]) / 300.0
    nu = (tau - 0.5) / 3.0
    assert abs(rate / (nu * k * k) - 1.0) < 0.01


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_sound_speed(orc, c_l):
    """For eps = 3P the sound speed is 1/sqrt(3); a lattice cell is c_l times a
    light step, so a standing wave of wavenumber k (per cell) oscillates with
    omega = k / (sqrt(3) c_l) per step: its first node in time is at
    t = pi / (2 omega)."""
    L, A = 128, 1e-5
    p = orc.Params(nx=L, ny=1, nz=1, tau=0.52, c_l=c_l)
    x = np.arange(L)
    k = 2 * np.pi / L
    eps = 1.0 + A * np.cos(k * x)
    a = orc.init(p, eps**0.75, eps, np.zeros((3, 1, 1, L)))
    omega = k / (math.sqrt(3.0) * c_l)
    t_node = math.pi / (2 * omega)
    prev_t, prev_a = 0, A
    step = max(1, int(t_node / 40))
    t = 0
    while True:
        orc.run(p, a, step)
        t += step
        _, e_, _, _ = orc.macro(p, a)
        amp = 2.0 / L * np.sum((e_[0, 0] - 1.0) * np.cos(k * x))
        if amp <= 0.0:
            tz = prev_t + (t - prev_t) * prev_a / (prev_a - amp)
            break
        prev_t, prev_a = t, amp
        assert t < 3 * t_node
    assert abs(tz / t_node - 1.0) < 0.01


# --------------------------------------------------------------------------- Riemann
def test_shock_tube_paper_case_against_exact_riemann(orc):
    """The paper's Riemann test in lattice units (golden fixture with its
    citation), run at small tau (near-ideal fluid) to t = 3.2 fm/c = 400
    steps, against the exact ideal solution: the star plateau and the
    profile outside bands around the waves agree."""
    with open(os.path.join(GOLDEN, "paper_riemann_case.json")) as fh:
        gcase = json.load(fh)
    P0, P1, T0 = gcase["P0_lu"], gcase["P1_lu"], gcase["T0_lu"]
    T = int(round(gcase["t_compare_fm_per_c"] / gcase["dt_fm_per_c"]))
    assert T == 400
    nx = gcase["nz_cells"] + 2  # plus the two outflow ghost planes
    p = orc.Params(nx=nx, ny=1, nz=1, tau=0.52, c_l=gcase["c_l"], xbc=orc.XBC_OUTFLOW_BOTH)
    x = np.arange(nx)
    left = x < nx // 2
    eps = np.where(left, 3 * P0, 3 * P1)[None, None, :]
    n = np.where(left, P0 / T0, P1 / T0)[None, None, :]
    a = orc.init(p, n, eps, np.zeros((3, 1, 1, nx)))
    st = orc.Stats()
    orc.run(p, a, T, stats=st)
    assert st.n_unphysical == 0 and st.n_nonpositive_eq == 0
    nn, ee, bb, _ = orc.macro(p, a)
    sol = riemann.solve(3 * P0, P0 / T0, 3 * P1, P1 / T0)
    assert abs(sol.beta_star - gcase["beta_caption_approx"]) < 0.015  # "beta ~ 0.2"
    xi = (x + 0.5 - nx // 2) / T
    ex, nex, bex = sol.sample(xi)
    plateau = (xi > sol.xi_tail + 0.05) & (xi < sol.v_shock - 0.05)
    assert abs(bb[0, 0, 0][plateau].mean() - sol.beta_star) < 2e-4
    assert abs(ee[0, 0][plateau].mean() / sol.eps_star - 1) < 1e-4
    band = np.zeros(nx, bool)
    for xw in (sol.xi_head, sol.xi_tail, sol.beta_star, sol.v_shock):
        band |= np.abs(xi - xw) * T < 12
    keep = ~band & (x > 0) & (x < nx - 1)
    assert np.abs(bb[0, 0, 0][keep] - bex[keep]).mean() < 2e-3
    assert (np.abs(ee[0, 0][keep] - ex[keep]) / ex[keep]).mean() < 2e-3
    # the density has a contact jump; n follows the adiabat in the fan
    contact_l = (xi > sol.xi_tail + 0.05) & (xi < sol.beta_star - 0.05)
    assert abs(nn[0, 0][contact_l].mean() / sol.n_star_L - 1) < 2e-3


def test_exact_riemann_solution_is_consistent():
    """Self-checks of the exact solver: jump conditions of T^{0x}, T^{xx},
    N^x across the shock, and the rarefaction invariant."""
    s = riemann.solve(1.0, 1.0, 1 / 16, 1 / 8)
    g2 = 1 / (1 - s.beta_star**2)
    es, vs = s.eps_star, s.v_shock
    T00 = 4 / 3 * es * g2 - es / 3
    T0x = 4 / 3 * es * g2 * s.beta_star
    Txx = es / 3 + 4 / 3 * es * g2 * s.beta_star**2
    # conservation across the shock moving at vs into (eps_R, beta = 0)
    assert abs(vs * (T00 - s.eps_R) - (T0x - 0)) < 1e-13
    assert abs(vs * (T0x - 0) - (Txx - s.eps_R / 3)) < 1e-13
    gs = math.sqrt(g2)
    assert abs(vs * (s.n_star_R * gs - s.n_R) - s.n_star_R * gs * s.beta_star) < 1e-13
    inv = math.atanh(s.beta_star) + math.sqrt(3) / 4 * math.log(s.eps_star)
    assert abs(inv - math.sqrt(3) / 4 * math.log(s.eps_L)) < 1e-13
