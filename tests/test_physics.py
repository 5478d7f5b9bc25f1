"""The host-side physics of the Riemann validation (eta/s <-> tau, gluon-gas
relations, units) against closed forms and the oracle's measured transport,
and the oracle on the tachyon variant (c_l = 10) of the strong shock against
the exact ideal Riemann solution.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import riemann
from paper_0912_2913_gb300 import physics as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_entropy_of_a_boltzmann_gas():
    """s/n = 4 - mu/T for a massless Boltzmann gas with fugacity exp(mu/T):
    at lambda = 1 (n = n_eq) s = 4n; doubling n at fixed T lowers s/n by ln 2."""
    T = 0.03
    n = ph.n_eq(T)
    assert ph.entropy_density(n, T) == pytest.approx(4 * n, rel=1e-15)
    assert ph.entropy_density(2 * n, T) / (2 * n) == pytest.approx(4 - math.log(2), rel=1e-14)
    # n_eq scales as T^3 with the gluon degeneracy 16 and pi^-2
    assert ph.n_eq(2 * T) / ph.n_eq(T) == pytest.approx(8.0, rel=1e-14)
    assert ph.n_eq(math.pi ** (2 / 3) / 16 ** (1 / 3)) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_tau_eta_over_s_round_trip(c_l):
    su = ph.paper_setup_beta02()
    for ratio in (0.001, 0.01, 0.1, 0.5):
        tau = ph.tau_for_eta_over_s(ratio, su.P0, su.T0, c_l)
        assert tau > 0.5
        assert ph.eta_over_s(tau, su.P0, su.T0, c_l) == pytest.approx(ratio, rel=1e-12)
    # eta/s is linear in tau - 1/2 and vanishes at tau = 1/2
    assert ph.eta_over_s(0.5, su.P0, su.T0, c_l) == 0.0
    e1 = ph.eta_over_s(0.6, su.P0, su.T0, c_l)
    e2 = ph.eta_over_s(0.7, su.P0, su.T0, c_l)
    assert e2 == pytest.approx(2 * e1, rel=1e-13)


def test_units_quoted_by_the_paper():
    """T0 = 350 MeV = 0.0287 and P1 = 2.22 GeV/fm^3 = 3.2567e-6 with the
    conversions as taken (golden fixture of the paper's Riemann case)."""
    with open(os.path.join(GOLDEN, "paper_riemann_case.json")) as fh:
        g = json.load(fh)
    assert 350 * ph.MEV == pytest.approx(g["T0_lu"], rel=2e-3)
    assert 5.43 * ph.GEV_FM3 == pytest.approx(g["P0_lu"], rel=1e-12)
    assert 2.22 * ph.GEV_FM3 == pytest.approx(g["P1_lu"], rel=5e-3)
    su = ph.paper_setup_beta02()
    assert su.steps_for(g["t_compare_fm_per_c"]) == 400
    assert ph.paper_setup_tachyon().steps_for(3.2) == 4000


@pytest.mark.parametrize("c_l", [1.0, 10.0])
def test_shear_viscosity_matches_the_oracles_transport(orc, c_l):
    """The viscosity formula as used by the mapping, divided by the inertia
    eps + P = (4/3) eps, equals the kinematic viscosity the oracle's lattice
    actually shows (shear-wave decay, cells^2 per step, times c_l^2 to light
    units), within 1 %."""
    L, tau, A = 64, 0.8, 1e-4
    p = orc.Params(nx=L, ny=1, nz=1, tau=tau, c_l=c_l)
    x = np.arange(L)
    k = 2 * np.pi / L
    beta = np.zeros((3, 1, 1, L))
    beta[1, 0, 0] = A * np.sin(k * x)
    eps0 = 1.0
    a = orc.init(p, np.ones((1, 1, L)), np.full((1, 1, L), eps0), beta)
    amps = {}
    t = 0
    for t_next in (100, 400):
        orc.run(p, a, t_next - t)
        t = t_next
        _, _, b, _ = orc.macro(p, a)
        amps[t] = 2.0 / L * np.sum(b[1, 0, 0] * np.sin(k * x))
    nu_lattice = math.log(amps[100] / amps[400]) / 300.0 / (k * k)
    nu_formula = ph.shear_viscosity(eps0, tau, c_l) / (4.0 / 3.0 * eps0)
    assert nu_lattice * c_l ** 2 == pytest.approx(nu_formula, rel=0.01)


def test_oracle_tachyon_strong_shock_against_exact_riemann(orc):
    """The 1:16 strong shock (beta* = 0.541, beyond the c_l = 1 positivity
    bound) with numerical tachyons c_l = 10, 1600 cells, 4000 steps at tau =
    0.52: the star plateau matches the exact ideal solution."""
    import workloads as W

    P0, T0, P1, T1 = 1 / 3, 1 / 3, 1 / 48, 1 / 6  # eps 1 | 1/16, n 1 | 1/8
    w = W.riemann_tube(P0, P1, T0, T1, cells=1598, tau=0.52, c_l=10.0, steps=4000)
    p = orc.Params(**w.params())
    a = orc.init(p, w.n, w.eps, w.beta)
    st = orc.Stats()
    orc.run(p, a, w.steps, stats=st)
    assert st.n_unphysical == 0
    n, e, b, _ = orc.macro(p, a)
    sol = riemann.solve(3 * P0, P0 / T0, 3 * P1, P1 / T1)
    assert sol.beta_star == pytest.approx(0.540901, abs=1e-6)
    xi = (np.arange(w.nx) + 0.5 - w.nx // 2) * w.c_l / w.steps
    plateau = (xi > sol.xi_tail + 0.05) & (xi < sol.v_shock - 0.05)
    assert plateau.sum() > 200
    assert abs(b[0, 0, 0][plateau].mean() - sol.beta_star) < 3e-4
    assert abs(e[0, 0][plateau].mean() / sol.eps_star - 1) < 1e-3
