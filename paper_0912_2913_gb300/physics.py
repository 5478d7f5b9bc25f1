"""Host-side physics of the Riemann problem in viscous gluon matter (the
validation section of arXiv:0912.2913): unit conversions, the ideal
gluon-gas relations, and the mapping between the BGK relaxation time tau and
the ratio eta/s of shear viscosity to entropy density.

Relations used (all in lattice units, c = 1):

* equation of state eps = 3P and eps = 3 n T, so n = P / T;
* equilibrium gluon density n_eq = d_G T^3 / pi^2 with d_G = 16;
* fugacity lambda = n / n_eq and entropy density s = 4n - n ln(lambda);
* shear viscosity eta = (4/9) gamma^2 eps (tau - dt/2) c_l^2, dt = 1
  (the viscosity formula after Eqs. equil1s-equil2bs).

eta/s characterises a run at one fluid state; ``tau_for_eta_over_s`` solves
the last relation for tau at that state.  These are parameter mappings only:
no step of the lattice update runs here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

D_G = 16  # gluon degeneracy

# Lattice spacing and time step of the paper's 1x1x800 Riemann runs at c_l = 1.
DX_FM = 0.008
# Energy: 1 MeV = 8.2e-5 lattice units (T0 = 350 MeV = 0.0287).
MEV = 8.2e-5
# Energy density: the paper quotes P0 = 5.43 GeV/fm^3 = 7.9433e-6 and
# P1 = 2.22 GeV/fm^3 = 3.2567e-6 lattice units; the two ratios differ by 0.3 %.
# GeV/fm^3 -> lattice units is taken from the P0 pair.
GEV_FM3 = 7.9433e-6 / 5.43


def n_eq(T: float, d_g: int = D_G) -> float:
    """Equilibrium particle density of a gluon gas at temperature T."""
    return d_g * T ** 3 / math.pi ** 2


def number_density(P: float, T: float) -> float:
    """n from eps = 3P = 3nT."""
    return P / T


def entropy_density(n: float, T: float, d_g: int = D_G) -> float:
    """s = 4n - n ln(n / n_eq(T))."""
    return 4.0 * n - n * math.log(n / n_eq(T, d_g))


def shear_viscosity(eps: float, tau: float, c_l: float = 1.0, beta2: float = 0.0) -> float:
    """eta = (4/9) gamma^2 eps (tau - 1/2) c_l^2 with gamma^2 = 1 / (1 - beta^2)."""
    return 4.0 / 9.0 / (1.0 - beta2) * eps * (tau - 0.5) * c_l ** 2


def eta_over_s(tau: float, P: float, T: float, c_l: float = 1.0, beta2: float = 0.0) -> float:
    """eta/s of a fluid at pressure P and temperature T relaxed with tau."""
    n = number_density(P, T)
    return shear_viscosity(3.0 * P, tau, c_l, beta2) / entropy_density(n, T)


def tau_for_eta_over_s(ratio: float, P: float, T: float, c_l: float = 1.0, beta2: float = 0.0) -> float:
    """The relaxation time that gives eta/s = ratio at pressure P, temperature T."""
    n = number_density(P, T)
    s = entropy_density(n, T)
    return 0.5 + ratio * s * (1.0 - beta2) / (4.0 / 9.0 * 3.0 * P * c_l ** 2)


@dataclass
class RiemannSetup:
    """Two half spaces at rest in equilibrium, (P0, T0) left of the membrane
    and (P1, T1) right of it, in lattice units; dt in fm/c per step."""
    P0: float
    P1: float
    T0: float
    T1: float
    c_l: float = 1.0
    cells: int = 800

    @property
    def dt_fm(self) -> float:
        # dx stays 0.008 fm; the lattice speed c_l = dx/dt sets the time step
        return DX_FM / self.c_l

    def steps_for(self, t_fm: float) -> int:
        return int(round(t_fm / self.dt_fm))

    def tau_for(self, ratio: float) -> float:
        """tau giving eta/s = ratio in the left (high-pressure) initial state."""
        return tau_for_eta_over_s(ratio, self.P0, self.T0, self.c_l)


def paper_setup_beta02() -> RiemannSetup:
    """Figs. 3-4: P0 = 5.43 and P1 = 2.22 GeV/fm^3 (lattice values as quoted),
    one initial temperature T0 = 350 MeV = 0.0287, c_l = 1."""
    return RiemannSetup(P0=7.9433e-6, P1=3.2567e-6, T0=0.0287, T1=0.0287, c_l=1.0)


def paper_setup_tachyon() -> RiemannSetup:
    """Fig. 5: c_l = 10, P1 = 0.9532 GeV/fm^3, T0 = 0.0328 left and T1 = 0.0164
    right; P0 is not restated for this case and is kept at 5.43 GeV/fm^3."""
    return RiemannSetup(P0=7.9433e-6, P1=0.9532 * GEV_FM3, T0=0.0328, T1=0.0164, c_l=10.0)
