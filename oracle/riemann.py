"""Exact Riemann solution of an ideal ultra-relativistic fluid (P = eps/3).

TEST INFRASTRUCTURE ONLY (physics pin for the oracle).  The shock-tube test of
the paper (the Riemann problem in viscous gluon matter: two equilibrated half
spaces at pressures P0 and P1, membrane removed at t = 0) tends, as the
viscosity goes to zero, to the ideal solution computed here.  It is written
from the relativistic conservation laws d_mu T^{mu nu} = 0 and d_mu N^mu = 0
with T^{mu nu} = P eta^{mu nu} + (eps + P) u^mu u^nu and N^mu = n u^mu, and
the equation of state eps = 3P, all stated in the paper's model description.

Left state (eps_L, n_L) at rest for x < x0, right state (eps_R, n_R) at rest
for x > x0, eps_L > eps_R.  The solution is a left-moving rarefaction fan, a
contact and a right-moving shock.

* Rarefaction (simple wave, sound speed c_s = 1/sqrt(3)): along the fan
  artanh(beta) + (sqrt(3)/4) ln(eps) is constant, and the left-going
  characteristic through the point has speed xi = (beta - c_s)/(1 - beta c_s);
  the flow is isentropic, n proportional to eps^(3/4).
* Shock into matter at rest: the relative velocity of the two sides of a shock
  with eps ratio r = eps_b/eps_a is sqrt(3)(r - 1)/sqrt((3 + r)(3r + 1)); the
  shock speed follows from [T^{0x}] = v_s [T^{00}], the density from
  [N^x] = v_s [N^0].
* Contact: eps and beta continuous.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CS = 1.0 / math.sqrt(3.0)


def shock_beta(eps_post: float, eps_pre: float) -> float:
    r = eps_post / eps_pre
    return math.sqrt(3.0) * (r - 1.0) / math.sqrt((3.0 + r) * (3.0 * r + 1.0))


def rarefaction_beta(eps: float, eps_L: float) -> float:
    return math.tanh((math.sqrt(3.0) / 4.0) * math.log(eps_L / eps))


@dataclass
class RiemannSolution:
    eps_L: float
    n_L: float
    eps_R: float
    n_R: float
    eps_star: float
    beta_star: float
    n_star_L: float
    n_star_R: float
    v_shock: float
    xi_head: float
    xi_tail: float

    def sample(self, xi):
        """(eps, n, beta) at similarity coordinates xi = (x - x0)/t."""
        xi = np.asarray(xi, dtype=np.float64)
        eps = np.empty_like(xi)
        n = np.empty_like(xi)
        beta = np.empty_like(xi)
        left = xi <= self.xi_head
        fan = (xi > self.xi_head) & (xi <= self.xi_tail)
        starL = (xi > self.xi_tail) & (xi <= self.beta_star)
        starR = (xi > self.beta_star) & (xi <= self.v_shock)
        right = xi > self.v_shock
        eps[left], n[left], beta[left] = self.eps_L, self.n_L, 0.0
        # inside the fan: the left-going characteristic speed equals xi
        b = (xi[fan] + CS) / (1.0 + xi[fan] * CS)
        e = self.eps_L * np.exp(-(4.0 / math.sqrt(3.0)) * np.arctanh(b))
        eps[fan], beta[fan], n[fan] = e, b, self.n_L * (e / self.eps_L) ** 0.75
        eps[starL], n[starL], beta[starL] = self.eps_star, self.n_star_L, self.beta_star
        eps[starR], n[starR], beta[starR] = self.eps_star, self.n_star_R, self.beta_star
        eps[right], n[right], beta[right] = self.eps_R, self.n_R, 0.0
        return eps, n, beta


def solve(eps_L: float, n_L: float, eps_R: float, n_R: float, tol: float = 1e-15) -> RiemannSolution:
    """Solve for the star state by bisection on eps* in (eps_R, eps_L)."""
    assert eps_L > eps_R > 0.0
    lo, hi = eps_R, eps_L
    # g(eps) = beta_rarefaction(eps) - beta_shock(eps): decreasing in eps
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        g = rarefaction_beta(mid, eps_L) - shock_beta(mid, eps_R)
        if g > 0.0:
            lo = mid
        else:
            hi = mid
        if hi - lo <= tol * hi:
            break
    es = 0.5 * (lo + hi)
    bs = shock_beta(es, eps_R)
    gs = 1.0 / math.sqrt(1.0 - bs * bs)
    T00 = (4.0 / 3.0) * es * gs * gs - es / 3.0
    T0x = (4.0 / 3.0) * es * gs * gs * bs
    vs = T0x / (T00 - eps_R)
    # [N^x] = v_s [N^0]:  n* gamma* beta* = v_s (n* gamma* - n_R)
    nsR = vs * n_R / (gs * (vs - bs))
    nsL = n_L * (es / eps_L) ** 0.75
    xi_tail = (bs - CS) / (1.0 - bs * CS)
    return RiemannSolution(eps_L, n_L, eps_R, n_R, es, bs, nsL, nsR, vs, -CS, xi_tail)
