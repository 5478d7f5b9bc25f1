"""An independent numpy transcription of one RLB time step, for pinning the
oracle on tiny lattices (test infrastructure; it imports neither the oracle
nor the CUDA package).

The step is written from the paper's model description with numpy array
operations instead of the oracle's per-cell C loops:

* streaming (Eqs. lbe1/lbe2, f_i moves from x to x + c_i dt): ``np.roll`` of
  every population plane by e_i, so cell x receives the value of x - e_i;
* moments n gamma = sum f, T^00 = sum g, T^0i = c_l sum g e_i;
* the closed-form recovery for eps = 3P: eps = -T^00 + sqrt(4 T00^2 - 3|T0|^2),
  beta = 3 T^0 / (3 T^00 + eps), n = sum f / gamma;
* the equilibria Eqs. equil1s, equil2as, equil2bs with u = beta;
* BGK relaxation out = h - (h - eq)/tau;
* the x boundary planes of the lattice (not in the paper: the inflow ghost
  plane x = 0 is rewritten to the equilibrium of the inflow state after every
  step, the outflow ghost x = nx - 1 takes a copy of all 38 populations of
  x = nx - 2, and with outflow at both ends x = 0 takes a copy of x = 1).

States have shape (nz, ny, nx, 2, 19) with [..., 0, :] = f and [..., 1, :] = g.
"""
import numpy as np

XBC_PERIODIC = 0
XBC_INFLOW_OUTFLOW = 1
XBC_OUTFLOW_BOTH = 2

# D3Q19 of the lattice description, in the velocity order of the build: rest,
# +-x, +-y, +-z, then the twelve diagonals as opposite pairs.
E19 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
                (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
                (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], float)
W19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def equilibria(n, eps, beta, c_l):
    """f^eq and g^eq (last axis: 19 velocities) of fields n, eps (shape s) and
    beta (shape s + (3,)), Eqs. equil1s, equil2as, equil2bs with c_i = c_l e_i
    and u = beta."""
    n = np.asarray(n, float)
    eps = np.asarray(eps, float)
    beta = np.asarray(beta, float)
    b2 = (beta ** 2).sum(-1)
    gam2 = 1 / (1 - b2)
    cu = c_l * beta @ E19.T  # c_i . u
    feq = W19 * (n * np.sqrt(gam2))[..., None] * (1 + 3 * cu / c_l ** 2)
    eg = (eps * gam2)[..., None]
    geq = W19 * eg * (1 / (gam2[..., None] * c_l ** 2) + 4 * cu / c_l ** 2 + 6 * cu ** 2 / c_l ** 4
                      - 2 * b2[..., None] / c_l ** 2)
    geq[..., 0] = W19[0] * eps * gam2 * (4 - (2 + c_l ** 2) / (gam2 * c_l ** 2) - 2 * b2 / c_l ** 2)
    return feq, geq


def stream(h):
    """Pull streaming on a lattice periodic in every axis: out_i(x) = h_i(x - e_i)."""
    pulled = np.empty_like(h)
    for i in range(19):
        ex, ey, ez = (int(v) for v in E19[i])
        pulled[..., i] = np.roll(h[..., i], shift=(ez, ey, ex), axis=(0, 1, 2))
    return pulled


def collide(pulled, tau, c_l):
    """Moments, recovery, equilibria and BGK relaxation of gathered populations."""
    f, g = pulled[..., 0, :], pulled[..., 1, :]
    S = f.sum(-1)
    E = g.sum(-1)
    Mv = c_l * g @ E19
    eps = -E + np.sqrt(4 * E ** 2 - 3 * (Mv ** 2).sum(-1))
    beta = 3 * Mv / (3 * E + eps)[..., None]
    gam2 = 1 / (1 - (beta ** 2).sum(-1))
    n = S / np.sqrt(gam2)
    feq, geq = equilibria(n, eps, beta, c_l)
    eq = np.stack([feq, geq], axis=-2)
    return pulled - (pulled - eq) / tau


def step(h, tau, c_l, xbc=XBC_PERIODIC, inflow=None):
    """One time step.  For xbc != periodic the x = 0 and x = nx - 1 planes are
    ghosts: the interior cells 1..nx-2 pull from them (they never wrap in x),
    and after the collision they are refilled; ``inflow`` = (n, eps, beta) of
    the inflow ghost under XBC_INFLOW_OUTFLOW."""
    out = collide(stream(h), tau, c_l)
    if xbc == XBC_PERIODIC:
        return out
    out[:, :, -1] = out[:, :, -2]
    if xbc == XBC_OUTFLOW_BOTH:
        out[:, :, 0] = out[:, :, 1]
    else:
        n_in, eps_in, beta_in = inflow
        fi, gi = equilibria(n_in, eps_in, np.asarray(beta_in, float), c_l)
        out[:, :, 0, 0, :] = fi
        out[:, :, 0, 1, :] = gi
    return out
