"""Pins of the oracle's taped discrete adjoint against FP64 central finite
differences (h = 1e-6) and dot-product identities <J v, w> = <v, J^T w>."""
import numpy as np
import pytest

RNG = np.random.default_rng(4242)


def near_eq_state(orc, p, rng, solid=None, noise=1e-3, bmax=0.2):
    z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    eps = 1.0 + 0.2 * rng.uniform(-1, 1, size=x.shape)
    n = eps**0.75
    beta = bmax * rng.uniform(-1, 1, size=(3,) + x.shape) / np.sqrt(3)
    a = orc.init(p, n, eps, beta, solid)
    a *= 1.0 + noise * rng.uniform(-1, 1, size=a.shape)
    return a, (n, eps, beta)


def test_collision_adjoint_vs_fd(orc):
    for c_l in (1.0, 10.0):
        for _ in range(5):
            n, eps = RNG.uniform(0.3, 2), RNG.uniform(0.3, 2)
            beta = RNG.uniform(-0.25, 0.25, 3) * (2 if c_l > 1 else 1)
            f, g = orc.equilibrium(n, eps, beta, c_l)
            h = np.concatenate([f, g]) * (1 + 1e-2 * RNG.uniform(-1, 1, 38))
            mu = RNG.normal(size=38)
            tau = 0.8
            nu, dtau = orc.collision_adjoint(h, mu, tau, c_l)
            d = 1e-6
            fd = np.empty(38)
            for l in range(38):
                hp, hm = h.copy(), h.copy()
                hp[l] += d * abs(h[l])
                hm[l] -= d * abs(h[l])
                fd[l] = mu @ (orc.collide(hp, tau, c_l) - orc.collide(hm, tau, c_l)) / (2 * d * abs(h[l]))
            assert np.allclose(nu, fd, rtol=1e-6, atol=1e-7 * abs(nu).max())
            fdt = mu @ (orc.collide(h, tau + d, c_l) - orc.collide(h, tau - d, c_l)) / (2 * d)
            assert abs(dtau - fdt) <= 1e-6 * abs(fdt) + 1e-9


def test_deq_dfields_vs_fd(orc):
    for c_l in (1.0, 10.0):
        n, eps, beta = 0.8, 1.7, np.array([0.2, -0.1, 0.15])
        J = orc.deq_dfields(n, eps, beta, c_l)
        d = 1e-6
        x0 = np.array([n, eps, *beta])
        for r in range(5):
            xp, xm = x0.copy(), x0.copy()
            xp[r] += d
            xm[r] -= d
            fp = np.concatenate(orc.equilibrium(xp[0], xp[1], xp[2:], c_l))
            fm = np.concatenate(orc.equilibrium(xm[0], xm[1], xm[2:], c_l))
            assert np.allclose(J[:, r], (fp - fm) / (2 * d), rtol=1e-7, atol=1e-9)


CASES = [
    dict(nx=5, ny=4, nz=3, xbc=0, solid=None),
    dict(nx=6, ny=5, nz=4, xbc=0, solid=(3, 2, 2)),
    dict(nx=7, ny=3, nz=3, xbc=1, solid=(3, 1, 1)),
    dict(nx=8, ny=1, nz=1, xbc=2, solid=None),
]


def _params(orc, case, tau=0.8):
    return orc.Params(nx=case["nx"], ny=case["ny"], nz=case["nz"], tau=tau, c_l=1.0, xbc=case["xbc"], n_in=0.9,
                      eps_in=1.2, beta_in=(0.3, 0.05, -0.02))


def _solid(case):
    if case["solid"] is None:
        return None
    s = np.zeros((case["nz"], case["ny"], case["nx"]), np.uint8)
    x, y, z = case["solid"]
    s[z, y, x] = 1
    return s


@pytest.mark.parametrize("case", CASES, ids=["periodic", "solid", "inflow", "outflow2"])
def test_adjoint_step_dot_product_and_fd(orc, case):
    """<lam_in, J_step v> (central differences of the step along v) equals
    <lam_out, v>; d<lam_in, step>/dtau and d/dbeta_in match the adjoint sums."""
    p = _params(orc, case)
    solid = _solid(case)
    a, _ = near_eq_state(orc, p, RNG, solid)
    lam_in = RNG.normal(size=a.shape)
    v = RNG.normal(size=a.shape) * np.abs(a)
    if solid is not None:  # solid cells are never read; keep their content fixed
        v[solid.astype(bool)] = 0.0
    lam_out, dtau, dbeta = orc.adjoint_step(p, a, lam_in, solid)
    h = 1e-6
    fd = (orc.step(p, a + h * v, solid) - orc.step(p, a - h * v, solid)) / (2 * h)
    lhs = np.sum(lam_in * fd)
    rhs = np.sum(lam_out * v)
    assert abs(lhs - rhs) <= 1e-7 * np.sum(np.abs(lam_in * fd))
    pp = _params(orc, case, tau=p.tau + h)
    pm = _params(orc, case, tau=p.tau - h)
    fdt = np.sum(lam_in * (orc.step(pp, a, solid) - orc.step(pm, a, solid))) / (2 * h)
    assert abs(dtau - fdt) <= 1e-6 * abs(fdt) + 1e-8
    if p.xbc == 1:
        for comp in range(3):
            pp, pm = _params(orc, case), _params(orc, case)
            bp, bm = list(pp.beta_in), list(pm.beta_in)
            bp[comp] += h
            bm[comp] -= h
            pp.beta_in, pm.beta_in = tuple(bp), tuple(bm)
            fdb = np.sum(lam_in * (orc.step(pp, a, solid) - orc.step(pm, a, solid))) / (2 * h)
            assert abs(dbeta[comp] - fdb) <= 1e-6 * abs(fdb) + 1e-8
    else:
        assert np.all(dbeta == 0.0)


@pytest.mark.parametrize("case", CASES[:3], ids=["periodic", "solid", "inflow"])
def test_adjoint_macro_vs_fd(orc, case):
    p = _params(orc, case)
    solid = _solid(case)
    a, _ = near_eq_state(orc, p, RNG, solid)
    shp = (p.nz, p.ny, p.nx)
    dn, de, db = RNG.normal(size=shp), RNG.normal(size=shp), RNG.normal(size=(3,) + shp)
    if solid is not None:
        m = solid.astype(bool)
        dn[m] = de[m] = 0.0
        db[:, m] = 0.0
    lam = orc.adjoint_macro(p, a, dn, de, db, solid)
    v = RNG.normal(size=a.shape) * np.abs(a)
    h = 1e-6

    def obj(s):
        n, e, b, _ = orc.macro(p, s, solid)
        return np.nansum(dn * n) + np.nansum(de * e) + np.nansum(db * b)

    fd = (obj(a + h * v) - obj(a - h * v)) / (2 * h)
    assert abs(np.sum(lam * v) - fd) <= 1e-7 * abs(fd) + 1e-9


@pytest.mark.parametrize("case", CASES[:3], ids=["periodic", "solid", "inflow"])
def test_adjoint_fields_vs_fd(orc, case):
    p = _params(orc, case)
    solid = _solid(case)
    _, (n, eps, beta) = near_eq_state(orc, p, RNG, solid)
    lam0 = RNG.normal(size=(p.nz, p.ny, p.nx, 2, 19))
    dn, de, db, dbi = orc.adjoint_fields(p, n, eps, beta, lam0, solid)
    h = 1e-6
    vn, ve, vb = RNG.normal(size=n.shape), RNG.normal(size=n.shape), RNG.normal(size=beta.shape) * 0.1
    if solid is not None:  # the content of solid cells is never read: no gradient there
        m = solid.astype(bool)
        vn[m] = ve[m] = 0.0
        vb[:, m] = 0.0

    def obj(n_, e_, b_, pp=p):
        return np.sum(lam0 * orc.init(pp, n_, e_, b_, solid))

    fd = (obj(n + h * vn, eps + h * ve, beta + h * vb) - obj(n - h * vn, eps - h * ve, beta - h * vb)) / (2 * h)
    ad = np.sum(dn * vn) + np.sum(de * ve) + np.sum(db * vb)
    assert abs(ad - fd) <= 1e-7 * abs(fd) + 1e-9
    if p.xbc == 1:
        for comp in range(3):
            pp, pm = _params(orc, case), _params(orc, case)
            bp, bm = list(pp.beta_in), list(pm.beta_in)
            bp[comp] += h
            bm[comp] -= h
            pp.beta_in, pm.beta_in = tuple(bp), tuple(bm)
            fdb = (obj(n, eps, beta, pp) - obj(n, eps, beta, pm)) / (2 * h)
            assert abs(dbi[comp] - fdb) <= 1e-6 * abs(fdb) + 1e-9


def _loss_and_grad(orc, p, n0, e0, b0, target, T, solid=None, grad=True):
    """L = sum over non-ghost cells of (eps_T - target)^2 and its taped adjoint."""
    a = orc.init(p, n0, e0, b0, solid)
    tape = [a.copy()]
    for t in range(T):
        a = orc.step(p, a, solid, step_index=t)
        tape.append(a.copy())
    n, e, b, _ = orc.macro(p, a, solid)
    w = np.ones_like(e)
    if p.xbc != 0:
        w[..., 0] = w[..., -1] = 0.0
    if solid is not None:
        w[solid.astype(bool)] = 0.0
    r = np.where(w > 0, e - target, 0.0)
    L = np.sum(r * r)
    if not grad:
        return L
    lam = orc.adjoint_macro(p, a, np.zeros_like(e), 2 * r, np.zeros_like(b), solid)
    dtau, dbin = 0.0, np.zeros(3)
    for t in range(T - 1, -1, -1):
        lam, dt, db = orc.adjoint_step(p, tape[t], lam, solid)
        dtau += dt
        dbin += db
    dn, de, db0, dbi = orc.adjoint_fields(p, n0, e0, b0, lam, solid)
    return L, dtau, dbin + dbi, dn, de, db0


@pytest.mark.parametrize("xbc", [2, 1])
def test_taped_gradient_vs_fd(orc, xbc):
    """Gradient of a profile-mismatch loss with respect to tau, beta_in and
    the initial eps field through T steps, against central differences."""
    nx, T = 14, 12
    p = orc.Params(nx=nx, ny=1, nz=1, tau=0.9, c_l=1.0, xbc=xbc, n_in=1.0, eps_in=1.0, beta_in=(0.2, 0.0, 0.0))
    x = np.arange(nx)
    e0 = np.where(x < nx // 2, 1.0, 0.4)[None, None, :] * (1 + 0.05 * RNG.uniform(-1, 1, nx))
    n0 = e0**0.75
    b0 = np.zeros((3, 1, 1, nx))
    target = np.full((1, 1, nx), 0.7)
    L, dtau, dbin, dn, de, db0 = _loss_and_grad(orc, p, n0, e0, b0, target, T)
    h = 1e-6
    pp = orc.Params(**{**p.__dict__, "tau": p.tau + h})
    pm = orc.Params(**{**p.__dict__, "tau": p.tau - h})
    fd = (_loss_and_grad(orc, pp, n0, e0, b0, target, T, grad=False) -
          _loss_and_grad(orc, pm, n0, e0, b0, target, T, grad=False)) / (2 * h)
    assert abs(dtau - fd) <= 1e-6 * abs(fd)
    for j in (1, 5, 7, 12):
        ep, em = e0.copy(), e0.copy()
        ep[..., j] += h
        em[..., j] -= h
        fd = (_loss_and_grad(orc, p, n0, ep, b0, target, T, grad=False) -
              _loss_and_grad(orc, p, n0, em, b0, target, T, grad=False)) / (2 * h)
        assert abs(de[0, 0, j] - fd) <= 1e-6 * abs(fd) + 1e-10
    if xbc == 1:
        bp = orc.Params(**{**p.__dict__, "beta_in": (0.2 + h, 0.0, 0.0)})
        bm = orc.Params(**{**p.__dict__, "beta_in": (0.2 - h, 0.0, 0.0)})
        fd = (_loss_and_grad(orc, bp, n0, e0, b0, target, T, grad=False) -
              _loss_and_grad(orc, bm, n0, e0, b0, target, T, grad=False)) / (2 * h)
        assert abs(dbin[0] - fd) <= 1e-6 * abs(fd)
