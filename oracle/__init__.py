"""FP64 CPU oracle of the relativistic lattice Boltzmann scheme (arXiv:0912.2913).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_0912_2913_gb300``) never imports it, and this
package imports nothing from the product.

The arithmetic lives in ``rlb_oracle.c`` (plain C, binary64,
``-ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  The oracle's state layout is cell-major:
``state[cell, s, i]`` with ``s = 0`` for f and ``s = 1`` for g, shape
``(nz, ny, nx, 2, 19)``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

XBC_PERIODIC = 0
XBC_INFLOW_OUTFLOW = 1
XBC_OUTFLOW_BOTH = 2
EOS_ULTRA = 0
EOS_GAMMA_LAW = 1


def _src_hash() -> str:
    with open(_SRC, "rb") as fh:
        return hashlib.sha1(fh.read()).hexdigest()[:12]


def build(force: bool = False) -> str:
    """Compile ``rlb_oracle.c`` into a shared library (gcc, OpenMP) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, f"librlb_oracle_{_src_hash()}.so")
    if force or not os.path.exists(so):
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, so)
        for f in os.listdir(_BUILD):
            if f.startswith("librlb_oracle_") and f.endswith(".so") and os.path.join(_BUILD, f) != so:
                try:
                    os.remove(os.path.join(_BUILD, f))
                except OSError:
                    pass
    return so


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("xbc", ctypes.c_int32), ("tau", ctypes.c_double), ("c_l", ctypes.c_double),
                ("n_in", ctypes.c_double), ("eps_in", ctypes.c_double), ("beta_in", ctypes.c_double * 3),
                ("eos", ctypes.c_int32), ("pad", ctypes.c_int32), ("eos_gamma", ctypes.c_double),
                ("eos_mass", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("n_unphysical", ctypes.c_int64),
                ("first_bad", ctypes.c_int64), ("n_nonpositive_eq", ctypes.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, i64, u8, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint8, ctypes.c_int32
        L.orc_lattice.argtypes = [P(i32), P(d), P(i32)]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        L.orc_equilibrium.argtypes = [d, d, P(d), d, P(d), P(d)]
        L.orc_moments.argtypes = [P(d), d, P(d)]
        L.orc_recover.argtypes = [P(d), d, P(d), P(d), P(d)]
        L.orc_recover.restype = ctypes.c_int
        L.orc_init.argtypes = [P(_Params), P(d), P(d), P(d), P(u8), P(d)]
        L.orc_step.argtypes = [P(_Params), P(u8), P(d), P(d), i64, P(_Stats)]
        L.orc_run.argtypes = [P(_Params), P(u8), P(d), P(d), i64, i64, P(_Stats)]
        L.orc_macro.argtypes = [P(_Params), P(u8), P(d), P(d), P(d), P(d)]
        L.orc_macro.restype = i64
        L.orc_adjoint_step.argtypes = [P(_Params), P(u8), P(d), P(d), P(d), P(d), P(d)]
        L.orc_adjoint_macro.argtypes = [P(_Params), P(u8), P(d), P(d), P(d), P(d), P(d)]
        L.orc_adjoint_fields.argtypes = [P(_Params), P(u8), P(d), P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
        L.orc_deq_dfields.argtypes = [d, d, P(d), d, P(d)]
        L.orc_collision_adjoint.argtypes = [P(d), P(d), d, d, P(d)]
        L.orc_collision_adjoint.restype = d
        L.orc_collide.argtypes = [P(d), d, d, P(d)]
        L.orc_positivity_flag.argtypes = [P(d), d]
        L.orc_positivity_flag.restype = ctypes.c_int
        L.orc_eos_pressure.argtypes = [d, d, d, d]
        L.orc_eos_pressure.restype = d
        L.orc_equilibrium_general.argtypes = [d, d, d, P(d), d, P(d), P(d)]
        L.orc_recover_general.argtypes = [P(d), d, d, d, P(d), P(d), P(d), P(d), P(ctypes.c_int)]
        L.orc_recover_general.restype = ctypes.c_int
        for f in (L.orc_adjoint_step, L.orc_adjoint_macro, L.orc_adjoint_fields):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Lattice and physics parameters of one run (oracle side)."""
    nx: int
    ny: int
    nz: int
    tau: float
    c_l: float = 1.0
    xbc: int = XBC_PERIODIC
    n_in: float = 1.0
    eps_in: float = 1.0
    beta_in: tuple = (0.0, 0.0, 0.0)
    eos: int = EOS_ULTRA
    eos_gamma: float = 4.0 / 3.0
    eos_mass: float = 0.0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def _c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.nz, p.xbc = self.nx, self.ny, self.nz, self.xbc
        p.tau, p.c_l, p.n_in, p.eps_in = self.tau, self.c_l, self.n_in, self.eps_in
        for a in range(3):
            p.beta_in[a] = float(self.beta_in[a])
        p.eos, p.pad = int(self.eos), 0
        p.eos_gamma, p.eos_mass = float(self.eos_gamma), float(self.eos_mass)
        return p


@dataclass
class Stats:
    steps: int = 0
    n_unphysical: int = 0
    first_bad: int = -1
    n_nonpositive_eq: int = 0
    _c: _Stats = field(default=None, repr=False)

    def __post_init__(self):
        self._c = _Stats(self.steps, self.n_unphysical, self.first_bad, self.n_nonpositive_eq)

    def sync(self):
        self.steps, self.n_unphysical = self._c.steps, self._c.n_unphysical
        self.first_bad, self.n_nonpositive_eq = self._c.first_bad, self._c.n_nonpositive_eq
        return self


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def lattice():
    e = np.zeros(57, np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().orc_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w),
                      opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return e.reshape(19, 3), w, opp


def equilibrium(n, eps, beta, c_l):
    f = np.zeros(19)
    g = np.zeros(19)
    b = _f64(beta)
    lib().orc_equilibrium(float(n), float(eps), _dp(b), float(c_l), _dp(f), _dp(g))
    return f, g


def moments(h38, c_l):
    h = _f64(h38)
    m = np.zeros(5)
    lib().orc_moments(_dp(h), float(c_l), _dp(m))
    return m


def recover(m, c_l):
    mm = _f64(m)
    n = ctypes.c_double()
    eps = ctypes.c_double()
    b = np.zeros(3)
    bad = lib().orc_recover(_dp(mm), float(c_l), ctypes.byref(n), ctypes.byref(eps), _dp(b))
    return n.value, eps.value, b, bool(bad)


def collide(h38, tau, c_l):
    h = _f64(h38)
    out = np.zeros(38)
    lib().orc_collide(_dp(h), float(tau), float(c_l), _dp(out))
    return out


def collision_adjoint(h38, mu38, tau, c_l):
    h = _f64(h38)
    mu = _f64(mu38)
    nu = np.zeros(38)
    dtau = lib().orc_collision_adjoint(_dp(h), _dp(mu), float(tau), float(c_l), _dp(nu))
    return nu, dtau


def deq_dfields(n, eps, beta, c_l):
    out = np.zeros((38, 5))
    b = _f64(beta)
    lib().orc_deq_dfields(float(n), float(eps), _dp(b), float(c_l), _dp(out))
    return out


def eos_pressure(gamma_ad, mass, n, eps) -> float:
    """P = (Gamma - 1)(eps - n m)."""
    return float(lib().orc_eos_pressure(float(gamma_ad), float(mass), float(n), float(eps)))


def equilibrium_general(n, eps, P, beta, c_l):
    """Eqs. (equil1), (equil2a), (equil2b) at pressure P."""
    f = np.zeros(19)
    g = np.zeros(19)
    b = _f64(beta)
    lib().orc_equilibrium_general(float(n), float(eps), float(P), _dp(b), float(c_l), _dp(f), _dp(g))
    return f, g


def recover_general(m, c_l, gamma_ad, mass):
    """(n, eps, P, beta, unphysical, newton_iterations) from the five moments."""
    mm = _f64(m)
    n, eps, P = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    it = ctypes.c_int()
    b = np.zeros(3)
    bad = lib().orc_recover_general(_dp(mm), float(c_l), float(gamma_ad), float(mass), ctypes.byref(n),
                                    ctypes.byref(eps), ctypes.byref(P), _dp(b), ctypes.byref(it))
    return n.value, eps.value, P.value, b, bool(bad), it.value


def positivity_flag(beta, c_l) -> bool:
    b = _f64(beta)
    return bool(lib().orc_positivity_flag(_dp(b), float(c_l)))


def _solid_ptr(solid, N):
    if solid is None:
        return None, ctypes.POINTER(ctypes.c_uint8)()
    s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    assert s.size == N
    return s, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def init(p: Params, n, eps, beta, solid=None):
    """Equilibrium populations of the initial fields; beta has shape (3, nz, ny, nx)."""
    N = p.N
    n_ = _f64(n).reshape(-1)
    e_ = _f64(eps).reshape(-1)
    b_ = _f64(beta).reshape(-1)
    assert n_.size == N and e_.size == N and b_.size == 3 * N
    keep, sp = _solid_ptr(solid, N)
    state = np.zeros((p.nz, p.ny, p.nx, 2, 19))
    lib().orc_init(ctypes.byref(p._c()), _dp(n_), _dp(e_), _dp(b_), sp, _dp(state))
    return state


def run(p: Params, state, nsteps, solid=None, stats: Stats | None = None, step0: int = 0):
    """Advance ``state`` (modified in place) by ``nsteps`` steps."""
    assert state.dtype == np.float64 and state.flags.c_contiguous and state.size == 38 * p.N
    keep, sp = _solid_ptr(solid, p.N)
    scratch = np.empty_like(state)
    st = stats if stats is not None else Stats()
    lib().orc_run(ctypes.byref(p._c()), sp, _dp(state), _dp(scratch), int(nsteps), int(step0), ctypes.byref(st._c))
    st.sync()
    return state


def step(p: Params, state_in, solid=None, stats: Stats | None = None, step_index: int = 0):
    keep, sp = _solid_ptr(solid, p.N)
    a = _f64(state_in)
    out = np.empty_like(a)
    st = stats if stats is not None else Stats()
    lib().orc_step(ctypes.byref(p._c()), sp, _dp(a), _dp(out), int(step_index), ctypes.byref(st._c))
    st.sync()
    return out


def macro(p: Params, state, solid=None):
    """(n, eps, beta, n_unphysical) with n, eps of shape (nz, ny, nx), beta (3, nz, ny, nx)."""
    keep, sp = _solid_ptr(solid, p.N)
    a = _f64(state)
    n = np.empty((p.nz, p.ny, p.nx))
    e = np.empty((p.nz, p.ny, p.nx))
    b = np.empty((3, p.nz, p.ny, p.nx))
    bad = lib().orc_macro(ctypes.byref(p._c()), sp, _dp(a), _dp(n), _dp(e), _dp(b))
    return n, e, b, int(bad)


def adjoint_step(p: Params, state_t, lam_in, solid=None):
    """(lam_out, dL/dtau contribution, dL/dbeta_in contribution) of one step."""
    keep, sp = _solid_ptr(solid, p.N)
    a = _f64(state_t)
    li = _f64(lam_in)
    lo = np.empty_like(li)
    dtau = ctypes.c_double(0.0)
    db = np.zeros(3)
    if lib().orc_adjoint_step(ctypes.byref(p._c()), sp, _dp(a), _dp(li), _dp(lo), ctypes.byref(dtau), _dp(db)) != 0:
        raise ValueError("the oracle adjoint covers the eps = 3P equation of state only")
    return lo, dtau.value, db


def adjoint_macro(p: Params, state, dn, deps, dbeta, solid=None):
    keep, sp = _solid_ptr(solid, p.N)
    a = _f64(state)
    dn_, de_, db_ = _f64(dn).reshape(-1), _f64(deps).reshape(-1), _f64(dbeta).reshape(-1)
    lam = np.empty((p.nz, p.ny, p.nx, 2, 19))
    if lib().orc_adjoint_macro(ctypes.byref(p._c()), sp, _dp(a), _dp(dn_), _dp(de_), _dp(db_), _dp(lam)) != 0:
        raise ValueError("the oracle adjoint covers the eps = 3P equation of state only")
    return lam


def adjoint_fields(p: Params, n, eps, beta, lam0, solid=None):
    """(dL/dn0, dL/deps0, dL/dbeta0, dL/dbeta_in contribution of the initial inflow plane)."""
    keep, sp = _solid_ptr(solid, p.N)
    n_, e_, b_ = _f64(n).reshape(-1), _f64(eps).reshape(-1), _f64(beta).reshape(-1)
    l0 = _f64(lam0)
    dn = np.empty((p.nz, p.ny, p.nx))
    de = np.empty((p.nz, p.ny, p.nx))
    db = np.empty((3, p.nz, p.ny, p.nx))
    dbi = np.zeros(3)
    if lib().orc_adjoint_fields(ctypes.byref(p._c()), sp, _dp(n_), _dp(e_), _dp(b_), _dp(l0), _dp(dn), _dp(de),
                             _dp(db), _dp(dbi)) != 0:
        raise ValueError("the oracle adjoint covers the eps = 3P equation of state only")
    return dn, de, db, dbi
