"""Seeded synthetic inputs for the relativistic lattice Boltzmann runs.

This module only builds initial fields, obstacle masks and run parameters.  It
holds none of the scheme's arithmetic (no equilibria, moments or recovery), so
the oracle and the CUDA path can both take their inputs from here and still
share no code.  Fields use the layout (nz, ny, nx) with x fastest; beta is
(3, nz, ny, nx).  Random numbers come from numpy's PCG64 stream, which is the
same on every platform for a given seed.

Workloads (the paper's, plus the synthetic stand-ins the benchmarks use):

* ``shock_tube_1d``   -- the Riemann problem of the paper's 1D test
  (two equilibrated half spaces, membrane removed at t = 0), here with
  eps = 1, n = 1 on the left, eps = 1/16, n = 1/8 on the right, beta = 0,
  1600 x 1 x 1 cells, outflow ghost planes at both x ends, tau = 0.9.
* ``sphere_3d``       -- a relativistic shock hitting a fixed sphere (Fig. 1):
  200 x 100 x 100 cells, inflow plane x = 0 at beta_x = 0.5, eps = n = 1,
  interior at rest with n = 0.3 and eps = 1 (the inflow's energy density), a
  solid sphere of radius 15 at (60, 50, 50), outflow copy at x = 199, y and z
  periodic, tau = 0.8.  The flow switched on at beta = 0.5 drives a shock into
  the resting fluid that hits the sphere.  ``eps_int = 0.1`` gives the
  10:1 energy jump against the inflow that the scheme cannot carry: the
  gathered populations at the jump have |T^0i| > T^00 within 30 steps at
  c_l = 1 and at the first step for c_l >= 2.
* ``random_box``      -- a periodic box with eps = 1 + 0.2 phi, phi a
  Gaussian random field filtered with a Gaussian of sigma = 8 cells and
  normalised to max |phi| = 1 (a unit standard deviation reaches phi < -5 at
  512^3, eps < 0), n = eps^(3/4), and beta the curl of a three-component
  field filtered the same way, scaled to max |beta| = 0.3.
* ``perturbed_shock_tube`` -- the shock tube with eps multiplied by
  (1 + 0.05 U(-1, 1)) from seed 5 (gradient studies).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.fft as _fft

XBC_PERIODIC = 0
XBC_INFLOW_OUTFLOW = 1
XBC_OUTFLOW_BOTH = 2


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    c_l: float
    xbc: int
    steps: int
    n: np.ndarray
    eps: np.ndarray
    beta: np.ndarray
    solid: Optional[np.ndarray] = None
    n_in: float = 1.0
    eps_in: float = 1.0
    beta_in: tuple = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)
    eos: int = 0  # 0: eps = 3P; 1: P = (eos_gamma - 1)(eps - n eos_mass)
    eos_gamma: float = 4.0 / 3.0
    eos_mass: float = 0.0

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def params(self) -> dict:
        d = dict(nx=self.nx, ny=self.ny, nz=self.nz, tau=self.tau, c_l=self.c_l, xbc=self.xbc,
                 n_in=self.n_in, eps_in=self.eps_in, beta_in=tuple(self.beta_in))
        if self.eos:
            d.update(eos=self.eos, eos_gamma=self.eos_gamma, eos_mass=self.eos_mass)
        return d


def shock_tube_1d(nx: int = 1600, tau: float = 0.9, steps: int = 2000, eps_l: float = 1.0, n_l: float = 1.0,
                  eps_r: float = 1.0 / 16.0, n_r: float = 1.0 / 8.0, c_l: float = 1.0) -> Workload:
    x = np.arange(nx)
    left = x < nx // 2
    eps = np.where(left, eps_l, eps_r).astype(np.float64)[None, None, :]
    n = np.where(left, n_l, n_r).astype(np.float64)[None, None, :]
    beta = np.zeros((3, 1, 1, nx))
    return Workload("shock_tube_1d", nx, 1, 1, tau, c_l, XBC_OUTFLOW_BOTH, steps, n, eps, beta)


def riemann_tube(P0: float, P1: float, T0: float, T1: float, cells: int = 800, tau: float = 0.52,
                 c_l: float = 1.0, steps: int = 400) -> Workload:
    """Riemann problem of two equilibrated half spaces at rest: pressure P0 and
    temperature T0 left of the membrane, P1 and T1 right of it (eps = 3P,
    n = P/T), cells interior cells plus an outflow ghost plane at each end."""
    nx = cells + 2
    x = np.arange(nx)
    left = x < nx // 2
    eps = np.where(left, 3.0 * P0, 3.0 * P1).astype(np.float64)[None, None, :]
    n = np.where(left, P0 / T0, P1 / T1).astype(np.float64)[None, None, :]
    beta = np.zeros((3, 1, 1, nx))
    return Workload("riemann_tube", nx, 1, 1, tau, c_l, XBC_OUTFLOW_BOTH, steps, n, eps, beta)


def perturbed_shock_tube(nx: int = 1600, tau: float = 0.9, steps: int = 2000, seed: int = 5,
                         amp: float = 0.05) -> Workload:
    w = shock_tube_1d(nx=nx, tau=tau, steps=steps)
    rng = np.random.default_rng(seed)
    w.eps = w.eps * (1.0 + amp * rng.uniform(-1.0, 1.0, size=w.eps.shape))
    w.name = "perturbed_shock_tube"
    return w


def sphere_mask(nx: int, ny: int, nz: int, center=(60, 50, 50), radius: float = 15.0) -> np.ndarray:
    """Solid cells: (x - cx)^2 + (y - cy)^2 + (z - cz)^2 <= r^2 on integer cell indices."""
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cx, cy, cz = center
    return (((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) <= radius * radius).astype(np.uint8)


def sphere_3d(nx: int = 200, ny: int = 100, nz: int = 100, tau: float = 0.8, steps: int = 5000,
              center=None, radius: Optional[float] = None, beta_in: float = 0.5, eps_int: float = 1.0,
              n_int: float = 0.3, c_l: float = 1.0) -> Workload:
    """The 3D shock-on-a-sphere workload; smaller grids scale the sphere with the box."""
    if center is None:
        center = (round(60 * nx / 200), round(50 * ny / 100), round(50 * nz / 100))
    if radius is None:
        radius = 15.0 * min(nx / 200, ny / 100, nz / 100)
    n = np.full((nz, ny, nx), n_int)
    eps = np.full((nz, ny, nx), eps_int)
    beta = np.zeros((3, nz, ny, nx))
    solid = sphere_mask(nx, ny, nz, center, radius)
    return Workload("sphere_3d", nx, ny, nz, tau, c_l, XBC_INFLOW_OUTFLOW, steps, n, eps, beta, solid,
                    n_in=1.0, eps_in=1.0, beta_in=(beta_in, 0.0, 0.0),
                    extra=dict(center=center, radius=radius))


def _filtered_noise(shape, sigma: float, rng: np.random.Generator, ncomp: int):
    """White noise filtered in Fourier space by exp(-k^2 sigma^2 / 2); returns the
    real fields and their spectra (for spectral derivatives)."""
    nz, ny, nx = shape
    kz = 2 * np.pi * np.fft.fftfreq(nz)[:, None, None]
    ky = 2 * np.pi * np.fft.fftfreq(ny)[None, :, None]
    kx = 2 * np.pi * np.fft.rfftfreq(nx)[None, None, :]
    filt = np.exp(-0.5 * sigma * sigma * (kx * kx + ky * ky + kz * kz))
    spectra = []
    for _ in range(ncomp):
        w = rng.standard_normal(shape)
        spectra.append(_fft.rfftn(w, workers=-1) * filt)
    return spectra, (kx, ky, kz)


def random_box(L: int = 512, tau: float = 0.7, steps: int = 1000, sigma: float = 8.0, seeds=(1, 2, 3, 4),
               amp: float = 0.2, beta_max: float = 0.3, c_l: float = 1.0) -> Workload:
    shape = (L, L, L)
    (phi_hat,), _ = _filtered_noise(shape, sigma, np.random.default_rng(seeds[0]), 1)
    phi = _fft.irfftn(phi_hat, s=shape, axes=(0, 1, 2), workers=-1)
    del phi_hat
    phi = phi - phi.mean()
    phi /= np.abs(phi).max()
    eps = 1.0 + amp * phi
    del phi
    if not np.all(eps > 0):
        raise ValueError("random_box: eps must stay positive")
    n = eps ** 0.75
    beta = np.empty((3,) + shape)
    A = []
    for s in seeds[1:4]:
        (a_hat,), k = _filtered_noise(shape, sigma, np.random.default_rng(s), 1)
        A.append(a_hat)
    kx, ky, kz = k
    # beta = curl A, spectrally: (dAz/dy - dAy/dz, dAx/dz - dAz/dx, dAy/dx - dAx/dy)
    beta[0] = _fft.irfftn(1j * ky * A[2] - 1j * kz * A[1], s=shape, axes=(0, 1, 2), workers=-1)
    beta[1] = _fft.irfftn(1j * kz * A[0] - 1j * kx * A[2], s=shape, axes=(0, 1, 2), workers=-1)
    beta[2] = _fft.irfftn(1j * kx * A[1] - 1j * ky * A[0], s=shape, axes=(0, 1, 2), workers=-1)
    del A
    bmag = np.sqrt((beta * beta).sum(0)).max()
    beta *= beta_max / bmag
    return Workload("random_box", L, L, L, tau, c_l, XBC_PERIODIC, steps, n, eps, beta,
                    extra=dict(sigma=sigma, seeds=tuple(seeds)))


def shear_wave(L: int = 64, amp: float = 1e-4, tau: float = 0.8, c_l: float = 1.0) -> Workload:
    x = np.arange(L)
    beta = np.zeros((3, 1, 1, L))
    beta[1, 0, 0] = amp * np.sin(2 * np.pi * x / L)
    return Workload("shear_wave", L, 1, 1, tau, c_l, XBC_PERIODIC, 0, np.ones((1, 1, L)), np.ones((1, 1, L)), beta)


def smooth_random_fields(nx: int, ny: int, nz: int, seed: int, amp_eps: float = 0.3, bmax: float = 0.3):
    """Small smooth random fields for parity tests on tiny and ragged grids."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 8)
    eps = 1.0 + amp_eps * np.sin(2 * np.pi * x / nx + ph[0]) * np.cos(2 * np.pi * y / ny + ph[1]) \
        * np.cos(2 * np.pi * z / nz + ph[6])
    eps = eps * (1.0 + 0.02 * rng.uniform(-1, 1, size=eps.shape))
    n = eps ** 0.75 * (1.0 + 0.1 * np.cos(2 * np.pi * z / nz + ph[2]))
    beta = np.stack([np.sin(2 * np.pi * y / ny + ph[3]), np.sin(2 * np.pi * z / nz + ph[4]),
                     np.sin(2 * np.pi * x / nx + ph[5])]) * (bmax / np.sqrt(3))
    beta = beta + 0.01 * bmax * rng.uniform(-1, 1, size=beta.shape)
    return n, eps, beta
