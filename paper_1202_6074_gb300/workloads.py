"""Seeded synthetic input fields shaped like the paper's workloads.

This module holds no lattice Boltzmann arithmetic: it only builds macroscopic fields
(density, velocity, force) on a grid, in float64 numpy arrays with shape [nz, ny, nx]
for scalars and [3, nz, ny, nx] for vectors. The tests feed the same arrays to the CUDA
library and to the CPU oracle.

Workloads (the paper itself has no experiments; these follow its problem class: forced,
possibly turbulent, Galilean-invariant flows in a box or channel):
  poiseuille        body-force channel, rest state
  taylor_green      decaying Taylor-Green vortex, optional uniform background velocity
  hit_forcing       time-constant solenoidal forcing on the shells 0 < |k| <= 2
  random_solenoidal random divergence-free velocity on |k| <= kmax
  gaussian_force    per-cell Gaussian force field
  channel           turbulent-channel start: parabolic profile scaled to a bulk speed + noise
"""
import itertools
import math

import numpy as np


def _grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def rest(nx, ny, nz=1, background=(0.0, 0.0, 0.0)):
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    for d in range(3):
        u[d] += background[d]
    return rho, u


def taylor_green(nx, ny, nz, u0=0.05, background=(0.0, 0.0, 0.0), two_d=False, xp=np, device=None):
    """u = u0 sin x cos y cos z, v = -u0 cos x sin y cos z, w = 0 (x = 2 pi i / L), plus U.

    Pressure of the incompressible solution, p = rho0 u0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2),
    sets rho = 1 + 3 p. two_d drops the z dependence (exact Navier-Stokes solution decaying
    as exp(-2 nu k^2 t) for a square box). xp = numpy or torch (with ``device``).
    """
    kw = {} if xp is np else {"device": device, "dtype": xp.float64}
    X = (xp.arange(nx, **kw) * (2 * math.pi / nx)).reshape(1, 1, nx)
    Y = (xp.arange(ny, **kw) * (2 * math.pi / ny)).reshape(1, ny, 1)
    Z = (xp.arange(nz, **kw) * (2 * math.pi / nz)).reshape(nz, 1, 1)
    cz = xp.ones_like(Z) if two_d else xp.cos(Z)
    u = xp.zeros((3, nz, ny, nx), **kw)
    u[0] = u0 * xp.sin(X) * xp.cos(Y) * cz
    u[1] = -u0 * xp.cos(X) * xp.sin(Y) * cz
    if two_d:
        p = u0 * u0 / 4.0 * (xp.cos(2 * X) + xp.cos(2 * Y)) + 0.0 * Z
    else:
        p = u0 * u0 / 16.0 * (xp.cos(2 * X) + xp.cos(2 * Y)) * (xp.cos(2 * Z) + 2.0)
    rho = 1.0 + 3.0 * p
    for d in range(3):
        u[d] += background[d]
    return rho, u


def _shell_vectors(kmax2):
    ks = []
    r = int(math.isqrt(kmax2))
    for k in itertools.product(range(-r, r + 1), repeat=3):
        n2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
        if 0 < n2 <= kmax2:
            ks.append(k)
    # one representative of each +-k pair
    reps = [k for k in ks if k > tuple(-c for c in k)]
    return reps


def hit_modes(seed=1, f_rms=5e-6):
    """The 16 +-pairs with 0 < |k| <= 2: (k, A_k perp k, phi_k), scaled so that rms |F| = f_rms.

    On a periodic box the modes are orthogonal and <cos^2> = 1/2, so rms^2 = sum |A_k|^2 / 2.
    """
    rng = np.random.default_rng(seed)
    modes = []
    for k in _shell_vectors(4):
        kv = np.array(k, dtype=np.float64)
        a = rng.standard_normal(3)
        a -= kv * (a @ kv) / (kv @ kv)
        phi = rng.uniform(0.0, 2 * math.pi)
        modes.append((k, a, phi))
    rms = math.sqrt(sum(float(a @ a) for _, a, _ in modes) / 2.0)
    return [(k, a * (f_rms / rms), phi) for k, a, phi in modes]


def hit_forcing(nx, ny, nz, seed=1, f_rms=5e-6, xp=np, device=None):
    """F = sum_k A_k cos(2 pi k.x / L + phi_k) as a [3, nz, ny, nx] float64 array.

    xp is numpy (default) or torch (then ``device`` places the field, e.g. on the GPU).
    """
    kw = {} if xp is np else {"device": device, "dtype": xp.float64}
    ax = [xp.arange(n, **kw) * (1.0 / n) if xp is np else xp.arange(n, **kw) / n for n in (nx, ny, nz)]
    F = xp.zeros((3, nz, ny, nx), **kw)
    for k, a, phi in hit_modes(seed, f_rms):
        arg = (2 * math.pi * k[2] * ax[2]).reshape(nz, 1, 1) + (2 * math.pi * k[1] * ax[1]).reshape(1, ny, 1) \
            + (2 * math.pi * k[0] * ax[0]).reshape(1, 1, nx) + phi
        c = xp.cos(arg)
        for d in range(3):
            F[d] += float(a[d]) * c
    return F


def random_solenoidal(nx, ny, nz, seed=2, kmax=4, u_rms=0.02):
    """Divergence-free velocity from seeded Fourier modes with |k| <= kmax, rms |u| = u_rms."""
    rng = np.random.default_rng(seed)
    x, y, z = _grid(nx, ny, nz)
    u = np.zeros((3, nz, ny, nx))
    for k in _shell_vectors(kmax * kmax):
        kv = np.array(k, dtype=np.float64)
        for _ in range(2):
            a = rng.standard_normal(3)
            a -= kv * (a @ kv) / (kv @ kv)
            phi = rng.uniform(0.0, 2 * math.pi)
            arg = 2 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + phi
            c = np.cos(arg) / (kv @ kv)
            for d in range(3):
                u[d] += a[d] * c
    rms = math.sqrt(float(np.mean(np.sum(u * u, axis=0))))
    rho = np.ones((nz, ny, nx))
    return rho, u * (u_rms / rms)


def gaussian_force(nx, ny, nz, seed=3, std=1e-5):
    rng = np.random.default_rng(seed)
    return std * rng.standard_normal((3, nz, ny, nx))


def channel(nx, ny, nz, u_tau=0.005, bulk_over_utau=15.7, noise=0.05, seed=5):
    """Turbulent-channel start with walls at y = -1/2 and y = ny - 1/2.

    A parabolic (laminar-shape) streamwise profile scaled to the bulk speed
    bulk_over_utau * u_tau, plus seeded Gaussian noise of relative amplitude ``noise`` of the
    centreline speed on every component. Returns (rho, u, F) with the streamwise body force
    F_x = u_tau^2 / h, h = ny / 2.
    """
    rng = np.random.default_rng(seed)
    x, y, z = _grid(nx, ny, nz)
    H = float(ny)
    eta = y + 0.5
    shape = 6.0 * eta * (H - eta) / (H * H)       # mean over the channel = 1
    ub = bulk_over_utau * u_tau
    u = np.zeros((3, nz, ny, nx))
    u[0] = ub * shape
    ucl = 1.5 * ub
    u += noise * ucl * rng.standard_normal(u.shape) * (shape / 1.5)  # vanishes at the walls
    rho = np.ones((nz, ny, nx))
    h = H / 2.0
    F = np.zeros((3, nz, ny, nx))
    F[0] = u_tau * u_tau / h
    return rho, u, F


def tau_from_reynolds(u0, length, re):
    """tau = 3 nu + 1/2 with nu = u0 L / Re."""
    return 3.0 * u0 * length / re + 0.5
