"""Seeded synthetic inputs for the vectorial lattice Boltzmann scheme.

This module holds the initial conditions and problem sets that both the CUDA
path (through its Python binding) and the FP64 oracle consume.  It contains
none of the scheme's arithmetic: no equilibria, no relaxation, no transport,
no moments.  Every function returns plain float64 numpy arrays on a periodic
Cartesian lattice whose node (i, j[, k]) sits at ((i+1/2)dx, (j+1/2)dx[, ...])
(half-integer lattice, Section 2 of the paper), x fastest in memory:

    velocity  u   : shape (d, n_y, n_x)        (3D: (3, n_z, n_y, n_x))
    potential phi : shape (n_y, n_x)           (3D: (n_z, n_y, n_x))

``phi`` is the pressure-like Lagrange multiplier of the incompressible
Navier-Stokes system (Eq. 1 of the paper); the scheme turns it into the
density perturbation at initialisation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi

# Seed base of the batched problem set (independent periodic problems).
BATCH_SEED_BASE = 20261202
BATCH_SIDES = (64, 128, 256, 512, 1024)


def node_coords(n: int, length: float = TWO_PI) -> np.ndarray:
    """Half-integer node coordinates (i + 1/2) * dx, dx = length / n."""
    dx = length / n
    return (np.arange(n, dtype=np.float64) + 0.5) * dx


def taylor_green_2d(n: int, t: float = 0.0, nu: float = 0.0, ny: int | None = None):
    """Taylor-Green vortex on [0, 2pi)^2 (Section 6.1 of the paper).

    u = (sin x cos y, -cos x sin y) e^{-2 nu t},
    phi = (cos 2x + cos 2y) / 4 * e^{-4 nu t}.
    This is also the closed-form solution used to measure the scheme's error.
    Returns (u, phi, dx).
    """
    ny = n if ny is None else ny
    dx = TWO_PI / n
    x = node_coords(n)
    y = (np.arange(ny, dtype=np.float64) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")  # shape (ny, nx)
    decay = math.exp(-2.0 * nu * t)
    u = np.empty((2, ny, n), dtype=np.float64)
    u[0] = np.sin(X) * np.cos(Y) * decay
    u[1] = -np.cos(X) * np.sin(Y) * decay
    phi = 0.25 * (np.cos(2.0 * X) + np.cos(2.0 * Y)) * math.exp(-4.0 * nu * t)
    return u, phi, dx


def double_shear_layer(n: int, width: float = 80.0, delta: float = 0.05):
    """Periodic double shear layer on [0, 2pi)^2 (Phi = 0).

    u_x = tanh(width (y - pi/2)) for y <= pi, tanh(width (3pi/2 - y)) otherwise;
    u_y = delta sin x.  Returns (u, phi, dx).
    """
    dx = TWO_PI / n
    x = node_coords(n)
    y = node_coords(n)
    X, Y = np.meshgrid(x, y, indexing="xy")
    u = np.empty((2, n, n), dtype=np.float64)
    u[0] = np.where(Y <= math.pi, np.tanh(width * (Y - 0.5 * math.pi)),
                    np.tanh(width * (1.5 * math.pi - Y)))
    u[1] = delta * np.sin(X)
    phi = np.zeros((n, n), dtype=np.float64)
    return u, phi, dx


def shear_wave(n: int, amplitude: float, mode: int, axis: int = 0, ny: int | None = None):
    """Single-mode shear wave on [0, 2pi)^2 with rho = rho_bar (phi = 0).

    axis = 0: u = (0, A sin(m x));  axis = 1: u = (A sin(m y), 0).
    Returns (u, phi, dx).
    """
    ny = n if ny is None else ny
    dx = TWO_PI / n
    x = node_coords(n)
    y = (np.arange(ny, dtype=np.float64) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    u = np.zeros((2, ny, n), dtype=np.float64)
    if axis == 0:
        u[1] = amplitude * np.sin(mode * X)
    else:
        u[0] = amplitude * np.sin(mode * Y)
    return u, np.zeros((ny, n), dtype=np.float64), dx


def random_lattice_state(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-scale, scale) float64 array: generic seeded noise for tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=shape)


def random_fourier_field(side: int, seed: int, k_peak: float = 8.0):
    """Seeded divergence-free random Fourier velocity field on [0, 2pi)^2.

    A stream function psi gets random phases and a modulus chosen so that the
    shell energy spectrum is E(k) ~ k^4 exp(-2 (k/k_peak)^2); the velocity
    u = (d psi/dy, -d psi/dx) is taken spectrally and normalised so that
    mean(|u|^2) = 1 (unit RMS speed).  Returns (u, phi = 0, dx).
    """
    rng = np.random.default_rng(seed)
    kx = np.fft.rfftfreq(side, d=1.0 / side)          # 0 .. side/2
    ky = np.fft.fftfreq(side, d=1.0 / side)           # signed
    KX, KY = np.meshgrid(kx, ky, indexing="xy")       # shape (side, side//2+1)
    k = np.sqrt(KX ** 2 + KY ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        spectrum = k ** 4 * np.exp(-2.0 * (k / k_peak) ** 2)
        amp = np.sqrt(spectrum / (math.pi * k ** 3))
    amp[k == 0] = 0.0
    # drop the Nyquist lines so that the real field is exactly divergence-free
    amp[:, -1] = 0.0 if side % 2 == 0 else amp[:, -1]
    amp[side // 2, :] = 0.0 if side % 2 == 0 else amp[side // 2, :]
    phase = rng.uniform(0.0, TWO_PI, size=amp.shape)
    psi_hat = amp * np.exp(1j * phase)
    ux = np.fft.irfft2(1j * KY * psi_hat, s=(side, side))
    uy = np.fft.irfft2(-1j * KX * psi_hat, s=(side, side))
    rms = math.sqrt(float(np.mean(ux ** 2 + uy ** 2)))
    u = np.stack([ux, uy]) / rms
    return u.astype(np.float64), np.zeros((side, side), dtype=np.float64), TWO_PI / side


@dataclass(frozen=True)
class BatchProblem:
    """One independent periodic problem of the batched workload."""
    index: int
    side: int
    nu: float
    seed: int


def batched_problem_set(count: int = 512, seed_base: int = BATCH_SEED_BASE):
    """Problem list of the batched workload: side ~ U{64..1024}, nu log-uniform.

    Problem p draws from numpy.random.default_rng(seed_base + p): first the side
    from BATCH_SIDES, then log10(nu) ~ U[-4, -2].  Its initial velocity is
    random_fourier_field(side, seed_base + p + 10**6).
    """
    out = []
    for p in range(count):
        rng = np.random.default_rng(seed_base + p)
        side = int(rng.choice(BATCH_SIDES))
        nu = float(10.0 ** rng.uniform(-4.0, -2.0))
        out.append(BatchProblem(index=p, side=side, nu=nu, seed=seed_base + p + 10 ** 6))
    return out


def taylor_green_3d(n: int):
    """3D Taylor-Green vortex on [0, 2pi)^3.

    u = (sin x cos y cos z, -cos x sin y cos z, 0),
    phi = (cos 2x + cos 2y)(cos 2z + 2) / 16.  Returns (u, phi, dx) with
    u of shape (3, n, n, n) in [component][z][y][x] order.
    """
    dx = TWO_PI / n
    c = node_coords(n)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.empty((3, n, n, n), dtype=np.float64)
    u[0] = np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    u[2] = 0.0
    phi = (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    return u, phi, dx


def poiseuille_channel(n: int, nx: int | None = None, height: float = 1.0, u_max: float = 1.0,
                       reynolds: float = 100.0):
    """Steady Poiseuille profile of the channel test (Section 6.2) at the cell centres.

    n cells across the channel (height L), nx (default n) along it (length nx dx), dx = L / n:
    u_x = 4 U y (L - y) / L^2, u_y = 0, phi = 8 nu U (nx dx - x) / L^2, nu = U L / Re.
    Returns (u (2, n, nx), phi (n, nx), dx, nu, u_in) with u_in = u_x at the left side's cells.
    """
    nx = n if nx is None else nx
    dx = height / n
    nu = u_max * height / reynolds
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(n) + 0.5) * dx, indexing="xy")
    u = np.stack([4.0 * u_max * Y * (height - Y) / height ** 2, np.zeros_like(Y)])
    phi = 8.0 * nu * u_max * (nx * dx - X) / height ** 2
    return u, phi, dx, nu, u[0][:, 0].copy()
