"""Pins of the FP64 oracle: checks against what the paper and the mathematics fix.

Each pin takes an `oracle.Oracle` (the committed one, or a copy with a planted
mistake) and returns the measured error; PIN_LIMITS holds the bar each must
meet.  None of them re-types the oracle's own formula:

  shear_wave     exact 4-state recurrence of a single-axis shear wave (a closed
                 form of the transport + relaxation of Section 2 for that family)
  one_step       discrete conservation form of one step from equilibrium
                 (Section 2: equilibria are fixed points of the relaxation, then
                 transport shifts them)
  conservation   per-step conservation of each field's zeroth moment (Section 2)
  forms          population relaxation (Eq. LBM_scheme) against the moment-form
                 relaxation of the proof of Prop. 1
  fixed_point    a uniform equilibrium stays uniform, bitwise
  fourier        small Fourier modes evolve by the eigenvalues of the linearised
                 amplification matrix of Section 5 (itself pinned by Lemmas 1-2)
  symmetry       reflection and diagonal-exchange symmetries of the Taylor-Green run
  init_macros    initialisation and moment extraction invert each other
                 (Section 2 and the pressure expansion of Prop. 1)
  tgv_decay      Taylor-Green vortex against its closed-form decay (Section 6.1)
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from oracle import spectral
import synthetic

PIN_LIMITS = {
    "shear_wave": 1e-12,
    "one_step": 1e-12,
    "conservation": 1e-13,
    "forms": 1e-14,
    "fixed_point": 0.0,
    "fourier": 1e-6,
    "symmetry": 1e-12,
    "init_macros": 1e-12,
    "tgv_decay": 1.0,
}

# parameters that give every field its own omega and alpha, so that a mix-up
# between fields changes the result
MIXED = dict(mu=8.0, omega=(1.2, 1.3, 1.1), alpha=(0.075, 0.02, 0.03))


def _params(n, dx, **kw):
    base = dict(MIXED)
    base.update(kw)
    return oracle.Params(n=tuple(n), dx=dx, **base)


def shear_wave(orc, n=32, ny=24, mode=3, nsteps=150, amplitude=0.3):
    """Max relative error of a shear wave against 1^T (S C)^n v (both axes)."""
    worst = 0.0
    for axis in (0, 1):
        nx_, ny_ = (n, ny) if axis == 0 else (ny, n)
        dx = synthetic.TWO_PI / n
        p = _params((nx_, ny_), dx)
        if axis == 0:
            u, phi, _ = synthetic.shear_wave(nx_, amplitude, mode, axis=0, ny=ny_)
            k = 2                     # the q_y field carries the wave
        else:
            # a wave in y on an (ny x n) lattice: the period along y is n cells
            x = synthetic.node_coords(nx_, nx_ * dx)
            y = synthetic.node_coords(ny_, ny_ * dx)
            X, Y = np.meshgrid(x, y, indexing="xy")
            u = np.zeros((2, ny_, nx_))
            u[0] = amplitude * np.sin(mode * Y)
            phi = np.zeros((ny_, nx_))
            k = 1
        f = orc.init(p, u, phi)
        f = orc.run(p, f, nsteps)
        rho, um, _ = orc.macros(p, f)
        theta = mode * dx
        gain = spectral.shear_wave_gain(theta, nsteps, p.omega[k], p.alpha[k])
        expect = u[k - 1] * gain
        err = np.max(np.abs(um[k - 1] - expect)) / (amplitude * abs(gain))
        err_other = np.max(np.abs(um[2 - k])) / amplitude
        err_rho = np.max(np.abs(rho - 1.0))
        worst = max(worst, err, err_other, err_rho)
    return worst


def _shift(g, dx_, dy_):
    """g(i + dx_, j + dy_) with periodic wrap (arrays are [y][x])."""
    return np.roll(np.roll(g, -dx_, axis=1), -dy_, axis=0)


def one_step(orc, n=(12, 10), seed=7, gamma=1.0):
    """Max relative error of one step from equilibrium against its conservation form.

    From f = f^eq(rho, q), relaxation leaves f unchanged and transport gives
      rho'   = rho + a_r L(rho) - h [D_x q_x + D_y q_y]
      dx q_x' = dx q_x + dx a_x L(q_x) - D_x F_xx - D_y F_xy
      dx q_y' = dx q_y + dx a_y L(q_y) - D_x F_yx - D_y F_yy
    with L(g) = sum of the 4 neighbours - 4 g, D_x g = g(i+1) - g(i-1),
    h = dx/(2 mu), c = dx^2/(2 mu), F_xx = c q_x^2/rho + P/(2 mu),
    F_xy = F_yx = c q_x q_y / rho, F_yy = c q_y^2/rho + P/(2 mu).
    """
    dx = 0.1
    p = _params(n, dx, gamma=gamma)
    rng = np.random.default_rng(seed)
    ny, nx = n[1], n[0]
    rho = 1.0 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    u = rng.uniform(-1, 1, (2, ny, nx))
    phi = (rho ** gamma - 1.0) / (dx * dx)
    f = orc.init(p, u, phi)
    rho0, u0, _ = orc.macros(p, f)
    qx, qy = rho0 * u0[0], rho0 * u0[1]
    f1 = orc.run(p, f, 1)
    rho1, u1, _ = orc.macros(p, f1)
    mu = p.mu
    h, c = dx / (2 * mu), dx * dx / (2 * mu)
    P = rho0 ** gamma
    ar, ax, ay = p.alpha[:3]

    def L(g):
        return _shift(g, 1, 0) + _shift(g, -1, 0) + _shift(g, 0, 1) + _shift(g, 0, -1) - 4 * g

    def Dx(g):
        return _shift(g, 1, 0) - _shift(g, -1, 0)

    def Dy(g):
        return _shift(g, 0, 1) - _shift(g, 0, -1)

    Fxx = c * qx * qx / rho0 + P / (2 * mu)
    Fxy = c * qx * qy / rho0
    Fyy = c * qy * qy / rho0 + P / (2 * mu)
    rho_e = rho0 + ar * L(rho0) - h * (Dx(qx) + Dy(qy))
    Qx_e = dx * qx + dx * ax * L(qx) - Dx(Fxx) - Dy(Fxy)
    Qy_e = dx * qy + dx * ay * L(qy) - Dx(Fxy) - Dy(Fyy)
    e1 = np.max(np.abs(rho1 - rho_e))
    e2 = np.max(np.abs(dx * rho1 * u1[0] - Qx_e)) / np.max(np.abs(Qx_e))
    e3 = np.max(np.abs(dx * rho1 * u1[1] - Qy_e)) / np.max(np.abs(Qy_e))
    return max(e1, e2, e3)


def conservation(orc, n=(16, 12), nsteps=40, seed=3):
    """Conservation of each field's zeroth moment (Section 2).

    Relaxation keeps sum_l f^k_l node by node and transport permutes values,
    so the lattice total of every field is constant.  Returns the largest
    node-wise or per-step change, relative to the field's sum of |f|.
    """
    dx = 0.2
    p = _params(n, dx)
    rng = np.random.default_rng(seed)
    # a generic off-equilibrium state: equilibrium plus noise on every population
    u = rng.uniform(-1, 1, (2, n[1], n[0]))
    phi = rng.uniform(-1, 1, (n[1], n[0]))
    f = orc.init(p, u, phi) + 1e-3 * rng.uniform(-1, 1, p.shape())
    tot0 = f.reshape(p.fields, -1).sum(axis=1)
    scale = np.abs(f).reshape(p.fields, -1).sum(axis=1)
    worst = 0.0
    for _ in range(nsteps):
        fs = orc.collide(p, f)
        node_scale = np.abs(f).sum(axis=1).max(axis=(1, 2))
        node = (np.abs(fs.sum(axis=1) - f.sum(axis=1)).max(axis=(1, 2)) / node_scale).max()
        f = orc.stream(p, fs)
        tot = f.reshape(p.fields, -1).sum(axis=1)
        worst = max(worst, float(np.max(np.abs(tot - tot0) / scale)), float(node))
    return worst


def forms(orc, count=500, seed=11):
    """Population relaxation against the moment-form relaxation, generic node states."""
    worst = 0.0
    for dim in (2, 3):
        n = (4,) * dim
        om = (1.2, 1.3, 1.1, 1.7)[: dim + 1]
        al = (0.075, 0.02, 0.03, 0.01)[: dim + 1]
        p = oracle.Params(n=n, dx=0.3, mu=8.0, omega=om, alpha=al, gamma=1.4)
        rng = np.random.default_rng(seed + dim)
        f = rng.uniform(-0.1, 0.1, (count, p.fields, p.q))
        f[:, 0, :] += 0.25          # keep rho near 1.25
        a = orc.collide_nodes(p, f, oracle.COLLIDE_POPULATIONS)
        b = orc.collide_nodes(p, f, oracle.COLLIDE_MOMENTS)
        worst = max(worst, float(np.max(np.abs(a - b))))
    return worst


def fixed_point(orc, n=(9, 7)):
    """Largest change of a uniform equilibrium state over 25 steps (must be 0)."""
    p = _params(n, 0.37)
    u = np.empty((2, n[1], n[0]))
    u[0], u[1] = 0.31, -0.77
    phi = np.full((n[1], n[0]), 2.5)
    f0 = orc.init(p, u, phi)
    f1 = orc.run(p, f0, 25)
    # uniform in space, and the relaxation of an equilibrium is the identity up
    # to the rounding of (1 - w) f + w f: compare every node with node (0, 0)
    spread = np.max(np.abs(f1 - f1[..., :1, :1]))
    return float(spread)


def fourier(orc, n=(24, 16), eps=1e-7, nsteps=8):
    """Small Fourier modes against lambda^n v of the amplification matrix.

    Returns max |f_n - fbar - 2 eps Re(lambda^n v e^{i theta.x})| / eps over
    every eigenpair, two wave vectors and two base states.
    """
    dx = 0.05
    p = _params(n, dx)
    worst = 0.0
    idx = np.arange(n[0])[None, :], np.arange(n[1])[:, None]
    for base in ((1.0, 0.0, 0.0), (1.1, 0.3, -0.2)):
        u_b = np.empty((2, n[1], n[0]))
        u_b[0], u_b[1] = base[1] / base[0], base[2] / base[0]
        phi_b = np.full((n[1], n[0]), (base[0] - 1.0) / (dx * dx))
        fbar = orc.init(p, u_b, phi_b)
        for m in ((2, 1), (5, 3)):
            theta = (2 * math.pi * m[0] / n[0], 2 * math.pi * m[1] / n[1])
            E = spectral.amplification_matrix(theta, dx, p.mu, p.omega, p.alpha, base)
            lam, V = np.linalg.eig(E)
            phase = np.exp(1j * (theta[0] * idx[0] + theta[1] * idx[1]))   # (ny, nx)
            for i in range(len(lam)):
                if abs(lam[i]) ** nsteps < 1e-3:
                    continue
                v = V[:, i] / np.linalg.norm(V[:, i])
                pert = 2 * eps * np.real(v[:, None, None] * phase[None])
                f0 = fbar + pert.reshape(p.shape())
                fn = orc.run(p, f0, nsteps)
                expect = fbar + (2 * eps * np.real((lam[i] ** nsteps) * v[:, None, None] * phase[None])).reshape(p.shape())
                worst = max(worst, float(np.max(np.abs(fn - expect))) / eps)
    return worst


def symmetry(orc, n=24, nsteps=60):
    """Exact lattice symmetries of the Taylor-Green run.

    The Taylor-Green data are invariant under the reflection x -> -x (with
    u_x -> -u_x), under y -> -y (with u_y -> -u_y) and under the exchange of x
    and y composed with a half-period shift along x; the scheme of Section 2
    commutes with each of them (with omega_qx = omega_qy, alpha_qx = alpha_qy),
    so they hold at every step up to rounding.  Returns the largest violation.
    """
    u, phi, dx = synthetic.taylor_green_2d(n)
    p = oracle.make_params((n, n), dx, nu=0.01)
    f = orc.run(p, orc.init(p, u, phi), nsteps)
    _, (ux, uy), _ = orc.macros(p, f)
    h = n // 2
    viol = [
        np.abs(ux[:, ::-1] + ux), np.abs(uy[:, ::-1] - uy),
        np.abs(ux[::-1, :] - ux), np.abs(uy[::-1, :] + uy),
        np.abs(ux - np.roll(uy.T, h, axis=1)), np.abs(uy - np.roll(ux.T, h, axis=1)),
    ]
    return float(max(v.max() for v in viol))


def init_macros(orc, n=(10, 6), seed=5):
    """Init then moment extraction returns (u, phi), with rho = (1 + dx^2 phi)^(1/gamma)."""
    worst = 0.0
    for gamma in (1.0, 1.4):
        dx = 0.05
        p = _params(n, dx, gamma=gamma)
        rng = np.random.default_rng(seed)
        u = rng.uniform(-1, 1, (2, n[1], n[0]))
        phi = rng.uniform(-3, 3, (n[1], n[0]))
        rho, um, phim = orc.macros(p, orc.init(p, u, phi))
        worst = max(worst, float(np.max(np.abs(um - u))), float(np.max(np.abs(phim - phi))) * dx * dx,
                    float(np.max(np.abs(rho - (1.0 + dx * dx * phi) ** (1.0 / gamma)))))
    return worst


def tgv_error(orc, n, t_final, nu=0.01, omega_rho=1.2, alpha_rho=0.075, omega_q=1.15):
    """L2 error on u_x of the Taylor-Green vortex at step round(t mu / dx^2).

    e2 = (dx^2 sum (u_x - u_x^ex)^2)^(1/2), the exact solution taken at n dt.
    """
    u, phi, dx = synthetic.taylor_green_2d(n)
    p = oracle.make_params((n, n), dx, nu=nu, omega_rho=omega_rho, alpha_rho=alpha_rho, omega_q=omega_q)
    nsteps = int(round(t_final / p.dt))
    f = orc.run(p, orc.init(p, u, phi), nsteps)
    _, um, _ = orc.macros(p, f)
    ue, _, _ = synthetic.taylor_green_2d(n, t=nsteps * p.dt, nu=nu)
    return math.sqrt(dx * dx * float(np.sum((um[0] - ue[0]) ** 2))), float(np.max(np.abs(um - ue)))


def tgv_decay(orc, n=32, t_final=0.2):
    """Max-abs velocity error of a short Taylor-Green run divided by dx^2.

    A second-order scheme keeps this O(1) (about 0.36 here); a wrong term gives
    an O(1) error, i.e. a ratio of order 1/dx^2.
    """
    dx = synthetic.TWO_PI / n
    return tgv_error(orc, n, t_final)[1] / (dx * dx)


FAST_PINS = {
    "shear_wave": shear_wave,
    "one_step": one_step,
    "conservation": conservation,
    "forms": forms,
    "fixed_point": fixed_point,
    "fourier": fourier,
    "symmetry": symmetry,
    "init_macros": init_macros,
    "tgv_decay": tgv_decay,
}


# ------------------------------------------------------------------------- 3D

MIXED3 = dict(mu=8.0, omega=(1.2, 1.3, 1.1, 1.4), alpha=(0.05, 0.02, 0.03, 0.015))


def shear_wave_3d(orc, n=(12, 10, 8), mode=2, nsteps=60, amplitude=0.3):
    """D3Q7: a momentum field varying along one axis follows the 4-state recurrence.

    Every (carrier field j, wave axis d) pair with j != d is checked on a
    non-cubic lattice.
    """
    dx = 0.2
    worst = 0.0
    p = oracle.Params(n=n, dx=dx, **MIXED3)
    grid = tuple(reversed(n))                        # (nz, ny, nx)
    idx = np.meshgrid(*[np.arange(m) for m in grid], indexing="ij")   # z, y, x index arrays
    axis_index = {0: idx[2], 1: idx[1], 2: idx[0]}
    for d in range(3):
        for j in range(3):
            if j == d:
                continue
            u = np.zeros((3,) + grid)
            theta = 2 * math.pi * mode / n[d]
            u[j] = amplitude * np.sin(theta * (axis_index[d] + 0.5))
            f = orc.run(p, orc.init(p, u, np.zeros(grid)), nsteps)
            rho, um, _ = orc.macros(p, f)
            gain = spectral.shear_wave_gain(theta, nsteps, p.omega[j + 1], p.alpha[j + 1], dim=3)
            err = np.max(np.abs(um[j] - u[j] * gain)) / (amplitude * abs(gain))
            others = max(np.max(np.abs(um[i])) for i in range(3) if i != j) / amplitude
            worst = max(worst, err, others, float(np.max(np.abs(rho - 1.0))))
    return worst


def conservation_3d(orc, n=(6, 5, 4), nsteps=20, seed=4):
    """D3Q7 per-step conservation of the four population totals."""
    p = oracle.Params(n=n, dx=0.2, **MIXED3)
    rng = np.random.default_rng(seed)
    grid = tuple(reversed(n))
    f = orc.init(p, rng.uniform(-1, 1, (3,) + grid), rng.uniform(-1, 1, grid)) + 1e-3 * rng.uniform(-1, 1, p.shape())
    tot0 = f.reshape(p.fields, -1).sum(axis=1)
    scale = np.abs(f).reshape(p.fields, -1).sum(axis=1)
    f = orc.run(p, f, nsteps)
    return float(np.max(np.abs(f.reshape(p.fields, -1).sum(axis=1) - tot0) / scale))


def fourier_3d(orc, n=(8, 6, 4), eps=1e-7, nsteps=6):
    """D3Q7 small Fourier modes against the 28 x 28 amplification matrix."""
    dx = 0.05
    p = oracle.Params(n=n, dx=dx, **MIXED3)
    grid = tuple(reversed(n))
    base = (1.05, 0.2, -0.1, 0.3)
    u_b = np.empty((3,) + grid)
    for d in range(3):
        u_b[d] = base[1 + d] / base[0]
    fbar = orc.init(p, u_b, np.full(grid, (base[0] - 1.0) / (dx * dx)))
    iz, iy, ix = np.meshgrid(*[np.arange(m) for m in grid], indexing="ij")
    worst = 0.0
    for m in ((1, 2, 1), (3, 1, 2)):
        theta = tuple(2 * math.pi * m[d] / n[d] for d in range(3))
        E = spectral.amplification_matrix(theta, dx, p.mu, p.omega, p.alpha, base)
        lam, V = np.linalg.eig(E)
        phase = np.exp(1j * (theta[0] * ix + theta[1] * iy + theta[2] * iz))
        for i in range(len(lam)):
            if abs(lam[i]) ** nsteps < 1e-3:
                continue
            v = V[:, i] / np.linalg.norm(V[:, i])
            f0 = fbar + (2 * eps * np.real(v[:, None, None, None] * phase[None])).reshape(p.shape())
            fn = orc.run(p, f0, nsteps)
            expect = fbar + (2 * eps * np.real(lam[i] ** nsteps * v[:, None, None, None] * phase[None])).reshape(p.shape())
            worst = max(worst, float(np.max(np.abs(fn - expect))) / eps)
    return worst


PIN_LIMITS.update({"shear_wave_3d": 1e-12, "conservation_3d": 1e-13, "fourier_3d": 1e-6})
FAST_PINS.update({"shear_wave_3d": shear_wave_3d, "conservation_3d": conservation_3d, "fourier_3d": fourier_3d})


def failing_pins(orc):
    """Names of the fast pins this oracle fails (a crash or NaN counts as failing)."""
    bad = []
    for name, fn in FAST_PINS.items():
        try:
            err = fn(orc)
        except Exception:
            bad.append(name)
            continue
        if not (err <= PIN_LIMITS[name]):
            bad.append(name)
    return bad
