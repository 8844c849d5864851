"""Poiseuille flow in [0, L]^2 with the ghost-cell boundary conditions of Section 6.2.

TEST INFRASTRUCTURE (part of the oracle; imports nothing from the CUDA package).

The interior update is the oracle's own scheme (``Oracle.collide``: the relaxation of
Eq. LBM_scheme on the equilibria of Section 2); this module adds what the periodic
oracle does not have, the boundary treatment of Section 6.2.1, and the Poiseuille setting
of Section 6.2:

* exact steady solution u_x = 4U y (L - y) / L^2, u_y = 0, Phi = 8 nu U (L - x) / L^2,
  nu = U L / Re (L = 1, U = 1, Re = 100);
* conserved moments (rho, q_x, q_y) of ghost cells at distance dx/2 outside each side, from
  the interior cells of the current time:
    left   (x = -dx/2):   rho by linear extrapolation from the cells at dx/2 and 3dx/2, q = 2 rho_bar u_ex(y) - q(dx/2)
    right  (x = L+dx/2):  rho = 2 rho_bar (1 + dx^2 Phi_ex(L)) - rho(L - dx/2), q by linear extrapolation
    lower  (y = -dx/2):   rho by linear extrapolation, q = 2 rho_bar u_ex(0) - q(dx/2)
    upper  (y = L+dx/2):  the same as the lower side
  (Phi_ex(L) = 0; the density-pressure relation P(rho) = P(rho_bar) + dx^2 rho_bar Phi of
  Section 3 with gamma = 1);
* the post-relaxation population that streams from a ghost cell into the domain is its
  equilibrium (Eqs. BCPoiseuilleLeftEquilibrium, BCPoiseuilleRightEquilibrium,
  BCPoiseuilleLowerEquilibrium); with ``corrected`` the lower and upper ones also get the
  non-equilibrium part of the same population at the adjacent interior cell
  (Eq. BCPoiseuilleLowerEquilibriumPlusCorrection).

Populations of a ghost cell that no interior cell pulls (D2Q5 has no diagonal velocities) are
never formed.  One time step: ghost populations from the moments of the current
post-relaxation state, pull transport, relaxation.

Readings where Section 6.2 is silent (listed with the other readings of the paper):
  mu = 8, as for the Taylor-Green vortex; the initial state is the equilibrium of the exact
  solution (rho = rho_bar (1 + dx^2 Phi_ex), q = rho u_ex); n = floor(t mu / dx^2) steps (the
  last time level not after t: at 112 cells, t mu / dx^2 = 5017.6, and 5017 steps reproduce
  all four printed errors of that row while 5018 miss two by more than a printed unit); the
  error is (dx^2 sum (u_x - u_x^ex)^2)^(1/2) over the cell centres.  With these, the oracle
  reproduces all 16 errors of Table 2 (75, 112, 168 and 253 cells) to the four printed digits.
"""
from __future__ import annotations

import math

import numpy as np

from . import Oracle, Params, alpha_from_nu


def exact(n: int, L: float = 1.0, U: float = 1.0, re: float = 100.0, nx: int | None = None):
    """(u (2, n, nx), phi (n, nx), dx, nu) of the steady Poiseuille profile at the cell centres of
    n cells across the channel (height L) and nx (default n) along it (length nx dx)."""
    nx = n if nx is None else nx
    dx = L / n
    nu = U * L / re
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(n) + 0.5) * dx, indexing="xy")
    u = np.stack([4.0 * U * Y * (L - Y) / L ** 2, np.zeros_like(Y)])
    phi = 8.0 * nu * U * (nx * dx - X) / L ** 2
    return u, phi, dx, nu


def params(n: int, omega_q: float, mu: float = 8.0, omega_rho: float = 1.2, alpha_rho: float = 0.075,
           L: float = 1.0, U: float = 1.0, re: float = 100.0, nx: int | None = None) -> Params:
    dx = L / n
    nu = U * L / re
    aq = alpha_from_nu(nu, mu, omega_q)
    return Params(n=(n if nx is None else nx, n), dx=dx, mu=mu, omega=(omega_rho, omega_q, omega_q),
                  alpha=(alpha_rho, aq, aq))


class Poiseuille:
    """Poiseuille flow on n cells across (height L = 1) and nx (default n) along the channel
    (U = 1, Re = 100)."""

    def __init__(self, orc: Oracle, n: int, omega_q: float, corrected: bool = False, mu: float = 8.0,
                 nx: int | None = None):
        self.orc = orc
        self.n = n
        self.nx = n if nx is None else nx
        self.p = params(n, omega_q, mu=mu, nx=nx)
        self.corrected = corrected
        u, phi, dx, nu = exact(n, nx=nx)
        self.u_ex, self.dx, self.nu = u, dx, nu
        self.rho_bar = self.p.rho_bar
        self.uex_y = u[0][:, 0]                 # u_x^ex at the cell centres' y (the left side's profile)
        self.f = orc.collide(self.p, orc.init(self.p, u, phi))     # post-relaxation state at t = 0
        self.steps = 0

    def _moments(self, f):
        rho, u, _ = self.orc.macros(self.p, f)
        return rho, u[0] * rho, u[1] * rho

    def _equilibria(self, rho, qx, qy):
        """Equilibria (3, 5, m) of m ghost cells from their conserved moments."""
        m = rho.size
        g = Params(n=(m, 1), dx=self.p.dx, mu=self.p.mu, omega=self.p.omega, alpha=self.p.alpha,
                   gamma=self.p.gamma, rho_bar=self.p.rho_bar)
        u = np.stack([qx / rho, qy / rho]).reshape(2, 1, m)
        phi = ((rho ** g.gamma - g.rho_bar ** g.gamma) / (g.dx ** 2 * g.rho_bar)).reshape(1, m)
        return self.orc.init(g, u, phi)[:, :, 0, :]

    def step(self, count: int = 1) -> None:
        ny, nx, rb, dx = self.n, self.nx, self.rho_bar, self.dx
        for _ in range(count):
            f = self.f
            rho, qx, qy = self._moments(f)                       # (ny, nx): [y, x]
            F = np.zeros((3, 5, ny + 2, nx + 2))
            F[:, :, 1:-1, 1:-1] = f
            # left side (x = -dx/2): the +x populations enter
            e = self._equilibria(2 * rho[:, 0] - rho[:, 1], 2 * rb * self.uex_y - qx[:, 0], -qy[:, 0])
            F[:, 1, 1:-1, 0] = e[:, 1, :]
            # right side (x = L + dx/2): the -x populations enter (Phi_ex(L) = 0)
            e = self._equilibria(2 * rb * (1.0 + dx * dx * 0.0) - rho[:, -1], 2 * qx[:, -1] - qx[:, -2],
                                 2 * qy[:, -1] - qy[:, -2])
            F[:, 2, 1:-1, -1] = e[:, 2, :]
            # lower side (y = -dx/2): the +y populations enter (u_ex = 0 on the wall)
            e = self._equilibria(2 * rho[0, :] - rho[1, :], -qx[0, :], -qy[0, :])
            low = e[:, 3, :]
            # upper side (y = L + dx/2): the -y populations enter
            e = self._equilibria(2 * rho[-1, :] - rho[-2, :], -qx[-1, :], -qy[-1, :])
            up = e[:, 4, :]
            if self.corrected:
                # non-equilibrium part of the same population at the adjacent interior cell
                e0 = self._equilibria(rho[0, :], qx[0, :], qy[0, :])
                e1 = self._equilibria(rho[-1, :], qx[-1, :], qy[-1, :])
                low = low + (f[:, 3, 0, :] - e0[:, 3, :])
                up = up + (f[:, 4, -1, :] - e1[:, 4, :])
            F[:, 3, 0, 1:-1] = low
            F[:, 4, -1, 1:-1] = up
            # pull transport: velocity l at x takes F_l(x - c_l)
            g = np.empty_like(f)
            g[:, 0] = F[:, 0, 1:-1, 1:-1]
            g[:, 1] = F[:, 1, 1:-1, 0:-2]
            g[:, 2] = F[:, 2, 1:-1, 2:]
            g[:, 3] = F[:, 3, 0:-2, 1:-1]
            g[:, 4] = F[:, 4, 2:, 1:-1]
            self.f = self.orc.collide(self.p, g)
            self.steps += 1

    def run_to(self, t: float) -> int:
        """Advance by the whole steps that fit in t (n = floor(t mu / dx^2): the last time
        level not after t); returns the step count."""
        n_steps = int(math.floor(t * self.p.mu / self.dx ** 2 + 1e-6))
        self.step(n_steps - self.steps)
        return n_steps

    def l2_error_ux(self) -> float:
        _, u, _ = self.orc.macros(self.p, self.f)
        return math.sqrt(self.dx ** 2 * float(np.sum((u[0] - self.u_ex[0]) ** 2)))
