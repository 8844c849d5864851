"""Linearised amplification matrix of the vectorial scheme (Section 5 of the paper).

TEST INFRASTRUCTURE (numpy only; independent of the CUDA path).

For a base state (rho_b, q_b) and a pressure law P(rho) = rho^gamma (Section 5
uses gamma = 1), a Fourier mode f(x) = f_hat exp(i xi . x) of the scheme's
populations is advanced by one time step through

    f_hat(t + dt) = E(xi dx) f_hat(t),   E = S(xi dx) C,

with C the Jacobian of the relaxation of Eq. LBM_scheme,
    C = (I - Omega) + Omega J M,
M the map from populations to conserved moments (rho = sum f^rho,
q_d = sum f^{q_d} / dx), J the Jacobian of the equilibria of Section 2 with
respect to (rho, q), Omega = diag(omega_k) per field, and S the transport
phases: the population moving along s e_d picks up exp(-i s theta_d).
Populations are ordered field-major, velocity-minor (k * Q + l) with the
velocity order rest, +x, -x, +y, -y(, +z, -z), the same as the oracle.

J is written out from the equilibria by hand (derivatives of each printed
entry), so this module shares no code with vlbm_oracle.c.  It is pinned by
Lemma 1 (characteristic polynomial at the checkerboard mode) and by Lemma 2
(low-frequency eigenvalues of the relaxation scheme).
"""
from __future__ import annotations

import numpy as np


def equilibrium_jacobian(dim, dx, mu, alpha, rho_b, q_b, gamma=1.0):
    """d f^eq / d (rho, q_1..q_d) at (rho_b, q_b); shape (F*Q, F)."""
    Q = 2 * dim + 1
    F = dim + 1
    c = dx * dx / (2.0 * mu)
    dP = gamma * rho_b ** (gamma - 1.0)          # P'(rho)
    J = np.zeros((F * Q, F))
    # field rho: rest (1 - 2 d alpha) rho; direction s e_d: alpha rho + s dx/(2mu) q_d
    J[0, 0] = 1.0 - 2.0 * dim * alpha[0]
    for d in range(dim):
        for s, l in ((+1.0, 1 + 2 * d), (-1.0, 2 + 2 * d)):
            J[l, 0] = alpha[0]
            J[l, 1 + d] = s * dx / (2.0 * mu)
    # field q_j: rest dx (1 - 2 d alpha_j) q_j;
    # direction s e_d: dx alpha_j q_j + s (c q_j q_d / rho + delta_jd P(rho) / (2 mu))
    for j in range(dim):
        row0 = (j + 1) * Q
        aj = alpha[j + 1]
        J[row0, 1 + j] = dx * (1.0 - 2.0 * dim * aj)
        for d in range(dim):
            for s, l in ((+1.0, 1 + 2 * d), (-1.0, 2 + 2 * d)):
                r = row0 + l
                J[r, 1 + j] += dx * aj
                J[r, 0] += s * (-c * q_b[j] * q_b[d] / rho_b ** 2 + (dP / (2.0 * mu) if j == d else 0.0))
                J[r, 1 + j] += s * c * q_b[d] / rho_b
                J[r, 1 + d] += s * c * q_b[j] / rho_b
    return J


def moment_map(dim, dx):
    """M: populations -> (rho, q_1..q_d); shape (F, F*Q)."""
    Q = 2 * dim + 1
    F = dim + 1
    M = np.zeros((F, F * Q))
    M[0, :Q] = 1.0
    for j in range(dim):
        M[1 + j, (j + 1) * Q:(j + 2) * Q] = 1.0 / dx
    return M


def collision_matrix(dim, dx, mu, omega, alpha, rho_b, q_b, gamma=1.0):
    Q = 2 * dim + 1
    F = dim + 1
    Om = np.diag(np.repeat(np.asarray(omega[:F], dtype=np.float64), Q))
    J = equilibrium_jacobian(dim, dx, mu, alpha, rho_b, q_b, gamma)
    M = moment_map(dim, dx)
    return np.eye(F * Q) - Om + Om @ J @ M


def transport_phases(dim, theta):
    """Diagonal of S: exp(-i s theta_d) for the population moving along s e_d."""
    Q = 2 * dim + 1
    ph = np.ones(Q, dtype=np.complex128)
    for d in range(dim):
        ph[1 + 2 * d] = np.exp(-1j * theta[d])
        ph[2 + 2 * d] = np.exp(+1j * theta[d])
    return np.tile(ph, dim + 1)


def amplification_matrix(theta, dx, mu, omega, alpha, base=(1.0, 0.0, 0.0), gamma=1.0):
    """E(theta) for theta = (xi_x dx, xi_y dx[, xi_z dx]); base = (rho_b, q_b...)."""
    dim = len(theta)
    rho_b = float(base[0])
    q_b = np.zeros(dim)
    q_b[: len(base) - 1] = base[1:1 + dim]
    C = collision_matrix(dim, dx, mu, omega, alpha, rho_b, q_b, gamma)
    return transport_phases(dim, theta)[:, None] * C


def checkerboard_charpoly(z, omega, alpha):
    """Lemma 1: prod_i (z - omega_i + 1)^3 (z^2 - omega_i (1 - 8 alpha_i) z + omega_i - 1), 2D."""
    out = np.ones_like(np.asarray(z, dtype=np.complex128))
    for w, a in zip(omega[:3], alpha[:3]):
        out = out * (z - w + 1.0) ** 3 * (z * z - w * (1.0 - 8.0 * a) * z + w - 1.0)
    return out


def shear_wave_gain(theta, nsteps, omega_q, alpha_q, dim=2):
    """Amplitude factor of an exact shear wave after nsteps.

    A momentum field that varies along one axis only, with rho = rho_bar and the
    other momenta zero, is carried by the linear 4-state recurrence on
    (f_0, f_+, f_-, s) of that field, s being the sum of the populations that
    move across the wave (uniform along their direction, so transport leaves
    them in place): relaxation C = (1 - w) I + w v 1^T with
    v = (1 - 2 d a, a, a, 2 (d - 1) a) and transport phases
    (1, e^{-i theta}, e^{i theta}, 1).  The gain is 1^T (S C)^n v (real).
    """
    v = np.array([1.0 - 2.0 * dim * alpha_q, alpha_q, alpha_q, 2.0 * (dim - 1) * alpha_q])
    C = (1.0 - omega_q) * np.eye(4) + omega_q * np.outer(v, np.ones(4))
    S = np.diag([1.0, np.exp(-1j * theta), np.exp(1j * theta), 1.0])
    G = np.linalg.matrix_power(S @ C, nsteps)
    return float(np.real(np.ones(4) @ G @ v))
