"""FP64 CPU oracle of the vectorial lattice Boltzmann scheme (Section 2 of the paper).

TEST INFRASTRUCTURE.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2607_24059_b300``) and imports nothing from it.

The arithmetic lives in ``vlbm_oracle.c`` (plain loops, FP64, no FP
contraction); this module only marshals numpy arrays through ctypes.
``spectral.py`` holds the linearised amplification matrix of Section 5.

Parity status of each function (what pins it, see tests/test_oracle_pins.py):
  equilibrium / collide (both forms) / stream / run / init / macros:
      pinned by the exact shear-wave recurrence, the one-step closed form,
      per-step conservation, the fixed point, agreement of the two collision
      forms, Fourier-mode decay against the pinned spectrum, and the
      Taylor-Green closed-form decay with second-order convergence (Table 1),
      and by Table 2: with the ghost-cell boundaries of Section 6.2.1
      (poiseuille.py) the scheme reproduces the printed Poiseuille errors to
      their four digits.
  invariants: pinned by direct sums on hand-built states.
  3D (D3Q7, reading R4 in vlbm_oracle.c): pinned by the shear-wave
      recurrence for every carrier-field / axis pair, conservation, Fourier
      modes against the 28 x 28 amplification matrix, and agreement of the
      two relaxation forms.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

COLLIDE_POPULATIONS = 0
COLLIDE_MOMENTS = 1


class _CParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_long * 3),
        ("dx", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("rho_bar", ctypes.c_double),
        ("omega", ctypes.c_double * 4),
        ("alpha", ctypes.c_double * 4),
    ]


def alpha_from_nu(nu: float, mu: float, omega: float) -> float:
    """Viscosity relation of Prop. 1: nu = 2 mu alpha (1/omega - 1/2)."""
    return nu / (2.0 * mu * (1.0 / omega - 0.5))


@dataclass
class Params:
    """Scheme parameters (Section 2; defaults from Section 6.1, Eq. params).

    omega/alpha are per field (rho, q_x, q_y[, q_z]).
    """
    n: tuple
    dx: float
    mu: float = 8.0
    omega: tuple = (1.2, 1.15, 1.15, 1.15)
    alpha: tuple = (0.075, 0.0, 0.0, 0.0)
    gamma: float = 1.0
    rho_bar: float = 1.0

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def q(self) -> int:
        return 5 if self.dim == 2 else 7

    @property
    def fields(self) -> int:
        return self.dim + 1

    @property
    def nodes(self) -> int:
        return int(np.prod(self.n))

    @property
    def dt(self) -> float:
        return self.dx * self.dx / self.mu

    def shape(self):
        """Lattice array shape (fields, Q, [nz,] ny, nx)."""
        return (self.fields, self.q) + tuple(reversed(self.n))

    def to_c(self) -> _CParams:
        c = _CParams()
        c.dim = self.dim
        for i in range(3):
            c.n[i] = int(self.n[i]) if i < self.dim else 1
        c.dx, c.mu, c.gamma, c.rho_bar = self.dx, self.mu, self.gamma, self.rho_bar
        for k in range(4):
            c.omega[k] = float(self.omega[k]) if k < len(self.omega) else 1.0
            c.alpha[k] = float(self.alpha[k]) if k < len(self.alpha) else 0.0
        return c


def make_params(n, dx, nu, mu=8.0, omega_rho=1.2, alpha_rho=0.075, omega_q=1.15, gamma=1.0, rho_bar=1.0):
    """Params with every momentum field sharing omega_q and alpha_q from nu (Prop. 1)."""
    dim = len(n)
    aq = alpha_from_nu(nu, mu, omega_q)
    return Params(n=tuple(int(v) for v in n), dx=dx, mu=mu,
                  omega=(omega_rho,) + (omega_q,) * dim,
                  alpha=(alpha_rho,) + (aq,) * dim, gamma=gamma, rho_bar=rho_bar)


_D = ctypes.POINTER(ctypes.c_double)


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class Oracle:
    """ctypes front of one compiled copy of vlbm_oracle.c."""

    def __init__(self, lib_path: str | None = None):
        path = lib_path or _build.build()
        self.path = path
        self.lib = ctypes.CDLL(path)
        L = self.lib
        P = ctypes.POINTER(_CParams)
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_equilibrium.argtypes = [P, ctypes.c_double, _D, _D]
        L.orc_collide_nodes.argtypes = [P, ctypes.c_long, _D, _D, ctypes.c_int]
        L.orc_collide_lattice.argtypes = [P, _D, _D, ctypes.c_int]
        L.orc_stream.argtypes = [P, _D, _D]
        L.orc_run.argtypes = [P, _D, _D, ctypes.c_long, ctypes.c_int]
        L.orc_init.argtypes = [P, _D, _D, _D]
        L.orc_macros.argtypes = [P, _D, _D, _D, _D]
        L.orc_invariants.argtypes = [P, _D, _D]

    def num_threads(self) -> int:
        return int(self.lib.orc_num_threads())

    def set_num_threads(self, n: int) -> None:
        """Threads of the OpenMP loops (timing only; results do not depend on it)."""
        self.lib.orc_set_num_threads(int(n))

    def equilibrium(self, p: Params, rho: float, q) -> np.ndarray:
        c = p.to_c()
        qa = np.zeros(3, dtype=np.float64)
        qa[: p.dim] = q
        out = np.zeros(p.fields * p.q, dtype=np.float64)
        self.lib.orc_equilibrium(ctypes.byref(c), float(rho), _ptr(qa), _ptr(out))
        return out.reshape(p.fields, p.q)

    def collide_nodes(self, p: Params, f_nodes: np.ndarray, form: int = COLLIDE_POPULATIONS) -> np.ndarray:
        """Relax an array of node population vectors, shape (count, fields, Q)."""
        f = np.ascontiguousarray(f_nodes, dtype=np.float64).reshape(-1, p.fields * p.q)
        out = np.empty_like(f)
        self.lib.orc_collide_nodes(ctypes.byref(p.to_c()), f.shape[0], _ptr(f), _ptr(out), form)
        return out.reshape(-1, p.fields, p.q)

    def collide(self, p: Params, f: np.ndarray, form: int = COLLIDE_POPULATIONS) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == p.shape()
        out = np.empty_like(f)
        self.lib.orc_collide_lattice(ctypes.byref(p.to_c()), _ptr(f), _ptr(out), form)
        return out

    def stream(self, p: Params, fs: np.ndarray) -> np.ndarray:
        fs = np.ascontiguousarray(fs, dtype=np.float64)
        assert fs.shape == p.shape()
        out = np.empty_like(fs)
        self.lib.orc_stream(ctypes.byref(p.to_c()), _ptr(fs), _ptr(out))
        return out

    def run(self, p: Params, f: np.ndarray, nsteps: int, form: int = COLLIDE_POPULATIONS) -> np.ndarray:
        """Advance a copy of f by nsteps (relax then transport); returns it."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        assert f.shape == p.shape()
        work = np.empty_like(f)
        self.lib.orc_run(ctypes.byref(p.to_c()), _ptr(f), _ptr(work), int(nsteps), form)
        return f

    def run_inplace(self, p: Params, f: np.ndarray, work: np.ndarray, nsteps: int,
                    form: int = COLLIDE_POPULATIONS) -> None:
        """Advance f itself by nsteps; work is scratch of f's shape (no copies)."""
        assert f.shape == p.shape() and work.shape == p.shape()
        self.lib.orc_run(ctypes.byref(p.to_c()), _ptr(f), _ptr(work), int(nsteps), form)

    def init(self, p: Params, u: np.ndarray, phi: np.ndarray | None = None) -> np.ndarray:
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (p.dim,) + tuple(reversed(p.n))
        f = np.empty(p.shape(), dtype=np.float64)
        if phi is None:
            self.lib.orc_init(ctypes.byref(p.to_c()), _ptr(u), None, _ptr(f))
        else:
            phi = np.ascontiguousarray(phi, dtype=np.float64)
            self.lib.orc_init(ctypes.byref(p.to_c()), _ptr(u), _ptr(phi), _ptr(f))
        return f

    def macros(self, p: Params, f: np.ndarray):
        """Returns (rho, u, phi)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        grid = tuple(reversed(p.n))
        rho = np.empty(grid)
        u = np.empty((p.dim,) + grid)
        phi = np.empty(grid)
        self.lib.orc_macros(ctypes.byref(p.to_c()), _ptr(f), _ptr(rho), _ptr(u), _ptr(phi))
        return rho, u, phi

    def invariants(self, p: Params, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(8)
        self.lib.orc_invariants(ctypes.byref(p.to_c()), _ptr(f), _ptr(out))
        return out


_default: Oracle | None = None


def default() -> Oracle:
    """The oracle built from the committed source (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default
