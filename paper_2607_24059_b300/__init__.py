"""B300-native vectorial lattice Boltzmann scheme for incompressible Navier-Stokes.

The scheme (Aregba-Driollet, Bellotti, Natalini, Tenna, Section 2): every
conserved field (rho, q_x, q_y[, q_z]) carries its own D2Q5 (3D: D3Q7)
population set, relaxes toward its own equilibrium with its own omega, and
streams on a periodic Cartesian lattice, with dt = dx^2 / mu.

The compute path is the C-ABI library libvlbm.so (include/vlbm.h) built from
hand-written sm_103a CUDA kernels; this package only binds it.  `Lattice` is a
convenience wrapper over the same calls.
"""
from __future__ import annotations

from . import _binding
from ._binding import *  # noqa: F401,F403  (the C ABI, same names)
from ._binding import VlbmError, PRECISIONS

__all__ = list(_binding.EXPORTED) + ["Lattice", "Batch", "Surrogate", "VlbmError", "PRECISIONS"]


class Lattice:
    """One periodic lattice on the current CUDA device (a vlbm handle).

    Parameters follow vlbm_params; `n` is (nx, ny) or (nx, ny, nz).  Arrays
    come back as torch tensors on `device` (default: the current CUDA device).
    """

    def __init__(self, n, dx, nu, precision="fp32", mu=8.0, omega_rho=1.2, alpha_rho=0.075, omega_q=1.15,
                 alpha_q=None, gamma=1.0, rho_bar=1.0, strict=False, stream=None):
        import torch
        self._torch = torch
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p = _binding.vlbm_params_default(self.dim, self.n, dx, nu, prec)
        p.mu = mu
        p.omega[0] = omega_rho
        p.alpha[0] = alpha_rho
        for k in range(1, 4):
            p.omega[k] = omega_q
            p.alpha[k] = -1.0 if alpha_q is None else alpha_q
        p.gamma = gamma
        p.rho_bar = rho_bar
        p.strict = int(bool(strict))
        self.params = p
        _, self.derived = _binding.vlbm_params_check(p)
        self.handle = _binding.vlbm_create(p, stream)
        self.grid = tuple(reversed(self.n))

    # -- lifecycle
    def close(self):
        if getattr(self, "handle", None):
            _binding.vlbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the scheme
    def init(self, u, phi=None):
        _binding.vlbm_init(self.handle, u, phi)

    def step(self, nsteps=1, check=False, graph=True):
        flags = (_binding.VLBM_STEP_CHECK_FINITE if check else 0) | (0 if graph else _binding.VLBM_STEP_NO_GRAPH)
        _binding.vlbm_step(self.handle, nsteps, flags)

    def step_record(self, nsteps, every=1, history=None):
        """Step with the invariants of every `every`-th state reduced in the step kernel."""
        return _binding.vlbm_step_record(self.handle, nsteps, every, history)

    def macros(self, dtype=None, device="cuda"):
        """(rho, u, phi) as tensors."""
        t = self._torch
        dtype = dtype or t.float64
        rho = t.empty(self.grid, dtype=dtype, device=device)
        u = t.empty((self.dim,) + self.grid, dtype=dtype, device=device)
        phi = t.empty(self.grid, dtype=dtype, device=device)
        _binding.vlbm_macros(self.handle, rho, u, phi)
        return rho, u, phi

    def invariants(self):
        return _binding.vlbm_invariants(self.handle)

    def vorticity_sq(self):
        """Sum over nodes of |curl u|^2 dx^d (centred differences): -dE/dt = nu times this."""
        return _binding.vlbm_vorticity_sq(self.handle)

    def populations(self, deviation=False, dtype=None, device="cuda"):
        t = self._torch
        q = 2 * self.dim + 1
        out = t.empty((self.dim + 1, q) + self.grid, dtype=dtype or t.float64, device=device)
        _binding.vlbm_get_populations(self.handle, out, deviation)
        return out

    def time(self):
        return _binding.vlbm_time(self.handle)

    def state(self):
        return _binding.vlbm_get_state(self.handle)

    def load_state(self, blob):
        _binding.vlbm_set_state(self.handle, blob)

    def set_option(self, key, value):
        _binding.vlbm_set_option(self.handle, key, value)

    def set_channel(self, u_in, phi_out=0.0, wall_correction=False):
        """Ghost-cell channel boundaries of Section 6.2.1 (2D, FP64/FP32): inflow velocity u_in(y)
        on the left, pressure potential phi_out on the right, no-slip walls below and above."""
        _binding.vlbm_set_boundary(self.handle, _binding.VLBM_BC_CHANNEL, u_in, phi_out, wall_correction)

    def set_periodic(self):
        _binding.vlbm_set_boundary(self.handle, _binding.VLBM_BC_PERIODIC)

    def launch_count(self):
        return _binding.vlbm_launch_count(self.handle)


class Batch:
    """Many independent periodic 2D problems advanced together (a vlbm_batch).

    problems: sequence of dicts with keys n=(nx, ny), dx, nu and optionally
    mu, omega_rho, alpha_rho, omega_q, alpha_q, gamma, rho_bar.
    """

    def __init__(self, problems, precision="fp16split", stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        plist = []
        for q in problems:
            n = tuple(int(v) for v in q["n"])
            p = _binding.vlbm_params_default(2, n, q["dx"], q["nu"], prec)
            p.mu = q.get("mu", 8.0)
            p.omega[0] = q.get("omega_rho", 1.2)
            p.alpha[0] = q.get("alpha_rho", 0.075)
            for k in range(1, 4):
                p.omega[k] = q.get("omega_q", 1.15)
                p.alpha[k] = q.get("alpha_q", -1.0) if q.get("alpha_q") is not None else -1.0
            p.gamma = q.get("gamma", 1.0)
            p.rho_bar = q.get("rho_bar", 1.0)
            plist.append(p)
        self.params = plist
        self.shapes = [tuple(reversed(tuple(int(v) for v in q["n"]))) for q in problems]
        self.handle = _binding.vlbm_batch_create(plist, stream)

    def close(self):
        if getattr(self, "handle", None):
            _binding.vlbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, problem, u, phi=None):
        _binding.vlbm_batch_init(self.handle, problem, u, phi)

    def step(self, nsteps=1, graph=True, persistent=False):
        """persistent: all nsteps in one cooperative launch (synchronises; VlbmError on a barrier timeout)."""
        flags = (0 if graph else _binding.VLBM_STEP_NO_GRAPH) | (_binding.VLBM_STEP_PERSISTENT if persistent else 0)
        _binding.vlbm_batch_step(self.handle, nsteps, flags)

    def velocity(self, problem, dtype=None, device="cuda"):
        import torch
        u = torch.empty((2,) + self.shapes[problem], dtype=dtype or torch.float64, device=device)
        _binding.vlbm_batch_macros(self.handle, problem, None, u, None)
        return u

    def invariants(self, problem):
        return _binding.vlbm_batch_invariants(self.handle, problem)

    def autotune(self, repeats=5):
        return _binding.vlbm_batch_autotune(self.handle, repeats)

    def set_config(self, threads, blocks_per_sm, lanes=4):
        _binding.vlbm_batch_set_config(self.handle, threads, blocks_per_sm, lanes)

    def info(self):
        return _binding.vlbm_batch_info(self.handle)


class Surrogate:
    """The learned surrogate (a vlbm_sur; an extension the paper has no counterpart for): five
    periodic 3x3 convolutions with 64 hidden channels and GELU, BF16 weights and activations, FP32
    accumulation, trained with Adam.

    States are (B, channels, H, W) FP32 CUDA tensors.  With divergence_input the network also
    reads in_scale[channels] times the divergence of channels 0, 1; with curl_output its channel 0
    is a stream function whose central-difference curl is the velocity increment (divergence-free
    in those differences).  forward(u) = net(in_scale u);
    advance(u) = u + out_scale net(in_scale u); train_step(u, target, lr) takes one Adam step on
    the mean squared error of net(in_scale u) against target (an increment divided by out_scale).
    """

    LAYERS = ((16, 64), (64, 64), (64, 64), (64, 64), (64, 16))

    def __init__(self, H, W, max_batch, channels=2, divergence_input=False, curl_output=False, seed=0, stream=None):
        self.H, self.W, self.max_batch, self.channels = int(H), int(W), int(max_batch), int(channels)
        self.curl_output = bool(curl_output)
        features = (_binding.VLBM_SUR_FEATURE_DIV if divergence_input else 0) | \
            (_binding.VLBM_SUR_FEATURE_CURL if curl_output else 0)
        self.inputs = self.channels + (1 if divergence_input else 0)
        self.handle = _binding.vlbm_sur_create(self.H, self.W, self.channels, features, self.max_batch, int(seed),
                                               stream)
        self.num_params = _binding.vlbm_sur_num_params(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _binding.vlbm_sur_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scaling(self, in_scale=None, out_scale=None):
        _binding.vlbm_sur_set_scaling(self.handle, in_scale, out_scale)

    def set_train_noise(self, sigma=None, seed=0):
        """Gaussian noise (std per input channel, in scaled-input units) added to training inputs."""
        _binding.vlbm_sur_set_train_noise(self.handle, sigma, seed)

    def _check_fields(self, u):
        if u.dtype.itemsize != 4 or not u.is_cuda or not u.is_contiguous() or u.dim() != 4 \
                or tuple(u.shape[1:]) != (self.channels, self.H, self.W) or not 1 <= u.shape[0] <= self.max_batch:
            raise ValueError(f"expected contiguous float32 CUDA states (B <= {self.max_batch}, {self.channels}, "
                             f"{self.H}, {self.W})")

    def forward(self, u, out=None):
        import torch
        self._check_fields(u)
        du = torch.empty_like(u) if out is None else out
        _binding.vlbm_sur_forward(self.handle, u, du, u.shape[0])
        return du

    def advance(self, u, out=None):
        """u + out_scale * net(in_scale * u) (out may be u itself)."""
        import torch
        self._check_fields(u)
        nxt = torch.empty_like(u) if out is None else out
        _binding.vlbm_sur_advance(self.handle, u, nxt, u.shape[0])
        return nxt

    def increment(self, u, out=None):
        """advance(u) - u, computed directly (out must not be u)."""
        import torch
        self._check_fields(u)
        du = torch.empty_like(u) if out is None else out
        _binding.vlbm_sur_increment(self.handle, u, du, u.shape[0])
        return du

    def train_step(self, u, target, lr, want_loss=True):
        self._check_fields(u)
        self._check_fields(target)
        return _binding.vlbm_sur_train_step(self.handle, u, target, u.shape[0], float(lr), want_loss)

    def params(self, device="cuda"):
        import torch
        p = torch.empty(self.num_params, dtype=torch.float32, device=device)
        _binding.vlbm_sur_get_params(self.handle, p)
        return p

    def grads(self, device="cuda"):
        import torch
        g = torch.empty(self.num_params, dtype=torch.float32, device=device)
        _binding.vlbm_sur_get_grads(self.handle, g)
        return g

    def load_params(self, p):
        import torch
        p = p.to(torch.float32).contiguous()
        if p.numel() != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters")
        _binding.vlbm_sur_set_params(self.handle, p)

    def status(self):
        _binding.vlbm_sur_status(self.handle)

    @classmethod
    def split_params(cls, p):
        """Views (W (cout, 9, cin), bias (cout,)) per layer of a flat parameter vector."""
        out, off = [], 0
        for cin, cout in cls.LAYERS:
            nw = cout * 9 * cin
            out.append((p[off:off + nw].view(cout, 9, cin), p[off + nw:off + nw + cout]))
            off += nw + cout
        return out
