"""The learned surrogate, an extension the paper has no counterpart for: data
from the scheme, training, and a checked rollout with the plain scheme as its
fallback.

The surrogate advances a coarse state by K fine lattice steps,
s(t + K dt) = s(t) + S net(s(t) / R), where s = (u_x, u_y, phi) holds the
pooled velocity and the pooled pressure potential phi of the scheme, net is the
five-layer periodic convolutional network of `Surrogate`, and R and S are the
per-channel RMS of the states and of their increments in the training data.
The pressure potential is part of the state because the scheme's velocity alone
does not determine its future: a fine lattice restarted from (u, phi) repeats
its trajectory to rounding, one restarted from (u, 0) does not.

The data are the scheme's own: fine-lattice runs from seeded divergence-free
random Fourier fields, past a warm-up in which phi settles from its initial
zero, average-pooled by a fixed factor every K steps.  During a rollout each
surrogate step is checked (kinetic-energy change per step and since the start,
divergence relative to the gradient); a state that fails is advanced instead
by the plain scheme on the coarse lattice, started from (u, phi), whose step is
factor^2 fine steps long (dt = dx^2 / mu), so K / factor^2 coarse steps.

Every array operation on this path is one of the library's kernels (lattice
steps and macros, pooling, pair gathering, the network's forward, backward and
Adam, field statistics, the rollout check and error norms); torch only provides
device memory, and the host runs the loops and draws the minibatch indices.  The
fallback decisions are taken on the device, so a rollout has no host round trip
between its steps.
"""
from __future__ import annotations

import math
import time
from dataclasses import asdict, dataclass

import numpy as np
import torch

from . import _binding as B
from . import Batch, Lattice, Surrogate


@dataclass
class Config:
    fine: int = 1024                  # side of the fine lattice the data come from
    factor: int = 4                   # pooling factor: coarse side = fine / factor
    nu: float = 1e-3                  # one viscosity for every run, so the map depends on u alone
    k_fine: int = 32                  # fine lattice steps per surrogate step
    warmup: int = 20                  # surrogate steps run before the first snapshot (phi settles)
    channels: int = 3                 # u_x, u_y, phi
    divergence_input: bool = False    # FP32 divergence of u as an extra input channel (rollouts go unstable)
    curl_output: bool = False         # velocity increment = curl of a predicted stream function (no
                                      # divergence fallbacks, but unstable past ~40 steps when fully trained)
    phi_weight: float = 0.1           # weight of the phi channel in the training loss
    noise_u: float = 0.0              # training-input noise (std, scaled units): velocity channels
    noise_phi: float = 0.0            # ... phi channel
    noise_div: float = 0.3            # ... divergence channel
    train_trajectories: int = 200
    pairs_per_trajectory: int = 100   # 200 x 100 = 20k training pairs
    test_trajectories: int = 8
    rollout_steps: int = 100
    seed_base: int = 20261203         # fields: seed_base + i (training), seed_base + 100000 + i (test)
    batch: int = 32
    epochs: float = 8.0
    lr: float = 1e-3
    lr_min: float = 2e-5
    net_seed: int = 1
    energy_step_tol: float = 2e-3     # |E_{k+1} / E_k - 1| allowed per surrogate step
    energy_drift_tol: float = 5e-2    # |E_k / E_0 - 1| allowed over the rollout
    div_factor: float = 1.5           # divergence / gradient ratio allowed: div_factor times the largest
    div_floor: float = 1e-3           # ratio of the training states (at least div_floor)

    @property
    def coarse(self) -> int:
        return self.fine // self.factor

    @property
    def coarse_steps(self) -> int:
        """Coarse lattice steps per surrogate step (dt scales with dx^2)."""
        q, r = divmod(self.k_fine, self.factor * self.factor)
        if r or q < 1:
            raise ValueError("k_fine must be a positive multiple of factor^2")
        return q

    def train_seeds(self):
        return [self.seed_base + i for i in range(self.train_trajectories)]

    def test_seeds(self):
        return [self.seed_base + 100000 + i for i in range(self.test_trajectories)]


def initial_field(side: int, seed: int) -> np.ndarray:
    """Seeded divergence-free random Fourier velocity (2, side, side), unit RMS, FP64."""
    import synthetic
    u, _, _ = synthetic.random_fourier_field(side, seed)
    return u


def generate(cfg: Config, seeds, steps: int, device="cuda", precision="fp32") -> torch.Tensor:
    """Pooled states (len(seeds), steps + 1, C, c, c) FP32 of fine-lattice runs, one every k_fine
    steps after `warmup` surrogate steps; channels u_x, u_y (and phi when C = 3)."""
    f, c, C = cfg.fine, cfg.coarse, cfg.channels
    out = torch.empty(len(seeds), steps + 1, C, c, c, dtype=torch.float32, device=device)
    lat = Lattice((f, f), 2 * math.pi / f, cfg.nu, precision=precision)
    ufine = torch.empty(2, f, f, dtype=torch.float32, device=device)
    pfine = torch.empty(1, f, f, dtype=torch.float32, device=device)
    try:
        for i, seed in enumerate(seeds):
            lat.init(torch.from_numpy(initial_field(f, seed)).to(device))
            if cfg.warmup:
                lat.step(cfg.warmup * cfg.k_fine)
            for k in range(steps + 1):
                if k:
                    lat.step(cfg.k_fine)
                B.vlbm_macros(lat.handle, None, ufine, pfine if C > 2 else None)
                B.vlbm_field_pool(ufine, out[i, k, 0:2].unsqueeze(0), cfg.factor)
                if C > 2:
                    B.vlbm_field_pool(pfine, out[i, k, 2:3].unsqueeze(0), cfg.factor)
        torch.cuda.synchronize()
    finally:
        lat.close()
    return out


def pair_starts(snaps: torch.Tensor) -> np.ndarray:
    """Flat indices (into snaps viewed as (T (P + 1), 2, c, c)) of every pair's first snapshot."""
    T, P1 = snaps.shape[:2]
    return (np.arange(T)[:, None] * P1 + np.arange(P1 - 1)[None, :]).ravel().astype(np.int64)


def channel_rms(snaps: torch.Tensor, increments: bool, chunk: int = 256) -> list:
    """Per-channel RMS over every pair of the store: of the states (increments=False) or of
    u_{k+1} - u_k (increments=True)."""
    T, P1, C, c, _ = snaps.shape
    flat = snaps.view(T * P1, C, c, c)
    starts = pair_starts(snaps)
    u = torch.empty(chunk, C, c, c, dtype=torch.float32, device=snaps.device)
    d = torch.empty_like(u)
    zero = torch.zeros(chunk * C, c, c, dtype=torch.float32, device=snaps.device)
    nrm = torch.empty(chunk * C, 2, dtype=torch.float64, device=snaps.device)
    idx = torch.from_numpy(starts).to(snaps.device)
    total = np.zeros(C)
    for i in range(0, len(starts), chunk):
        n = min(chunk, len(starts) - i)
        B.vlbm_sur_gather_pairs(flat, idx[i:i + n], u[:n], d[:n], [1.0] * C)
        src = d if increments else u
        B.vlbm_field_diff_norms(zero[:n * C], src[:n].view(n * C, c, c), nrm[:n * C])   # out[:, 1] = sum x^2
        total += nrm[:n * C, 1].view(n, C).sum(0).cpu().numpy()
    return [math.sqrt(t / (len(starts) * c * c)) for t in total]


def divergence_rms(snaps: torch.Tensor, chunk: int = 256) -> float:
    """RMS of the central-difference divergence of the velocity over every state of the store."""
    T, P1, C, c, _ = snaps.shape
    flat = snaps.view(T * P1, C, c, c)
    st = torch.empty(chunk, 3, dtype=torch.float64, device=snaps.device)
    total = 0.0
    for i in range(0, T * P1, chunk):
        n = min(chunk, T * P1 - i)
        B.vlbm_field_stats(flat[i:i + n], st[:n])
        total += float(st[:n, 1].sum().item())
    return math.sqrt(total / (T * P1 * c * c))


def divergence_ratio_max(snaps: torch.Tensor, chunk: int = 256) -> float:
    """Largest divergence-to-gradient ratio sqrt(sum div^2 / sum |grad u|^2) over the states of the store."""
    T, P1, C, c, _ = snaps.shape
    flat = snaps.view(T * P1, C, c, c)
    st = torch.empty(chunk, 3, dtype=torch.float64, device=snaps.device)
    best = 0.0
    for i in range(0, T * P1, chunk):
        n = min(chunk, T * P1 - i)
        B.vlbm_field_stats(flat[i:i + n], st[:n])
        h = st[:n].cpu().numpy()
        best = max(best, float(np.sqrt(h[:, 1] / h[:, 2]).max()))
    return best


def scaling(cfg: Config, snaps: torch.Tensor):
    """(input factors, output factors) of the network from the training store: inputs divided by
    their RMS, increments by theirs, the phi increment additionally by sqrt(phi_weight) so that
    its share of the loss is phi_weight."""
    in_rms = channel_rms(snaps, increments=False)
    inc_rms = channel_rms(snaps, increments=True)
    in_scale = [1.0 / x for x in in_rms]
    if cfg.divergence_input:
        in_scale.append(1.0 / divergence_rms(snaps))
    out_scale = list(inc_rms)
    if cfg.curl_output:                  # one scale for both velocity channels of the curl
        out_scale[0] = out_scale[1] = math.sqrt(0.5 * (inc_rms[0] ** 2 + inc_rms[1] ** 2))
    if cfg.channels > 2:
        out_scale[2] = inc_rms[2] / math.sqrt(cfg.phi_weight)
    return in_scale, out_scale


def train(net: Surrogate, snaps: torch.Tensor, cfg: Config, out_scale, log=None, max_seconds=None) -> dict:
    """Adam on random minibatches of pairs, cosine learning-rate decay; returns a summary."""
    T, P1, C, c, _ = snaps.shape
    flat = snaps.view(T * P1, C, c, c)
    starts = pair_starts(snaps)
    per_epoch = len(starts) // cfg.batch
    total = max(1, int(round(cfg.epochs * per_epoch)))
    rng = np.random.default_rng(cfg.seed_base + 7)
    u = torch.empty(cfg.batch, C, c, c, dtype=torch.float32, device=snaps.device)
    tgt = torch.empty_like(u)
    inv = [1.0 / x for x in out_scale]
    losses = []
    t0 = time.perf_counter()
    step = 0
    idx_dev = None
    for step in range(total):
        e, j = divmod(step, per_epoch)
        if j == 0:                                          # one upload of the epoch's shuffled indices
            perm = rng.permutation(starts)[:per_epoch * cfg.batch]
            idx_dev = torch.from_numpy(perm).to(snaps.device)
        B.vlbm_sur_gather_pairs(flat, idx_dev[j * cfg.batch:(j + 1) * cfg.batch], u, tgt, inv)
        lr = cfg.lr_min + 0.5 * (cfg.lr - cfg.lr_min) * (1.0 + math.cos(math.pi * step / total))
        want = step % 100 == 0 or step == total - 1
        loss = net.train_step(u, tgt, lr, want_loss=want)
        if want:
            losses.append((step, loss))
            if log:
                log(f"step {step}/{total} epoch {e} lr {lr:.2e} loss {loss:.4e} ({time.perf_counter() - t0:.1f} s)")
        if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
            break
    torch.cuda.synchronize()
    net.status()
    return {"steps": step + 1, "planned_steps": total, "seconds": time.perf_counter() - t0,
            "loss_first": losses[0][1], "loss_last": losses[-1][1], "losses": losses}


def one_step_error(net: Surrogate, snaps: torch.Tensor, chunk: int = 32) -> list:
    """Per-channel relative L2 error |du_pred - (s_{k+1} - s_k)| / |s_{k+1} - s_k| of the predicted
    increment over every pair of snaps."""
    T, P1, C, c, _ = snaps.shape
    flat = snaps.view(T * P1, C, c, c)
    idx = torch.from_numpy(pair_starts(snaps)).to(snaps.device)
    u = torch.empty(chunk, C, c, c, dtype=torch.float32, device=snaps.device)
    tgt, y = torch.empty_like(u), torch.empty_like(u)
    nrm = torch.empty(chunk * C, 2, dtype=torch.float64, device=snaps.device)
    err, ref = np.zeros(C), np.zeros(C)
    for i in range(0, len(idx), chunk):
        n = min(chunk, len(idx) - i)
        B.vlbm_sur_gather_pairs(flat, idx[i:i + n], u[:n], tgt[:n], [1.0] * C)
        net.increment(u[:n], out=y[:n])
        B.vlbm_field_diff_norms(y[:n].view(n * C, c, c), tgt[:n].view(n * C, c, c), nrm[:n * C])
        h = nrm[:n * C].view(n, C, 2).sum(0).cpu().numpy()
        err += h[:, 0]
        ref += h[:, 1]
    return np.sqrt(err / ref).tolist()


def velocity_errors(a: torch.Tensor, ref: torch.Tensor, nrm: torch.Tensor) -> list:
    """Relative L2 error of the velocity channels of states a against ref, per state."""
    n, C, c, _ = a.shape
    B.vlbm_field_diff_norms(a, ref, nrm[:n], n=2 * c * c)
    h = nrm[:n].cpu().numpy()
    return np.sqrt(h[:, 0] / h[:, 1]).tolist()


class Rollout:
    """Checked surrogate rollout of a batch of coarse states with the plain scheme as fallback."""

    def __init__(self, net: Surrogate, cfg: Config, batch: int, device="cuda", div_limit=None):
        """div_limit: largest divergence-to-gradient ratio a state may reach (None: div_factor
        times the starting state's ratio)."""
        c, C = cfg.coarse, cfg.channels
        self.net, self.cfg, self.div_limit = net, cfg, div_limit
        self.u = torch.empty(batch, C, c, c, dtype=torch.float32, device=device)
        self.nxt = torch.empty_like(self.u)
        self.stats = torch.empty(batch, 3, dtype=torch.float64, device=device)
        self.stats_prev = torch.empty_like(self.stats)
        self.stats_h = torch.empty(batch, 3, dtype=torch.float64).pin_memory()
        self.e0 = torch.empty(batch, dtype=torch.float64, device=device)
        self.r_max = torch.empty(batch, dtype=torch.float64, device=device)
        self.counts = torch.zeros(batch + 3, dtype=torch.int64, device=device)
        self.nrm = torch.empty(batch, 2, dtype=torch.float64, device=device)
        # the fallback: one coarse problem per state, advanced together; a failing step
        # re-initialises the flagged problems from their (u, phi) and reads them back
        # with one masked launch each
        self.coarse = Batch([dict(n=(c, c), dx=2 * math.pi / c, nu=cfg.nu)] * batch, precision="fp32")
        self.mask_d = torch.zeros(batch, dtype=torch.uint8, device=device)

    def close(self):
        self.coarse.close()

    def _read_stats(self, u):
        n = u.shape[0]
        B.vlbm_field_stats(u, self.stats[:n])
        self.stats_h[:n].copy_(self.stats[:n])             # synchronous: the host decides next
        s = self.stats_h[:n].numpy()
        ratio = np.sqrt(s[:, 1] / np.maximum(s[:, 2], 1e-300))
        return s[:, 0].copy(), ratio

    def run(self, u0: torch.Tensor, steps: int, check=True, reference=None, every=1):
        """Advance u0 (batch, C, c, c) by `steps` surrogate steps.

        With check, every step is decided on the device (vlbm_sur_rollout_check) and the flagged
        states are advanced by the coarse scheme through masked launches: no host round trip per
        step.  reference: optional (steps + 1, batch, C, c, c) states to measure the relative L2
        velocity error against every `every` steps.  Returns (final states, info dict).
        """
        cfg = self.cfg
        n = u0.shape[0]
        u, nxt = self.u[:n], self.nxt[:n]
        u.copy_(u0)
        curve, div_curve = [], []
        if check:
            cur, prev = self.stats[:n], self.stats_prev[:n]
            mask, counts = self.mask_d, self.counts[:n + 3]
            mask.zero_()                                       # entries past n stay unmasked
            counts.zero_()
            B.vlbm_field_stats(u, prev)
            self.e0[:n].copy_(prev[:, 0])
            if self.div_limit is None:
                r0 = torch.sqrt(prev[:, 1] / torch.clamp(prev[:, 2], min=1e-300))
                self.r_max[:n].copy_(torch.clamp(cfg.div_factor * r0, min=cfg.div_floor))
            else:
                self.r_max[:n].fill_(max(self.div_limit, cfg.div_floor))
        for k in range(steps):
            self.net.advance(u, out=nxt)
            if check:
                B.vlbm_field_stats(nxt, cur)
                B.vlbm_sur_rollout_check(cur, prev, self.e0[:n], self.r_max[:n], cfg.energy_step_tol,
                                         cfg.energy_drift_tol, mask[:n], counts)
                # the plain scheme on the coarse lattice for the flagged states: u[b] -> nxt[b]
                B.vlbm_batch_init_states(self.coarse.handle, u, mask)
                self.coarse.step(cfg.coarse_steps)
                B.vlbm_batch_macros_states(self.coarse.handle, nxt, mask)
                B.vlbm_field_stats(nxt, prev)                  # the accepted states: next step's reference
            u, nxt = nxt, u
            if reference is not None and ((k + 1) % every == 0 or k + 1 == steps):
                errs = velocity_errors(u, reference[k + 1], self.nrm)
                curve.append((k + 1, float(np.mean(errs)), errs))
                div_curve.append((k + 1, float(np.mean(self._read_stats(u)[1]))))
        if u.data_ptr() != self.u.data_ptr():
            self.u[:n].copy_(u)
        fallbacks, reasons = [0] * n, {"energy_step": 0, "energy_drift": 0, "divergence": 0}
        if check:
            c = counts.cpu().tolist()
            fallbacks = c[:n]
            reasons = {"energy_step": c[n], "energy_drift": c[n + 1], "divergence": c[n + 2]}
        return self.u[:n], {"fallbacks": fallbacks, "reasons": reasons, "curve": curve, "div_ratio": div_curve}


def coarse_scheme(cfg: Config, u0: torch.Tensor, steps: int, reference=None) -> tuple:
    """The plain scheme on the coarse lattice from each pooled state (u, phi):
    (final states, relative L2 velocity errors against reference)."""
    c, C = cfg.coarse, cfg.channels
    lat = Lattice((c, c), 2 * math.pi / c, cfg.nu, precision="fp32")
    out = torch.empty_like(u0)
    nrm = torch.empty(u0.shape[0], 2, dtype=torch.float64, device=u0.device)
    try:
        for b in range(u0.shape[0]):
            lat.init(u0[b, 0:2], u0[b, 2] if C > 2 else None)
            lat.step(steps * cfg.coarse_steps)
            B.vlbm_macros(lat.handle, None, out[b, 0:2], out[b, 2] if C > 2 else None)
    finally:
        lat.close()
    err = velocity_errors(out, reference, nrm) if reference is not None else None
    return out, err


def _event_ms(fn, repeats=1):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(repeats):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / repeats


def fine_time_to_t(cfg: Config, seed: int, repeats: int = 2) -> float:
    """Milliseconds for the plain FP32 scheme on the fine lattice to advance one state (u, phi)
    by rollout_steps K fine steps and return its pooled state (steps, macros, pooling)."""
    f, c, C, steps = cfg.fine, cfg.coarse, cfg.channels, cfg.rollout_steps
    dev = torch.device("cuda")
    lat = Lattice((f, f), 2 * math.pi / f, cfg.nu, precision="fp32")
    ufine = torch.empty(2, f, f, dtype=torch.float32, device=dev)
    pfine = torch.empty(1, f, f, dtype=torch.float32, device=dev)
    pooled = torch.empty(1, C, c, c, dtype=torch.float32, device=dev)
    try:
        lat.init(torch.from_numpy(initial_field(f, seed)).to(dev))
        lat.step(cfg.warmup * cfg.k_fine)
        B.vlbm_macros(lat.handle, None, ufine, pfine)
        u_start, p_start = ufine.clone(), pfine[0].clone()

        def fine_run():
            lat.init(u_start, p_start)
            lat.step(steps * cfg.k_fine)
            B.vlbm_macros(lat.handle, None, ufine, pfine if C > 2 else None)
            B.vlbm_field_pool(ufine, pooled[:, 0:2], cfg.factor)
            if C > 2:
                B.vlbm_field_pool(pfine, pooled[:, 2:3], cfg.factor)
        fine_run()
        return _event_ms(fine_run, repeats)
    finally:
        lat.close()


def time_to_t(cfg: Config, net: Surrogate, u0_coarse: torch.Tensor, seed: int, batch: int = 32,
              div_limit=None) -> dict:
    """Wall time on this GPU to advance one state by rollout_steps K fine steps, per state: the
    plain FP32 scheme on the fine lattice (steps, macros, pooling), the surrogate rollout with its
    checks (one state, and `batch` states at once), and the plain scheme on the coarse lattice."""
    c, C, steps = cfg.coarse, cfg.channels, cfg.rollout_steps
    dev = u0_coarse.device
    t_fine = fine_time_to_t(cfg, seed)
    ro = Rollout(net, cfg, batch, div_limit=div_limit)
    try:
        one = u0_coarse[:1].contiguous()
        many = u0_coarse[torch.arange(batch) % u0_coarse.shape[0]].contiguous()
        ro.run(one, 3)
        t_sur1 = _event_ms(lambda: ro.run(one, steps), 2)
        t_surb = _event_ms(lambda: ro.run(many, steps), 2) / batch
        t_sur1_nocheck = _event_ms(lambda: ro.run(one, steps, check=False), 2)
        t_surb_nocheck = _event_ms(lambda: ro.run(many, steps, check=False), 2) / batch
    finally:
        ro.close()
    lat = Lattice((c, c), 2 * math.pi / c, cfg.nu, precision="fp32")
    out = torch.empty(C, c, c, dtype=torch.float32, device=dev)
    try:
        def coarse_run():
            lat.init(one[0, 0:2], one[0, 2] if C > 2 else None)
            lat.step(steps * cfg.coarse_steps)
            B.vlbm_macros(lat.handle, None, out[0:2], out[2] if C > 2 else None)
        coarse_run()
        t_coarse = _event_ms(coarse_run, 2)
    finally:
        lat.close()
    # the coarse scheme with the same batching as the surrogate: `batch` states, one launch per step
    cb = Batch([dict(n=(c, c), dx=2 * math.pi / c, nu=cfg.nu)] * batch, precision="fp32")
    mask = torch.ones(batch, dtype=torch.uint8, device=dev)
    outs = torch.empty_like(many)
    try:
        def coarse_batch_run():
            B.vlbm_batch_init_states(cb.handle, many, mask)
            cb.step(steps * cfg.coarse_steps)
            B.vlbm_batch_macros_states(cb.handle, outs, mask)
        coarse_batch_run()
        t_coarse_b = _event_ms(coarse_batch_run, 2) / batch
    finally:
        cb.close()
    return {"fine_fp32_ms": t_fine, "surrogate_b1_ms": t_sur1, "surrogate_b1_nocheck_ms": t_sur1_nocheck,
            f"surrogate_b{batch}_ms_per_state": t_surb, f"surrogate_b{batch}_nocheck_ms_per_state": t_surb_nocheck,
            "coarse_fp32_ms": t_coarse, f"coarse_fp32_b{batch}_ms_per_state": t_coarse_b,
            "speedup_b1": t_fine / t_sur1, f"speedup_b{batch}": t_fine / t_surb}


@dataclass
class Trained:
    """A trained surrogate with its data and the quantities derived from them."""
    net: Surrogate
    train_snaps: torch.Tensor
    test_snaps: torch.Tensor
    in_scale: list
    out_scale: list
    div_limit: float
    summary: dict
    data_seconds: float


def train_surrogate(cfg: Config, log=print, max_seconds=None) -> Trained:
    """Generate the training and test data with the scheme, then train a network on them."""
    t0 = time.perf_counter()
    torch.cuda.synchronize()
    train_snaps = generate(cfg, cfg.train_seeds(), cfg.pairs_per_trajectory)
    test_snaps = generate(cfg, cfg.test_seeds(), cfg.rollout_steps)
    t_data = time.perf_counter() - t0
    in_scale, out_scale = scaling(cfg, train_snaps)
    div_limit = cfg.div_factor * divergence_ratio_max(train_snaps)
    log(f"data: {tuple(train_snaps.shape)} + {tuple(test_snaps.shape)} in {t_data:.1f} s; input factors {in_scale}, "
        f"output factors {out_scale}, divergence-ratio limit {div_limit:.3e}")
    net = Surrogate(cfg.coarse, cfg.coarse, max(cfg.batch, 32), channels=cfg.channels,
                    divergence_input=cfg.divergence_input, curl_output=cfg.curl_output, seed=cfg.net_seed)
    net.set_scaling(in_scale, out_scale)
    sigma = [cfg.noise_u, cfg.noise_u] + [cfg.noise_phi] * (cfg.channels - 2) + ([cfg.noise_div] if cfg.divergence_input else [])
    net.set_train_noise(sigma, seed=cfg.seed_base + 11)
    summary = train(net, train_snaps, cfg, out_scale, log=log, max_seconds=max_seconds)
    return Trained(net, train_snaps, test_snaps, in_scale, out_scale, div_limit, summary, t_data)


def run_pipeline(cfg: Config, log=print, weights_out=None) -> dict:
    """Data, training, evaluation and timing; returns the report."""
    t0 = time.perf_counter()
    tr = train_surrogate(cfg, log)
    net = tr.net
    val = one_step_error(net, tr.test_snaps)
    log(f"one-step relative increment error on test pairs, per channel: {val}")
    ref = tr.test_snaps.transpose(0, 1).contiguous()          # (steps + 1, states, C, c, c)
    u0 = ref[0].contiguous()
    ro = Rollout(net, cfg, u0.shape[0], div_limit=tr.div_limit)
    try:
        _, checked = ro.run(u0, cfg.rollout_steps, check=True, reference=ref, every=10)
        _, free = ro.run(u0, cfg.rollout_steps, check=False, reference=ref, every=10)
        ref_div = [(k, float(np.mean(ro._read_stats(ref[k].contiguous())[1])))
                   for k in range(10, cfg.rollout_steps + 1, 10)]
    finally:
        ro.close()
    _, coarse_err = coarse_scheme(cfg, u0, cfg.rollout_steps, reference=ref[-1])
    # persistence (s(t) = s(0)) as the floor any useful surrogate must beat
    nrm = torch.empty(u0.shape[0], 2, dtype=torch.float64, device=u0.device)
    persistence = velocity_errors(u0, ref[-1], nrm)
    timing = time_to_t(cfg, net, u0, cfg.test_seeds()[0], div_limit=tr.div_limit)
    if weights_out:
        torch.save({"params": net.params().cpu(), "in_scale": tr.in_scale, "out_scale": tr.out_scale,
                    "div_limit": tr.div_limit, "config": asdict(cfg)}, weights_out)
    net.status()
    net.close()
    return {"config": asdict(cfg), "in_scale": tr.in_scale, "out_scale": tr.out_scale, "div_limit": tr.div_limit,
            "data_seconds": tr.data_seconds,
            "train": {k: v for k, v in tr.summary.items() if k != "losses"}, "loss_curve": tr.summary["losses"],
            "one_step_rel_error": val,
            "rollout_checked": {"l2_rel_final": checked["curve"][-1][2], "l2_rel_final_mean": checked["curve"][-1][1],
                                "curve": [(k, m) for k, m, _ in checked["curve"]], "fallbacks": checked["fallbacks"],
                                "reasons": checked["reasons"], "div_ratio": checked["div_ratio"]},
            "rollout_unchecked": {"l2_rel_final": free["curve"][-1][2], "l2_rel_final_mean": free["curve"][-1][1],
                                  "curve": [(k, m) for k, m, _ in free["curve"]], "div_ratio": free["div_ratio"]},
            "reference_div_ratio": ref_div,
            "coarse_scheme_l2_rel_final": coarse_err, "persistence_l2_rel_final": persistence,
            "timing": timing, "seconds": time.perf_counter() - t0}


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    for name, val in asdict(Config()).items():
        kind = (lambda x: x.lower() in ("1", "true", "yes")) if isinstance(val, bool) else type(val)
        ap.add_argument("--" + name.replace("_", "-"), type=kind, default=val)
    ap.add_argument("--report", default=None)
    ap.add_argument("--weights", default=None)
    a = vars(ap.parse_args(argv))
    report_path, weights = a.pop("report"), a.pop("weights")
    cfg = Config(**a)
    rep = run_pipeline(cfg, log=lambda m: print(m, flush=True), weights_out=weights)
    text = json.dumps(rep, indent=1)
    if report_path:
        with open(report_path, "w") as fh:
            fh.write(text)
    print(json.dumps({k: rep[k] for k in ("one_step_rel_error", "rollout_checked", "rollout_unchecked",
                                          "coarse_scheme_l2_rel_final", "persistence_l2_rel_final", "timing")}))


if __name__ == "__main__":
    main()
