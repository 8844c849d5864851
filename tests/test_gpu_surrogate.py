"""The surrogate's data path on the GPU: pooling, pair gathering, field statistics, data
generation from the scheme, and the checked rollout with the plain scheme as fallback."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2607_24059_b300 as v  # noqa: E402
from paper_2607_24059_b300 import surrogate as sg  # noqa: E402


def test_pool_matches_avg_pool():
    g = torch.Generator(device="cuda").manual_seed(1)
    x = torch.randn(3, 2, 36, 44, device="cuda", generator=g)
    out = torch.empty(3, 2, 9, 11, device="cuda")
    v.vlbm_field_pool(x, out, 4)
    ref = torch.nn.functional.avg_pool2d(x.double(), 4)
    assert (out.double() - ref).abs().max().item() <= 1e-6


def test_gather_pairs_exact():
    g = torch.Generator(device="cuda").manual_seed(2)
    snaps = torch.randn(7, 2, 8, 12, device="cuda", generator=g)
    idx = torch.tensor([0, 5, 3, 3], dtype=torch.int64, device="cuda")
    u = torch.empty(4, 2, 8, 12, device="cuda")
    t = torch.empty_like(u)
    v.vlbm_sur_gather_pairs(snaps, idx, u, t, 0.25)
    assert torch.equal(u, snaps[idx])
    assert torch.equal(t, (snaps[idx + 1] - snaps[idx]) * 0.25)


def test_field_stats_and_norms_match_fp64():
    g = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn(3, 2, 20, 28, device="cuda", generator=g)
    st = torch.empty(3, 3, dtype=torch.float64, device="cuda")
    v.vlbm_field_stats(u, st)
    d = u.double()
    ux, uy = d[:, 0], d[:, 1]
    dxx = 0.5 * (ux.roll(-1, 2) - ux.roll(1, 2))
    dxy = 0.5 * (ux.roll(-1, 1) - ux.roll(1, 1))
    dyx = 0.5 * (uy.roll(-1, 2) - uy.roll(1, 2))
    dyy = 0.5 * (uy.roll(-1, 1) - uy.roll(1, 1))
    e = 0.5 * (ux ** 2 + uy ** 2).sum((1, 2))
    div = ((dxx + dyy) ** 2).sum((1, 2))
    grad = (dxx ** 2 + dxy ** 2 + dyx ** 2 + dyy ** 2).sum((1, 2))
    ref = torch.stack([e, div, grad], 1)
    assert ((st - ref).abs() / ref.abs()).max().item() <= 1e-6
    w = torch.randn(3, 2, 20, 28, device="cuda", generator=g)
    nrm = torch.empty(3, 2, dtype=torch.float64, device="cuda")
    v.vlbm_field_diff_norms(w, u, nrm)
    ref2 = torch.stack([((w.double() - d) ** 2).sum((1, 2, 3)), (d ** 2).sum((1, 2, 3))], 1)
    assert ((nrm - ref2).abs() / ref2).max().item() <= 1e-12


def tiny_config(**kw):
    base = dict(fine=64, factor=4, nu=1e-3, k_fine=16, warmup=2, train_trajectories=4, pairs_per_trajectory=8,
                test_trajectories=2, rollout_steps=5, batch=8, epochs=3.0, seed_base=77)
    base.update(kw)
    return sg.Config(**base)


def test_generate_matches_lattice_and_pooling():
    cfg = tiny_config()
    snaps = sg.generate(cfg, [5, 6], 3)
    assert snaps.shape == (2, 4, 3, 16, 16)
    lat = v.Lattice((64, 64), 2 * math.pi / 64, cfg.nu, precision="fp32")
    for i, seed in enumerate([5, 6]):
        lat.init(torch.from_numpy(sg.initial_field(64, seed)).cuda())
        lat.step(cfg.warmup * cfg.k_fine)
        for k in range(4):
            if k:
                lat.step(cfg.k_fine)
            _, u, phi = lat.macros(dtype=torch.float32)
            ref = torch.nn.functional.avg_pool2d(torch.cat([u, phi[None]]).double().unsqueeze(0), 4)[0]
            assert (snaps[i, k].double() - ref).abs().max().item() <= 1e-6
    lat.close()


def test_rollout_fallback_is_the_plain_coarse_scheme():
    cfg = tiny_config(energy_step_tol=-1.0)           # every surrogate step fails its check
    net = v.Surrogate(16, 16, max_batch=4, channels=3, seed=1)
    net.set_scaling(None, [1e-2] * 3)
    u0 = sg.generate(cfg, [11, 12], 0)[:, 0].contiguous()
    ro = sg.Rollout(net, cfg, 4)
    out, info = ro.run(u0, 3)
    out = out.clone()
    ro.close()
    assert info["fallbacks"] == [3, 3]
    lat = v.Lattice((16, 16), 2 * math.pi / 16, cfg.nu, precision="fp32")
    for b in range(2):
        s = u0[b].clone()
        for _ in range(3):
            lat.init(s[0:2], s[2])
            lat.step(cfg.coarse_steps)
            v.vlbm_macros(lat.handle, None, s[0:2], s[2])
        assert torch.allclose(out[b], s, rtol=1e-6, atol=1e-7)
    lat.close()
    net.close()


def test_batch_state_entry_points_match_single_problem_calls():
    """Masked init / read-out of a batch equal the per-problem calls, and skip unmasked problems."""
    c, n = 16, 3
    cfg = tiny_config()
    st = sg.generate(cfg, [21, 22, 23], 0)[:, 0].contiguous()          # (3, 3, 16, 16)
    bt = v.Batch([dict(n=(c, c), dx=2 * math.pi / c, nu=1e-3)] * n, precision="fp32")
    mask = torch.tensor([1, 0, 1], dtype=torch.uint8, device="cuda")
    v.vlbm_batch_init_states(bt.handle, st, mask)
    bt.init(1, st[1, 0:2], st[1, 2])
    bt.step(2)
    out = torch.full_like(st, 7.0)
    v.vlbm_batch_macros_states(bt.handle, out, mask)
    assert torch.equal(out[1], torch.full_like(out[1], 7.0))        # unmasked: untouched
    lat = v.Lattice((c, c), 2 * math.pi / c, 1e-3, precision="fp32")
    for b in (0, 2):
        lat.init(st[b, 0:2], st[b, 2])
        lat.step(2)
        ref = torch.empty(3, c, c, device="cuda")
        v.vlbm_macros(lat.handle, None, ref[0:2], ref[2])
        assert torch.allclose(out[b], ref, rtol=1e-6, atol=1e-7)
    lat.close()
    bt.close()


def test_rollout_check_matches_the_host_rule():
    """The device check flags exactly the states the FP64 host rule flags, NaN included, and
    accumulates its counts."""
    rng = np.random.default_rng(5)
    n = 40
    stats = np.abs(rng.normal(1.0, 0.01, (n, 3)))
    stats[:, 1] *= rng.uniform(0.5, 2.0, n) * 1e-4
    prev = np.abs(rng.normal(1.0, 0.01, (n, 3)))
    prev[:, 0] = stats[:, 0] * (1.0 + rng.normal(0.0, 3e-3, n))
    e0 = np.abs(rng.normal(1.0, 0.05, n))
    r_max = np.full(n, 0.012)
    stats[3, 0] = np.nan
    stats[5, 1] = np.nan
    stats[7, 2] = 0.0
    stats[9, 2] = np.nan
    prev[11, 0] = stats[11, 0]
    tol_step, tol_drift = 5e-3, 5e-2
    e = stats[:, 0]
    with np.errstate(all="ignore"):
        ratio = np.sqrt(stats[:, 1] / np.maximum(stats[:, 2], 1e-300))
        b_step = ~(np.abs(e / prev[:, 0] - 1.0) <= tol_step)
        b_drift = ~(np.abs(e / e0 - 1.0) <= tol_drift)
        b_div = ~(ratio <= r_max)
    bad = b_step | b_drift | b_div
    assert 0 < bad.sum() < n and 0 < b_step.sum() and 0 < b_drift.sum() and 0 < b_div.sum()

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    mask = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
    counts = torch.zeros(n + 3, dtype=torch.int64, device="cuda")
    for _ in range(2):
        v.vlbm_sur_rollout_check(dev(stats), dev(prev), dev(e0), dev(r_max), tol_step, tol_drift, mask, counts)
    assert np.array_equal(mask.cpu().numpy(), bad.astype(np.uint8))
    c = counts.cpu().numpy()
    assert np.array_equal(c[:n], 2 * bad.astype(np.int64))
    assert list(c[n:]) == [2 * int(b_step.sum()), 2 * int(b_drift.sum()), 2 * int(b_div.sum())]


def test_rollout_without_fallback_is_the_surrogate():
    cfg = tiny_config(energy_step_tol=1e9, energy_drift_tol=1e9, div_factor=1e9)
    net = v.Surrogate(16, 16, max_batch=4, channels=3, seed=2)
    net.set_scaling([1.0, 1.0, 0.5], [0.05, 0.05, 0.1])
    u0 = sg.generate(cfg, [13, 14, 15], 0)[:, 0].contiguous()
    ro = sg.Rollout(net, cfg, 4)
    out, info = ro.run(u0, 4)
    out = out.clone()
    ro.close()
    assert info["fallbacks"] == [0, 0, 0]
    u = u0.clone()
    for _ in range(4):
        u = net.advance(u)
    assert torch.equal(out, u)
    # advance = u + out_scale * forward(u), per channel
    y = net.forward(u0)
    step = net.advance(u0)
    sc = torch.tensor([0.05, 0.05, 0.1], device="cuda").view(1, 3, 1, 1)
    assert torch.allclose(step, u0 + sc * y, rtol=1e-6, atol=1e-7)
    net.close()


def test_divergence_input_channel():
    """With the derived channel, forward(u) equals forward of a net without it whose input carries
    the divergence as a stored channel (same weights, same factors)."""
    H = W = 16
    g = torch.Generator(device="cuda").manual_seed(4)
    u = torch.randn(2, 3, H, W, device="cuda", generator=g)
    a = v.Surrogate(H, W, max_batch=2, channels=3, divergence_input=True, seed=5)
    b = v.Surrogate(H, W, max_batch=2, channels=4, seed=6)
    p = a.params()
    b.load_params(p)
    a.set_scaling([1.0, 2.0, 0.5, 30.0], [1.0, 1.0, 1.0])
    b.set_scaling([1.0, 2.0, 0.5, 30.0], [1.0, 1.0, 1.0, 1.0])
    div = 0.5 * (u[:, 0].roll(-1, 2) - u[:, 0].roll(1, 2)) + 0.5 * (u[:, 1].roll(-1, 1) - u[:, 1].roll(1, 1))
    u4 = torch.cat([u, div[:, None]], 1).contiguous()
    ya = a.forward(u.contiguous())
    yb = b.forward(u4)
    # the derived channel is rounded once to BF16 on both sides; FP32 differences may differ in the last bit
    assert (ya - yb[:, :3]).abs().max().item() <= 1e-2 * yb[:, :3].abs().max().item()
    a.close()
    b.close()


def test_tiny_pipeline_runs_and_learns():
    cfg = tiny_config(epochs=40.0, lr=2e-3)
    rep = sg.run_pipeline(cfg, log=lambda m: None)
    assert rep["train"]["loss_last"] < 0.5 * rep["train"]["loss_first"]
    assert all(np.isfinite(rep["one_step_rel_error"]))
    assert len(rep["rollout_checked"]["l2_rel_final"]) == 2
    assert all(np.isfinite(rep["rollout_checked"]["l2_rel_final"]))
    t = rep["timing"]
    assert t["fine_fp32_ms"] > 0 and t["surrogate_b1_ms"] > 0


def test_train_noise_only_in_training():
    H = W = 16
    g = torch.Generator(device="cuda").manual_seed(9)
    u = torch.randn(2, 3, H, W, device="cuda", generator=g)
    t = 0.1 * torch.randn(2, 3, H, W, device="cuda", generator=g)
    a = v.Surrogate(H, W, max_batch=2, channels=3, divergence_input=True, seed=5)
    y0 = a.forward(u)
    l0 = a.train_step(u, t, 0.0)
    a.set_train_noise([0.0, 0.0, 0.5, 2.0], seed=3)
    l1 = a.train_step(u, t, 0.0)
    l2 = a.train_step(u, t, 0.0)
    assert torch.equal(a.forward(u), y0)                 # lr = 0 and no noise outside training
    assert l1 != l0 and l2 != l1                          # fresh draws every step
    a.set_train_noise(None)
    assert a.train_step(u, t, 0.0) == l0
    a.close()
