"""Host logic of the surrogate pipeline that runs without a GPU: the configuration's step
arithmetic, the seed split, the pair indexing and the initial fields."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_24059_b300 import surrogate as sg  # noqa: E402


def test_coarse_steps_follow_the_parabolic_scaling():
    # dt = dx^2 / mu: a lattice `factor` times coarser takes factor^2 times longer steps
    cfg = sg.Config()
    assert cfg.coarse == 256
    assert cfg.coarse_steps == 2                      # 32 fine steps of 1024^2 = 2 steps of 256^2
    assert sg.Config(k_fine=48, factor=4).coarse_steps == 3
    assert sg.Config(fine=512, factor=2, k_fine=8).coarse_steps == 2
    for bad in (sg.Config(k_fine=24, factor=4), sg.Config(k_fine=8, factor=4)):
        with pytest.raises(ValueError):
            bad.coarse_steps


def test_training_and_test_seeds_are_disjoint():
    cfg = sg.Config(train_trajectories=50, test_trajectories=8)
    train, test = cfg.train_seeds(), cfg.test_seeds()
    assert len(train) == 50 and len(set(train)) == 50
    assert len(test) == 8 and len(set(test)) == 8
    assert not set(train) & set(test)


def test_pairs_never_cross_a_trajectory_boundary():
    T, P1 = 3, 5
    snaps = torch.zeros(T, P1, 2, 4, 4)
    idx = sg.pair_starts(snaps)
    assert len(idx) == T * (P1 - 1)
    assert len(set(idx.tolist())) == len(idx)
    # a pair starts at any snapshot but the last of its trajectory, and its successor is in the same one
    assert all(i % P1 != P1 - 1 for i in idx)
    assert all((i + 1) // P1 == i // P1 for i in idx)


def test_initial_field_is_divergence_free_with_unit_rms_speed():
    side = 64
    u = sg.initial_field(side, 11)
    assert u.shape == (2, side, side) and u.dtype == np.float64
    assert math.isclose(float(np.mean(u[0] ** 2 + u[1] ** 2)), 1.0, rel_tol=1e-12)
    # spectral divergence of the periodic field: i kx u_x^ + i ky u_y^ (x along the last axis)
    k = np.fft.fftfreq(side, d=1.0 / side)
    KX, KY = np.meshgrid(k, k, indexing="xy")
    div = np.fft.ifft2(1j * KX * np.fft.fft2(u[0]) + 1j * KY * np.fft.fft2(u[1]))
    assert float(np.abs(div).max()) < 1e-9
    # seeded: the same seed gives the same field, another seed another one
    assert np.array_equal(u, sg.initial_field(side, 11))
    assert not np.allclose(u, sg.initial_field(side, 12))
