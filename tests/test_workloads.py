"""Checks of the seeded input generators (shapes, ranges, closed-form powers)."""
import numpy as np

import workloads as wl


def test_qam_unit_power_closed_form():
    # The full constellation of each square QAM has mean power exactly 1 after scaling.
    for order in wl.QAM_ORDERS:
        lv = wl.qam_levels(order)
        pts = (lv[:, None] + 1j * lv[None, :]).ravel() / np.sqrt(2.0 * (order - 1) / 3.0)
        assert np.isclose(np.mean(np.abs(pts) ** 2), 1.0, rtol=1e-14)
        assert len(lv) ** 2 == order


def test_precoder_unit_columns():
    W = wl.precoder_unit_columns(np.random.default_rng(1), 64, 36)
    assert W.shape == (64, 36)
    assert np.allclose(np.linalg.norm(W, axis=0), 1.0, rtol=1e-13)
    assert wl.precoder_unit_columns(np.random.default_rng(1), 64, 0).shape == (64, 0)


def test_seeded_repeatable():
    a, b = wl.config_small(seed=0, n_blocks=4), wl.config_small(seed=0, n_blocks=4)
    assert np.array_equal(a.S[0], b.S[0]) and np.array_equal(a.W[0], b.W[0])


def test_config_shapes():
    c1 = wl.config_small()
    assert c1.total_blocks == 1024 and c1.f_of_group == [8] and c1.S[0].shape == (1024, 8, 60)
    c2 = wl.config_fullband(n_rb=5)
    assert c2.total_blocks == 70 and set(c2.f_of_group) == {36} and c2.n_groups == 5
    assert c2.flops() == 70 * 8 * 64 * 60 * 36
    assert c2.algorithmic_bytes() == 5 * 64 * 36 * 8 + 70 * 36 * 60 * 8 + 70 * 64 * 60 * 8


def test_uneven_groups():
    c3 = wl.config_uneven(n_blocks=3000)
    assert c3.total_blocks == 3000
    assert all(1 <= n <= 64 for n in c3.n_blocks)
    assert all(0 <= f <= 36 for f in c3.f_of_group)
    assert 8 < np.mean(c3.n_blocks[:-1]) < 20


def test_reduced_noise_and_power():
    c4 = wl.config_reduced(copies=1, n_rb=20)
    S = np.concatenate([s.ravel() for s in c4.S])
    assert abs(np.mean(np.abs(S) ** 2) - (1 + 1e-3)) < 0.02


def test_serving_schedule():
    jobs = wl.serving_schedule(n_cells=8, n_tti=50)
    assert len(jobs) == 400
    assert all(25 <= j.n_rb <= 273 and 1 <= j.f <= 36 for j in jobs)
    assert all(jobs[i].arrival_s <= jobs[i + 1].arrival_s for i in range(len(jobs) - 1))
    # f is constant per cell within a 10-TTI precoder epoch
    for c in range(8):
        fs = {}
        for j in jobs:
            if j.cell == c:
                fs.setdefault(j.epoch, set()).add(j.f)
        assert all(len(v) == 1 for v in fs.values())


def test_pack_offsets():
    c = wl.config_uneven(n_blocks=100)
    flat, offs = c.pack_S()
    for g, s in enumerate(c.S):
        assert np.array_equal(flat[offs[g]:offs[g] + s.size], s.astype(np.complex64).ravel())
    assert c.r_offsets()[-1] == (c.total_blocks - c.n_blocks[-1]) * 64 * 60
