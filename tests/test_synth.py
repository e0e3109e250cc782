"""The seeded synthetic workloads follow their stated recipes: shapes, frame
rates, flow fields, threshold-noise statistics, activity levels, and
determinism per seed.  CPU only."""
import math

import numpy as np
import pytest

from paper_2209_04634_gb300 import synth

Q = 65536


def log_table():
    return np.array([math.floor(Q * math.log1p(v) + 0.5) for v in range(256)], dtype=np.int64)


def test_counter_rng_is_a_pure_function_of_the_seed():
    a, b, c = synth.Rng(7), synth.Rng(7), synth.Rng(8)
    ua, ub, uc = a.uniform(1000), b.uniform(1000), c.uniform(1000)
    assert np.array_equal(ua, ub) and not np.array_equal(ua, uc)
    assert 0.0 <= ua.min() and ua.max() < 1.0
    # successive draws continue the counter: the same numbers in one or two calls
    d = synth.Rng(7)
    assert np.array_equal(np.concatenate([d.uniform(400), d.uniform(600)]), ua)
    # uniform and normal moments
    u = synth.Rng(3).uniform(200_000)
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1 / 12) < 0.002
    z = synth.Rng(4).normal(200_000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_splitmix_finaliser_is_a_bijection_on_a_sample():
    x = np.arange(1 << 16, dtype=np.uint64) * np.uint64(0x10001)
    assert len(np.unique(synth.splitmix64(x))) == len(x)


def test_blob_translation_recipe():
    s = synth.blob_translation()
    assert s.frames.shape == (20, 180, 240) and s.frames.dtype == np.uint8
    assert s.substeps == 8 and s.c_pos == s.c_neg == 0.2
    assert np.all(s.flows[0] == 0)
    assert np.all(s.flows[1:, ..., 0] == np.float32(3.2))
    assert np.all(s.flows[1:, ..., 1] == np.float32(-1.7))
    assert np.array_equal(s.t_us, np.rint(np.arange(20) * 1e6 / 30).astype(np.int64))
    # frame j is frame 0 moved by j (3.2, -1.7): compare at whole-pixel shifts
    # (j = 10: (32, -17)) on the interior
    a, b = s.frames[0].astype(int), s.frames[10].astype(int)
    assert np.abs(b[20:160, 40:230] - a[37:177, 8:198]).max() <= 1
    # mid-grey base with blobs of both signs
    assert a.min() < 100 and a.max() > 156


def test_warped_texture_recipe():
    s = synth.warped_texture(width=160, height=120)
    assert s.frames.shape == (100, 120, 160)
    assert s.substeps == 0 and s.max_substeps == 8
    assert np.array_equal(s.t_us, np.arange(100, dtype=np.int64) * 50_000)  # 20 fps
    assert np.all(s.flows[0] == 0)
    mag = np.sqrt((s.flows.astype(np.float64) ** 2).sum(-1))
    assert 7.5 < mag.max() <= 8.0 + 1e-4            # scaled to 8 px/frame
    per_frame = mag.reshape(100, -1).max(1)[1:]
    assert per_frame.min() < 2.0                     # the magnitude oscillates in time
    # smooth: neighbouring flow vectors differ by a small fraction of a pixel
    assert np.abs(np.diff(s.flows[5], axis=1)).max() < 0.2
    # thresholds: N(0.2, 0.03) in Q16, floored at 0.01, the two maps independent
    for m in (s.cpos_map, s.cneg_map):
        v = m.astype(np.float64) / Q
        assert abs(v.mean() - 0.2) < 0.002 and abs(v.std() - 0.03) < 0.002
        assert v.min() >= 0.01 - 1e-5
    assert not np.array_equal(s.cpos_map, s.cneg_map)
    # the same seed gives the same stream; another seed another one
    t = synth.warped_texture(width=160, height=120, frames=3)
    assert np.array_equal(t.frames, s.frames[:3])
    u = synth.warped_texture(width=160, height=120, frames=3, seed=4210)
    assert not np.array_equal(u.frames, t.frames)


def test_moving_rectangles_recipe():
    s = synth.moving_rectangles(frames=8)
    assert s.frames.shape == (8, 720, 1280, 3)
    assert s.substeps == 10 and s.c_pos == 0.15
    assert np.array_equal(s.t_us, np.rint(np.arange(8) * 1e6 / 60).astype(np.int64))
    fl = s.flows[1:].reshape(-1, 2).astype(np.float64)
    moving = np.abs(fl).sum(1) > 0
    speeds = np.sqrt((fl[moving] ** 2).sum(1))
    assert 2.0 - 1e-5 <= speeds.min() and speeds.max() <= 12.0 + 1e-5
    assert len(np.unique(fl[moving], axis=0)) <= 6   # one velocity per rectangle
    # active pixels (log luma change of at least C) per frame: a few to 15 %
    lut = log_table()
    rgb = s.frames.astype(np.int64)
    luma = (77 * rgb[..., 0] + 150 * rgb[..., 1] + 29 * rgb[..., 2] + 128) >> 8
    L = lut[luma]
    c = round(0.15 * Q)
    frac = (np.abs(np.diff(L, axis=0)) >= c).reshape(7, -1).mean(1)
    assert np.all(frac > 0.02) and np.all(frac < 0.15)


@pytest.mark.parametrize("n", [2, 3, 6])
def test_pingpong_replays_forward_and_backward(n):
    seen = []
    for step in range(1, 4 * n):
        b, a, sign = synth.pingpong(step, n)
        assert abs(b - a) == 1 and 0 <= a < n and 0 <= b < n
        assert sign == (1 if b == a + 1 else -1)
        seen.append(b)
    assert set(seen) == set(range(n))
