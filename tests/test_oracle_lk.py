"""Pins of the oracle's pyramidal Lucas-Kanade flow (orc_flow_lk).

Lucas-Kanade takes a pixel's flow as the least-squares solution of the
linearised brightness-constancy equations over a window (the flow the
paper's sparse and difference simulators use, Sec. III-B, Sec. IV-A).  The
oracle is checked against what that definition fixes: no motion and no
texture give zero flow; frames built so that the linearised equations hold
exactly give the motion exactly; transposing or mirroring the frames
transposes or mirrors the flow exactly; a 1-D texture (the aperture
problem) is not tracked; a translated smooth texture is recovered to a
fraction of a pixel, and only coarse to fine when the motion exceeds the
window; RGB frames give the flow of their luma."""
import numpy as np
import pytest

import oracle

Q = 65536


def texture(W, H, seed=0, amp=40.0, blobs=30, dx=0.0, dy=0.0):
    """Smooth analytic texture (Gaussian blobs on mid grey), sampled at
    (x - dx, y - dy) and rounded to 8 bits."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(-20, W + 20, blobs)
    cy = rng.uniform(-20, H + 20, blobs)
    sg = rng.uniform(5, 12, blobs)
    a = rng.uniform(-amp, amp, blobs)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    xx -= dx
    yy -= dy
    v = 128.0 + sum(a[k] * np.exp(-((xx - cx[k]) ** 2 + (yy - cy[k]) ** 2) / (2 * sg[k] ** 2))
                    for k in range(blobs))
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def central2(f):
    """Twice the central differences of an 8-bit image, reads clamped (the
    textbook definition, in the test's own numpy)."""
    g = f.astype(np.int64)
    gx = np.concatenate([g[:, 1:], g[:, -1:]], 1) - np.concatenate([g[:, :1], g[:, :-1]], 1)
    gy = np.concatenate([g[1:], g[-1:]], 0) - np.concatenate([g[:1], g[:-1]], 0)
    return gx, gy


def test_identical_frames_give_zero_flow():
    f = texture(90, 70, seed=1)
    for L, r, K in ((1, 1, 1), (3, 3, 3), (4, 2, 5)):
        assert not oracle.flow_lk(f, f, levels=L, radius=r, iterations=K, min_eig=0.0).any()


def test_untextured_frames_are_not_tracked():
    a = np.full((40, 50), 90, np.uint8)
    b = np.full((40, 50), 140, np.uint8)
    assert not oracle.flow_lk(a, b, levels=3, radius=2, min_eig=0.0).any()


@pytest.mark.parametrize("u,v", [(2, 0), (0, -2), (2, -2), (-4, 2)])
def test_exactly_linear_motion_is_recovered_exactly(u, v):
    # f1 = f0 - (u Ix + v Iy) / 2 with Ix, Iy twice the central differences:
    # the linearised equations hold exactly at every pixel, so the
    # least-squares solution of every window is (u, v) exactly
    f0 = texture(64, 48, seed=2, amp=18.0)
    gx, gy = central2(f0)
    f1 = f0.astype(np.int64) - (u * gx + v * gy) // 2
    assert f1.min() >= 0 and f1.max() <= 255
    assert ((u * gx + v * gy) % 2 == 0).all()
    fl = oracle.flow_lk(f0, f1.astype(np.uint8), levels=1, radius=2, iterations=1, min_eig=1.0)
    tracked = (fl != 0).any(-1)
    assert tracked.mean() > 0.9
    assert (fl[tracked] == np.array([u * Q, v * Q])).all()


def test_transposed_frames_give_the_transposed_flow_at_one_step():
    # one level, one iteration: J is sampled at whole pixels (the bilinear
    # blends x before y, so fractional samples are not transpose-symmetric)
    f0 = texture(72, 56, seed=3)
    f1 = texture(72, 56, seed=3, dx=1.4, dy=-0.7)
    a = oracle.flow_lk(f0, f1, levels=1, radius=3, iterations=1)
    b = oracle.flow_lk(f0.T.copy(), f1.T.copy(), levels=1, radius=3, iterations=1)
    assert a.any()
    assert np.array_equal(b.transpose(1, 0, 2)[..., ::-1], a)


def test_mirrored_frames_give_the_mirrored_flow_at_one_step():
    # one level, one iteration: J is sampled at whole pixels, so a mirror in x
    # flips the sign of the horizontal flow exactly
    f0 = texture(60, 40, seed=4)
    f1 = texture(60, 40, seed=4, dx=0.8, dy=0.5)
    a = oracle.flow_lk(f0, f1, levels=1, radius=2, iterations=1)
    b = oracle.flow_lk(f0[:, ::-1].copy(), f1[:, ::-1].copy(), levels=1, radius=2, iterations=1)
    b = b[:, ::-1]
    assert np.array_equal(b[..., 0], -a[..., 0])
    assert np.array_equal(b[..., 1], a[..., 1])


def test_one_dimensional_texture_is_not_tracked():
    # vertical stripes: Iy = 0 everywhere, the gradient matrix is singular
    x = np.arange(80)
    row = np.clip(np.rint(128 + 60 * np.sin(x / 5.0)), 0, 255).astype(np.uint8)
    f0 = np.repeat(row[None], 50, 0)
    f1 = np.roll(f0, 1, axis=1)
    assert not oracle.flow_lk(f0, f1, levels=2, radius=3, min_eig=1.0).any()


def _interior_error(fl, dx, dy, m=12):
    e = np.hypot(fl[..., 0] / Q - dx, fl[..., 1] / Q - dy)
    return e[m:-m, m:-m]


def test_translation_is_recovered_to_a_fraction_of_a_pixel():
    dx, dy = 5.0, -3.0
    f0 = texture(160, 120, seed=5, blobs=80)
    f1 = texture(160, 120, seed=5, blobs=80, dx=dx, dy=dy)
    e = _interior_error(oracle.flow_lk(f0, f1, levels=3, radius=3, iterations=4), dx, dy)
    assert np.median(e) < 0.05
    assert np.percentile(e, 90) < 0.25


def test_motion_beyond_the_window_needs_the_pyramid():
    dx, dy = 6.0, 4.0
    f0 = texture(160, 120, seed=6, blobs=80)
    f1 = texture(160, 120, seed=6, blobs=80, dx=dx, dy=dy)
    one = _interior_error(oracle.flow_lk(f0, f1, levels=1, radius=2, iterations=4), dx, dy)
    three = _interior_error(oracle.flow_lk(f0, f1, levels=3, radius=2, iterations=4), dx, dy)
    assert np.median(one) > 1.0
    assert np.median(three) < 0.15


def test_rgb_frames_give_the_flow_of_their_luma():
    rng = np.random.default_rng(7)
    g0 = texture(50, 30, seed=8)
    g1 = texture(50, 30, seed=8, dx=1.3, dy=0.4)
    # RGB triples whose BT.601 luma is the grey value (r = g = b = v)
    c0 = np.repeat(g0[..., None], 3, 2)
    c1 = np.repeat(g1[..., None], 3, 2)
    assert np.array_equal(oracle.flow_lk(c0, c1), oracle.flow_lk(g0, g1))
    # and coloured frames: the flow of the luma the oracle's own BT.601 gives
    col0 = rng.integers(0, 256, (30, 50, 3), dtype=np.uint8)
    col1 = np.roll(col0, 1, axis=1)
    l0 = np.vectorize(oracle.luma)(col0[..., 0], col0[..., 1], col0[..., 2]).astype(np.uint8)
    l1 = np.vectorize(oracle.luma)(col1[..., 0], col1[..., 1], col1[..., 2]).astype(np.uint8)
    assert np.array_equal(oracle.flow_lk(col0, col1), oracle.flow_lk(l0, l1))


def test_no_window_passes_an_unreachable_eigenvalue_threshold():
    f0 = texture(60, 40, seed=12, blobs=80)
    f1 = texture(60, 40, seed=12, blobs=80, dx=1.0)
    assert oracle.flow_lk(f0, f1, levels=2, min_eig=0.0).any()
    assert not oracle.flow_lk(f0, f1, levels=2, min_eig=1e12).any()


def test_rejects_bad_parameters():
    f = np.zeros((8, 8), np.uint8)
    for kw in (dict(levels=0), dict(levels=9), dict(radius=0), dict(radius=8),
               dict(iterations=0), dict(iterations=17)):
        with pytest.raises(ValueError):
            oracle.flow_lk(f, f, **kw)
