"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(log table, BT.601 weights, bilinear sampling of a plane, ceil of a square
root), the special case that reduces to the Kaiser difference frame of
Sec. II / III, exhaustive enumeration of one-pixel inputs, exact integer
translations (where interpolation must reproduce shifted samples), the
reference-conservation invariant, and a second pixel-major restatement in
pure Python on random 8x8 inputs.

Paper: Ziegler et al., "Real-time event simulation with frame-based cameras",
arXiv 2209.04634 (Sec. III-A equations, Sec. III-B, Table I).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact

Q = 65536


def py_lut(linear=False):
    """Independent log table: log1p in double, round half up (no ties occur)."""
    if linear:
        return np.arange(256, dtype=np.int64) * Q
    return np.array([math.floor(Q * math.log1p(v) + 0.5) for v in range(256)], dtype=np.int64)


def counts_per_pixel(events, H, W):
    """Signed event count per pixel."""
    t, x, y, p = oracle.unpack(events)
    c = np.zeros((H, W), dtype=np.int64)
    np.add.at(c, (y, x), p)
    return c


def abs_counts_per_pixel(events, H, W):
    t, x, y, p = oracle.unpack(events)
    c = np.zeros((H, W), dtype=np.int64)
    np.add.at(c, (y, x), 1)
    return c


def zero_flows(frames):
    return np.zeros(frames.shape[:3] + (2,), np.float32)


def times(F, dt=1000):
    return np.arange(F, dtype=np.int64) * dt


def accum_process(seq, r0, cp, cn):
    """Scalar reference-accumulating threshold process on a value sequence.
    Returns a list of (k, signed count) and the final reference."""
    out, r = [], r0
    for k, v in enumerate(seq, 1):
        d = v - r
        if d >= cp:
            m = d // cp
            r += m * cp
            out.append((k, m))
        elif -d >= cn:
            m = (-d) // cn
            r -= m * cn
            out.append((k, -m))
    return out, r


def reset_process(seq, i0, cp, cn):
    out, prev = [], i0
    for k, v in enumerate(seq, 1):
        d = v - prev
        if d > cp:
            out.append((k, 1))
        elif d < -cn:
            out.append((k, -1))
        prev = v
    return out


def per_pixel_sequences(events, N=None):
    """{(x, y): [(k-rank by time, signed count), ...]} grouped by timestamp."""
    t, x, y, p = oracle.unpack(events)
    d = {}
    for ti, xi, yi, pi in zip(t, x, y, p):
        lst = d.setdefault((int(xi), int(yi)), [])
        if lst and lst[-1][0] == int(ti) and np.sign(lst[-1][1]) == pi:
            lst[-1] = (lst[-1][0], lst[-1][1] + int(pi))
        else:
            lst.append((int(ti), int(pi)))
    return d


# --------------------------------------------------------------------------
# tables and primitives

def test_lut_log_closed_form():
    L = oracle.lut(oracle.LOG)
    ref = py_lut()
    for v in range(256):
        e = Q * math.log1p(v)
        assert abs((e - math.floor(e)) - 0.5) > 1e-6, "tie in the log table"
    assert np.array_equal(L.astype(np.int64), ref)
    assert L[0] == 0
    assert L[255] == math.floor(8 * math.log(2.0) * Q + 0.5) == 363409
    assert np.all(np.diff(L) > 0)


def test_lut_linear():
    assert np.array_equal(oracle.lut(oracle.LINEAR).astype(np.int64), py_lut(True))


def test_luma_bt601():
    rng = np.random.default_rng(1)
    assert oracle.luma(0, 0, 0) == 0 and oracle.luma(255, 255, 255) == 255
    for r, g, b in rng.integers(0, 256, size=(500, 3)):
        y = oracle.luma(int(r), int(g), int(b))
        assert abs(y - (0.299 * r + 0.587 * g + 0.114 * b)) <= 1.0


def test_flow_q16():
    assert oracle.flow_q16(3.2)[0] == 209715
    assert oracle.flow_q16(-1.7)[0] == round(float(np.float32(-1.7)) * Q)
    assert oracle.flow_q16(float("nan")) == (0, False)
    assert oracle.flow_q16(2000.0) == (1024 * Q, True)
    assert oracle.flow_q16(-5000.0) == (-1024 * Q, True)
    # ties to even at half a Q16 step
    assert oracle.flow_q16(0.5 / Q)[0] == 0
    assert oracle.flow_q16(1.5 / Q)[0] == 2


@pytest.mark.parametrize("a,b,c", [(20, 1, 2), (200, -1, -1), (40, 2, 1), (100, 0, -2)])
def test_bilinear_of_a_plane(a, b, c):
    """Bilinear sampling of a plane returns the plane at the (clamped) position
    with the fraction truncated to 12 bits."""
    W, H = 48, 40
    yy, xx = np.mgrid[0:H, 0:W]
    v = a + b * xx + c * yy
    assert v.min() >= 0 and v.max() <= 255
    L = (v * Q).astype(np.int32)
    rng = np.random.default_rng(7)
    for px, py in rng.integers(-5 * Q, (W + 5) * Q, size=(400, 2)):
        py = int(py) % ((H + 10) * Q) - 5 * Q
        cx = min(max(int(px), 0), (W - 1) * Q)
        cy = min(max(py, 0), (H - 1) * Q)
        want = a * Q + b * (cx & ~15) + c * (cy & ~15)
        assert oracle.bilinear(L, int(px), py) == want


def test_bilinear_at_integer_positions_is_indexing():
    rng = np.random.default_rng(3)
    L = rng.integers(0, 363409, size=(9, 13)).astype(np.int32)
    for y in range(9):
        for x in range(13):
            assert oracle.bilinear(L, x * Q, y * Q) == L[y, x]


def test_adaptive_substeps_is_ceil_of_max_flow():
    rng = np.random.default_rng(5)
    for _ in range(300):
        m = int(rng.integers(0, 2 ** 53))
        s = math.isqrt(m)
        if s * s < m:
            s += 1
        want = max(1, -(-s // Q))
        assert oracle.adaptive_substeps(m, 1 << 20) == want
    assert oracle.adaptive_substeps(0, 8) == 1
    assert oracle.adaptive_substeps((100 * Q) ** 2, 8) == 8
    for n in range(1, 12):  # a flow of exactly n pixels needs exactly n substeps
        assert oracle.adaptive_substeps((n * Q) ** 2, 64) == n
        assert oracle.adaptive_substeps((n * Q) ** 2 + 1, 64) == n + 1


# --------------------------------------------------------------------------
# closed forms of the simulator

@pytest.mark.parametrize("mode", [oracle.DENSE, oracle.SPARSE])
@pytest.mark.parametrize("ref", [oracle.ACCUM, oracle.RESET])
@pytest.mark.parametrize("intensity", [oracle.LOG, oracle.LINEAR])
def test_identical_frames_zero_flow_no_events(mode, ref, intensity):
    rng = np.random.default_rng(11)
    f = rng.integers(0, 256, size=(1, 17, 23), dtype=np.uint8)
    frames = np.repeat(f, 4, axis=0)
    c = 13107 if intensity == oracle.LOG else 2 * Q
    r = oracle.run(frames, zero_flows(frames), times(4), mode=mode, ref_mode=ref,
                   intensity=intensity, substeps=5, c_pos_q16=c, c_neg_q16=c)
    assert len(r["events"]) == 0


@pytest.mark.parametrize("N", [1, 2, 5, 8, 10])
@pytest.mark.parametrize("cp,cn", [(13107, 13107), (9000, 17000)])
def test_uniform_step_gives_floor_of_difference_over_C(N, cp, cn):
    """Zero flow, uniform frames: a step of D in log intensity gives exactly
    floor(|D| / C) events per pixel, all of one sign, and the cumulative count
    never decreases over the substeps."""
    lut = py_lut()
    rng = np.random.default_rng(N)
    for v0, v1 in rng.integers(0, 256, size=(30, 2)):
        frames = np.stack([np.full((3, 4), v0), np.full((3, 4), v1)]).astype(np.uint8)
        r = oracle.run(frames, zero_flows(frames), times(2, 990), substeps=N,
                       c_pos_q16=cp, c_neg_q16=cn)
        D = int(lut[v1] - lut[v0])
        want = D // cp if D >= 0 else -((-D) // cn)
        cnt = counts_per_pixel(r["events"], 3, 4)
        assert np.all(cnt == want)
        assert len(r["events"]) == 12 * abs(want)
        t = r["events"]["t"]
        assert np.all(np.diff(t.astype(np.int64)) >= 0)


def test_alternating_steps_give_alternating_bursts():
    lut = py_lut()
    vals = [100, 180, 60, 200, 90, 91, 30]
    frames = np.array([np.full((2, 2), v) for v in vals], np.uint8)
    cp = cn = 13107
    r = oracle.run(frames, zero_flows(frames), times(len(vals)), substeps=6,
                   c_pos_q16=cp, c_neg_q16=cn)
    # the reference follows the scalar process R <- R +- m C
    R = int(lut[vals[0]])
    expect = []
    for v in vals[1:]:
        _, R2 = accum_process([int(lut[v])], R, cp, cn)
        expect.append((R2 - R) // (cp if R2 >= R else cn) if R2 != R else 0)
        R = R2
    assert list(r["ev_per_frame"][1:]) == [4 * abs(e) for e in expect]
    ev = r["events"]
    t, x, y, p = oracle.unpack(ev)
    for i, e in enumerate(expect, 1):
        sel = (t > (i - 1) * 1000) & (t <= i * 1000)
        if e:
            assert np.all(p[sel] == np.sign(e))
    assert np.all(r["R"] == R)


@pytest.mark.parametrize("N", [1, 7])
@pytest.mark.parametrize("intensity,c", [(oracle.LOG, 13107), (oracle.LOG, 3001),
                                         (oracle.LINEAR, 2 * Q), (oracle.LINEAR, 7 * Q + 5)])
def test_exhaustive_one_pixel_pairs(N, intensity, c):
    """Every (v0, v1) pair of 8-bit values, one pixel each, zero flow."""
    v1, v0 = np.meshgrid(np.arange(256), np.arange(256))
    frames = np.stack([v0, v1]).astype(np.uint8)
    r = oracle.run(frames, zero_flows(frames), times(2), substeps=N, intensity=intensity,
                   c_pos_q16=c, c_neg_q16=c)
    lut = py_lut(intensity == oracle.LINEAR)
    D = lut[v1] - lut[v0]
    want = np.where(D >= 0, D // c, -((-D) // c))
    assert np.array_equal(counts_per_pixel(r["events"], 256, 256), want)
    assert len(r["events"]) == int(np.abs(want).sum())


@pytest.mark.parametrize("m,N", [((1, 0), 3), ((0, -1), 4), ((1, -1), 2), ((-2, 1), 3)])
@pytest.mark.parametrize("ref", [oracle.ACCUM, oracle.RESET])
def test_integer_translation_reproduces_shifted_samples(m, N, ref):
    """Frame i = frame i-1 moved by F = N m whole pixels: every tap is exact and
    the interpolated frame k is frame i-1 moved by k m, so the events of an
    interior pixel are the threshold crossings of the 1-D sequence
    L0(x - k m), k = 1..N."""
    rng = np.random.default_rng(17)
    H, W = 30, 40
    f0 = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    F = (N * m[0], N * m[1])
    f1 = np.roll(f0, (F[1], F[0]), axis=(0, 1))
    frames = np.stack([f0, f1])
    flows = zero_flows(frames)
    flows[1, ..., 0] = F[0]
    flows[1, ..., 1] = F[1]
    cp, cn = 20000, 15000
    r = oracle.run(frames, flows, times(2, 1000), substeps=N, ref_mode=ref,
                   c_pos_q16=cp, c_neg_q16=cn)
    lut = py_lut()
    got = per_pixel_sequences(r["events"])
    margin = N * max(abs(m[0]), abs(m[1])) + 1
    checked = 0
    for y in range(margin, H - margin):
        for x in range(margin, W - margin):
            seq = [int(lut[f0[y - k * m[1], x - k * m[0]]]) for k in range(1, N + 1)]
            r0 = int(lut[f0[y, x]])
            if ref == oracle.ACCUM:
                exp, _ = accum_process(seq, r0, cp, cn)
            else:
                exp = reset_process(seq, r0, cp, cn)
            exp_t = [(k * 1000 // N, c) for k, c in exp]
            assert got.get((x, y), []) == exp_t, (x, y)
            checked += 1
    assert checked > 200


@pytest.mark.parametrize("N", [3, 8])
def test_plane_images_with_fractional_flow(N):
    """Linear intensity, frames that are planes with integer slopes, random
    fractional per-pixel flow: the samples have a closed form (the plane at the
    clamped, 12-bit-truncated position), so the events follow from the scalar
    threshold process on that closed form."""
    H, W = 24, 32
    yy, xx = np.mgrid[0:H, 0:W]
    f0 = (30 + 2 * xx + 1 * yy).astype(np.uint8)
    f1 = (90 + 1 * xx + 3 * yy).astype(np.uint8)
    P0, P1 = (30, 2, 1), (90, 1, 3)
    rng = np.random.default_rng(N)
    flows = np.zeros((2, H, W, 2), np.float32)
    flows[1] = rng.uniform(-3.0, 3.0, size=(H, W, 2)).astype(np.float32)
    cp, cn = 3 * Q + 1000, 2 * Q + 777
    frames = np.stack([f0, f1])
    r = oracle.run(frames, flows, times(2, 777), substeps=N, intensity=oracle.LINEAR,
                   c_pos_q16=cp, c_neg_q16=cn)

    def plane(P, px, py):
        cx = min(max(px, 0), (W - 1) * Q)
        cy = min(max(py, 0), (H - 1) * Q)
        return P[0] * Q + P[1] * (cx & ~15) + P[2] * (cy & ~15)

    got = per_pixel_sequences(r["events"])
    for y in range(H):
        for x in range(W):
            fx = int(np.rint(np.float64(flows[1, y, x, 0]) * Q))
            fy = int(np.rint(np.float64(flows[1, y, x, 1]) * Q))
            seq = []
            for k in range(1, N + 1):
                ox, oy = (fx * k) // N, (fy * k) // N
                s0 = plane(P0, x * Q - ox, y * Q - oy)
                s1 = plane(P1, x * Q + fx - ox, y * Q + fy - oy)
                w = (k * 8192 + N) // (2 * N)
                seq.append(s0 + ((s1 - s0) * w + 2048) // 4096)
            assert seq[-1] == int(f1[y, x]) * Q
            exp, rf = accum_process(seq, int(f0[y, x]) * Q, cp, cn)
            assert got.get((x, y), []) == [(k * 777 // N, c) for k, c in exp]
            assert r["R"][y, x] == rf


@pytest.mark.parametrize("N", [2, 5, 8])
def test_plane_with_subpixel_flow_at_unit_resolution(N):
    """Both frames the same plane, sub-pixel flows, thresholds of a few Q16
    units: the event counts then trace every interpolated value to within one
    threshold step, so the closed form pins the offset rounding, the 12-bit
    position truncation and the rounding of each blend at unit resolution."""
    H, W = 12, 16
    yy, xx = np.mgrid[0:H, 0:W]
    P = (40, 3, -2)
    f = (P[0] + P[1] * xx + P[2] * yy + 2 * H).astype(np.uint8)
    P = (P[0] + 2 * H, P[1], P[2])
    rng = np.random.default_rng(100 + N)
    flows = np.zeros((2, H, W, 2), np.float32)
    flows[1] = rng.uniform(-0.02, 0.02, size=(H, W, 2)).astype(np.float32)
    cp, cn = 5, 7
    frames = np.stack([f, f])
    r = oracle.run(frames, flows, times(2, 1000), substeps=N, intensity=oracle.LINEAR,
                   c_pos_q16=cp, c_neg_q16=cn)

    def plane(px, py):
        cx = min(max(px, 0), (W - 1) * Q)
        cy = min(max(py, 0), (H - 1) * Q)
        return P[0] * Q + P[1] * (cx & ~15) + P[2] * (cy & ~15)

    got = per_pixel_sequences(r["events"])
    for y in range(H):
        for x in range(W):
            fx = int(np.rint(np.float64(flows[1, y, x, 0]) * Q))
            fy = int(np.rint(np.float64(flows[1, y, x, 1]) * Q))
            seq = []
            for k in range(1, N + 1):
                ox, oy = (fx * k) // N, (fy * k) // N
                s0 = plane(x * Q - ox, y * Q - oy)
                s1 = plane(x * Q + fx - ox, y * Q + fy - oy)
                # the blend of two Q16 samples must land within half a unit of
                # the exact rational blend at the rounded weight
                w = (k * 8192 + N) // (2 * N)
                exact_blend = s0 + (s1 - s0) * w / 4096
                i_k = s0 + ((s1 - s0) * w + 2048) // 4096
                assert abs(i_k - exact_blend) <= 0.5
                seq.append(i_k)
            exp, rf = accum_process(seq, int(f[y, x]) * Q, cp, cn)
            assert got.get((x, y), []) == [(k * 1000 // N, c) for k, c in exp]


def test_blend_is_within_half_a_unit_of_the_exact_line():
    """Zero flow, threshold of one Q16 unit: the cumulative event count after
    substep k is the interpolated value minus frame i-1 exactly, which must lie
    within 1/2 + |D| / 8192 of the straight line D k / N (half a unit of final
    rounding plus the rounding of the Q12 weight)."""
    lut = py_lut()
    for N in (3, 7, 10):
        for v0, v1 in [(100, 101), (101, 100), (50, 53), (200, 197), (10, 11)]:
            frames = np.stack([np.full((1, 1), v0), np.full((1, 1), v1)]).astype(np.uint8)
            r = oracle.run(frames, zero_flows(frames), times(2, 1000 * N), substeps=N,
                           c_pos_q16=1, c_neg_q16=1)
            D = int(lut[v1] - lut[v0])
            t, x, y, p = oracle.unpack(r["events"])
            for k in range(1, N + 1):
                c_k = int(p[t <= k * 1000].sum())
                assert abs(c_k - D * k / N) <= 0.5 + abs(D) / 8192, (N, v0, v1, k)
            assert int(p.sum()) == D


def test_conservation_and_band_invariant():
    """R_end = R_0 + Cp #pos - Cn #neg per pixel, and after the last substep of a
    frame (which lands exactly on frame i) the frame lies within (-Cn, Cp) of R."""
    rng = np.random.default_rng(23)
    F, H, W = 6, 20, 26
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    flows = rng.uniform(-4, 4, size=(F, H, W, 2)).astype(np.float32)
    cp, cn = 11000, 16000
    r = oracle.run(frames, flows, times(F), substeps=0, max_substeps=9,
                   c_pos_q16=cp, c_neg_q16=cn)
    lut = py_lut()
    t, x, y, p = oracle.unpack(r["events"])
    pos = np.zeros((H, W), np.int64)
    neg = np.zeros((H, W), np.int64)
    np.add.at(pos, (y[p > 0], x[p > 0]), 1)
    np.add.at(neg, (y[p < 0], x[p < 0]), 1)
    R0 = lut[frames[0]]
    assert np.array_equal(r["R"].astype(np.int64), R0 + cp * pos - cn * neg)
    D = lut[frames[-1]] - r["R"]
    assert np.all(D < cp) and np.all(D > -cn)


def test_kaiser_difference_frame_special_case():
    """Paper mode (linear intensity, consecutive differences, one substep, no
    flow) is the Kaiser et al. difference frame of Sec. II: an event wherever
    f_i - f_{i-1} > C_pos or < -C_neg (the equations of Sec. III-A), with the
    Table I dense-method threshold of 2."""
    rng = np.random.default_rng(29)
    F, H, W = 5, 16, 21
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    C = 2
    r = oracle.run(frames, zero_flows(frames), times(F), substeps=1,
                   intensity=oracle.LINEAR, ref_mode=oracle.RESET,
                   c_pos_q16=C * Q, c_neg_q16=C * Q)
    t, x, y, p = oracle.unpack(r["events"])
    for i in range(1, F):
        d = frames[i].astype(int) - frames[i - 1].astype(int)
        want = set(zip(*np.nonzero(d > C))) | set(zip(*np.nonzero(d < -C)))
        sel = t == i * 1000
        got = set(zip(y[sel], x[sel]))
        assert got == want
        for yy, xx, pp in zip(y[sel], x[sel], p[sel]):
            assert pp == np.sign(d[yy, xx])


def test_sparse_with_zero_activity_threshold_equals_dense():
    rng = np.random.default_rng(31)
    F, H, W = 5, 18, 22
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    flows = rng.uniform(-3, 3, size=(F, H, W, 2)).astype(np.float32)
    kw = dict(substeps=0, max_substeps=6, c_pos_q16=12000, c_neg_q16=14000)
    d = oracle.run(frames, flows, times(F), mode=oracle.DENSE, **kw)
    s = oracle.run(frames, flows, times(F), mode=oracle.SPARSE, c_act_q16=0, **kw)
    assert np.array_equal(d["events"], s["events"])
    assert np.array_equal(d["R"], s["R"])
    big = oracle.run(frames, flows, times(F), mode=oracle.SPARSE, c_act_q16=1 << 30, **kw)
    assert len(big["events"]) == 0
    assert np.array_equal(big["R"], py_lut()[frames[0]].astype(np.int32))


def test_sparse_misses_pixels_just_under_the_activity_threshold():
    """Sec. IV-B: a pixel whose own change stays just under the threshold is not
    interpolated and emits nothing, even when the flow sweeps an edge across it."""
    H, W = 8, 24
    f0 = np.full((H, W), 60, np.uint8)
    f0[:, :8] = 200
    f1 = np.full((H, W), 60, np.uint8)
    f1[:, :12] = 200
    frames = np.stack([f0, f1])
    flows = zero_flows(frames)
    flows[1, ..., 0] = 4.0
    lut = py_lut()
    kw = dict(substeps=4, c_pos_q16=13107, c_neg_q16=13107)
    d = oracle.run(frames, flows, times(2), **kw)
    cd = abs_counts_per_pixel(d["events"], H, W)
    assert cd[:, 8:12].min() > 0  # the edge sweeps these pixels
    # pixel 9 changes by lut[200]-lut[60]; an activity threshold one above that
    # disables the whole swept band in sparse mode
    cact = int(lut[200] - lut[60]) + 1
    s = oracle.run(frames, flows, times(2), mode=oracle.SPARSE, c_act_q16=cact, **kw)
    assert len(s["events"]) == 0
    s2 = oracle.run(frames, flows, times(2), mode=oracle.SPARSE, c_act_q16=cact - 1, **kw)
    cs = abs_counts_per_pixel(s2["events"], H, W)
    assert np.array_equal(cs[:, 8:12], cd[:, 8:12])


def test_time_order_and_raster_order():
    rng = np.random.default_rng(37)
    F, H, W = 4, 15, 19
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    flows = rng.uniform(-2, 2, size=(F, H, W, 2)).astype(np.float32)
    dts = [0, 1000, 333, 70001]
    t_us = np.cumsum(dts).astype(np.int64) + 5
    r = oracle.run(frames, flows, t_us, substeps=7, c_pos_q16=9000, c_neg_q16=9000)
    t, x, y, p = oracle.unpack(r["events"])
    key = t * (1 << 32) + y * (1 << 16) + x
    assert np.all(np.diff(key) >= 0)
    # substep times are t_{i-1} + floor(k dt / N); the last one lands on t_i
    for i in range(1, F):
        tp, dt = t_us[i - 1] - t_us[0], t_us[i] - t_us[i - 1]
        allowed = {tp + (k * dt) // 7 for k in range(1, 8)}
        sel = (t > tp) & (t <= tp + dt)
        assert set(t[sel].tolist()) <= allowed
        assert tp + dt in set(t[sel].tolist())


def test_rgb_input_uses_bt601_luma():
    rng = np.random.default_rng(41)
    F, H, W = 3, 10, 14
    rgb = rng.integers(0, 256, size=(F, H, W, 3), dtype=np.uint8)
    w = rgb.astype(np.int64)
    luma = ((77 * w[..., 0] + 150 * w[..., 1] + 29 * w[..., 2] + 128) >> 8).astype(np.uint8)
    flows = rng.uniform(-2, 2, size=(F, H, W, 2)).astype(np.float32)
    a = oracle.run(rgb, flows, times(F), substeps=4)
    b = oracle.run(luma, flows, times(F), substeps=4)
    assert np.array_equal(a["events"], b["events"])


def test_per_pixel_threshold_maps():
    """A uniform map equals the uniform threshold; a map is read per pixel."""
    rng = np.random.default_rng(43)
    F, H, W = 4, 12, 16
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    flows = rng.uniform(-2, 2, size=(F, H, W, 2)).astype(np.float32)
    u = oracle.run(frames, flows, times(F), substeps=5, c_pos_q16=12345, c_neg_q16=23456)
    m = oracle.run(frames, flows, times(F), substeps=5,
                   cpos_map=np.full((H, W), 12345, np.uint16),
                   cneg_map=np.full((H, W), 23456, np.uint16))
    assert np.array_equal(u["events"], m["events"])
    # raising one pixel's thresholds past the log range silences that pixel only
    cp = np.full((H, W), 12345, np.uint16)
    cn = np.full((H, W), 23456, np.uint16)
    cp[5, 7] = cn[5, 7] = 65535
    q = oracle.run(frames, flows, times(F), substeps=5, cpos_map=cp, cneg_map=cn,
                   c_pos_q16=1, c_neg_q16=1)
    cu = abs_counts_per_pixel(u["events"], H, W)
    cq = abs_counts_per_pixel(q["events"], H, W)
    assert cq[5, 7] <= 363409 * 5 // 65535 + 5
    mask = np.ones((H, W), bool)
    mask[5, 7] = False
    assert np.array_equal(cu[mask], cq[mask])


def test_adaptive_substeps_per_frame():
    rng = np.random.default_rng(47)
    F, H, W = 6, 10, 12
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    flows = np.zeros((F, H, W, 2), np.float32)
    mags = [0, 0.0, 0.5, 3.0, 7.3, 30.0]
    for i in range(1, F):
        flows[i, 3, 4] = (mags[i] * 0.6, -mags[i] * 0.8) if i != 3 else (0.0, -3.0)
    r = oracle.run(frames, flows, times(F), substeps=0, max_substeps=8)
    for i in range(1, F):
        fx = int(np.rint(np.float64(flows[i, 3, 4, 0]) * Q))
        fy = int(np.rint(np.float64(flows[i, 3, 4, 1]) * Q))
        m = fx * fx + fy * fy
        s = math.isqrt(m)
        s += s * s < m
        assert r["n_per_frame"][i] == min(8, max(1, -(-s // Q)))


@pytest.mark.parametrize("case", range(200))
def test_second_restatement_on_random_8x8(case):
    """The substep-major C oracle and the pixel-major Python restatement agree
    event for event on random 8x8 inputs (frames, flows in [-3, 3]^2, N in
    1..6 or adaptive, all mode combinations)."""
    rng = np.random.default_rng(1000 + case)
    F = int(rng.integers(2, 4))
    H = W = 8
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    if case % 5 == 0:  # smoother content: more sub-threshold structure
        frames = np.clip(np.cumsum(rng.integers(-20, 21, size=(F, H, W)), axis=2) + 128,
                         0, 255).astype(np.uint8)
    flows = rng.uniform(-3, 3, size=(F, H, W, 2)).astype(np.float32)
    N = int(rng.integers(0, 7))
    linear = bool(case % 3 == 1)
    reset = bool(case % 4 == 2)
    sparse = bool(case % 2)
    if linear:
        cp, cn = int(rng.integers(Q, 40 * Q)), int(rng.integers(Q, 40 * Q))
    else:
        cp, cn = int(rng.integers(2000, 40000)), int(rng.integers(2000, 40000))
    cact = int(rng.integers(0, 30000)) if case % 6 == 1 else -1
    dts = rng.integers(1, 50000, size=F)
    t_us = np.cumsum(dts).astype(np.int64)
    r = oracle.run(frames, flows, t_us, mode=oracle.SPARSE if sparse else oracle.DENSE,
                   substeps=N, max_substeps=6,
                   intensity=oracle.LINEAR if linear else oracle.LOG,
                   ref_mode=oracle.RESET if reset else oracle.ACCUM,
                   c_pos_q16=cp, c_neg_q16=cn, c_act_q16=cact)
    fq = [[[(int(np.rint(np.float64(flows[i, y, x, 0]) * Q)),
             int(np.rint(np.float64(flows[i, y, x, 1]) * Q))) for x in range(W)]
           for y in range(H)] for i in range(F)]
    ev, R = exact.simulate([f.tolist() for f in frames], fq, t_us.tolist(), n_sub=N,
                           cp=cp, cn=cn, linear=linear, reset=reset, sparse=sparse,
                           c_act=cact, max_sub=6)
    t, x, y, p = oracle.unpack(r["events"])
    got = list(zip(t.tolist(), x.tolist(), y.tolist(), p.tolist()))
    assert got == ev
    if not reset:
        assert r["R"].tolist() == R


# ---------------------------------------------------------------------------
# Difference-frame interpolation (Sec. III-C): orc_run_diff


def test_diff_one_substep_is_the_kaiser_difference_frame():
    """With one substep and no flow, the interpolated difference frame is the
    difference frame D_i = L_i - L_{i-1} itself, thresholded with the Sec. III-A
    equations (strict): the Kaiser difference frame, from the third frame on
    (frames 0 and 1 only build the first difference frame)."""
    rng = np.random.default_rng(41)
    F, H, W = 6, 12, 17
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    for intensity, C in ((oracle.LINEAR, 2 * Q), (oracle.LOG, 13107)):
        r = oracle.run_diff(frames, zero_flows(frames), times(F), substeps=1,
                            intensity=intensity, c_pos_q16=C, c_neg_q16=C)
        lut = py_lut(intensity == oracle.LINEAR)
        t, x, y, p = oracle.unpack(r["events"])
        assert not np.any(t < 2 * 1000)
        for i in range(2, F):
            d = lut[frames[i]] - lut[frames[i - 1]]
            want = set(zip(*np.nonzero(d > C))) | set(zip(*np.nonzero(d < -C)))
            sel = t == i * 1000
            assert set(zip(y[sel], x[sel])) == want
            for yy, xx, pp in zip(y[sel], x[sel], p[sel]):
                assert pp == np.sign(d[yy, xx])
        assert list(r["n_per_frame"]) == [0, 0] + [1] * (F - 2)


@pytest.mark.parametrize("N", [4, 10])
@pytest.mark.parametrize("v", [(40, 120, 30), (200, 90, 210), (128, 130, 250)])
def test_diff_uniform_frames_follow_the_exact_line(N, v):
    """Uniform frames v0, v1, v2 and no flow: the difference frames are the
    constants D1 = L(v1) - L(v0) and D2 = L(v2) - L(v1), and interpolated
    difference frame k lies on the line D1 + (k/N)(D2 - D1) (within the blend's
    rounding).  Where that line is clear of the thresholds, substep k emits one
    event of its sign at every pixel."""
    H, W = 5, 7
    frames = np.stack([np.full((H, W), a, np.uint8) for a in v])
    C = 13107
    r = oracle.run_diff(frames, zero_flows(frames), times(3), substeps=N,
                        c_pos_q16=C, c_neg_q16=C)
    lut = py_lut()
    D1 = int(lut[v[1]] - lut[v[0]])
    D2 = int(lut[v[2]] - lut[v[1]])
    t, x, y, p = oracle.unpack(r["events"])
    checked = 0
    for k in range(1, N + 1):
        line = D1 + (D2 - D1) * k / N
        sel = t == 1000 + k * 1000 // N
        if abs(line - C) < 2 or abs(line + C) < 2:
            continue
        want = 1 if line > C else (-1 if line < -C else 0)
        if want == 0:
            assert not np.any(sel)
        else:
            assert sel.sum() == H * W and np.all(p[sel] == want)
        checked += 1
    assert checked >= N - 1


@pytest.mark.parametrize("s,N", [((1, 0), 3), ((0, -1), 4), ((1, 1), 2), ((-2, 1), 2)])
def test_diff_translation_reproduces_shifted_difference_samples(s, N):
    """Frames moving by m = N s whole pixels per frame: the difference frames
    move by m too (D_i(x) = D_{i-1}(x - m)), every tap is exact, and the
    interpolated difference frame k is D_{i-1} moved by k s.  Interior pixels
    emit exactly the threshold crossings of D_{i-1}(x - k s)."""
    rng = np.random.default_rng(53)
    H, W = 28, 36
    m = (N * s[0], N * s[1])
    base = rng.integers(0, 256, size=(H, W), dtype=np.uint8)
    frames = np.stack([np.roll(base, (j * m[1], j * m[0]), axis=(0, 1)) for j in range(3)])
    flows = zero_flows(frames)
    flows[2, ..., 0] = m[0]
    flows[2, ..., 1] = m[1]
    cp, cn = 20000, 15000
    r = oracle.run_diff(frames, flows, times(3), substeps=N, c_pos_q16=cp, c_neg_q16=cn)
    lut = py_lut()
    D1 = lut[frames[1]] - lut[frames[0]]
    got = per_pixel_sequences(r["events"])
    margin = 2 * N * max(abs(s[0]), abs(s[1])) + 1
    checked = 0
    for y in range(margin, H - margin):
        for x in range(margin, W - margin):
            exp = []
            for k in range(1, N + 1):
                d = int(D1[y - k * s[1], x - k * s[0]])
                if d > cp:
                    exp.append((1000 + k * 1000 // N, 1))
                elif d < -cn:
                    exp.append((1000 + k * 1000 // N, -1))
            assert got.get((x, y), []) == exp, (x, y)
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("case", range(60))
def test_diff_second_restatement_on_random_8x8(case):
    """orc_run_diff (substep-major C) and exact.simulate_diff (pixel-major
    Python) agree event for event on random 8x8 inputs."""
    rng = np.random.default_rng(5000 + case)
    F = int(rng.integers(3, 5))
    H = W = 8
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    if case % 3 == 0:
        frames = np.clip(np.cumsum(rng.integers(-20, 21, size=(F, H, W)), axis=2) + 128,
                         0, 255).astype(np.uint8)
    flows = rng.uniform(-3, 3, size=(F, H, W, 2)).astype(np.float32)
    N = int(rng.integers(0, 6))
    linear = bool(case % 4 == 1)
    if linear:
        cp, cn = int(rng.integers(Q, 40 * Q)), int(rng.integers(Q, 40 * Q))
    else:
        cp, cn = int(rng.integers(2000, 40000)), int(rng.integers(2000, 40000))
    t_us = np.cumsum(rng.integers(1, 50000, size=F)).astype(np.int64)
    r = oracle.run_diff(frames, flows, t_us, substeps=N, max_substeps=6,
                        intensity=oracle.LINEAR if linear else oracle.LOG,
                        c_pos_q16=cp, c_neg_q16=cn)
    fq = [[[(int(np.rint(np.float64(flows[i, y, x, 0]) * Q)),
             int(np.rint(np.float64(flows[i, y, x, 1]) * Q))) for x in range(W)]
           for y in range(H)] for i in range(F)]
    ev = exact.simulate_diff([f.tolist() for f in frames], fq, t_us.tolist(), n_sub=N,
                             cp=cp, cn=cn, linear=linear, max_sub=6)
    t, x, y, p = oracle.unpack(r["events"])
    assert list(zip(t.tolist(), x.tolist(), y.tolist(), p.tolist())) == ev


# ---------------------------------------------------------------------------
# Accumulated event frame (Fig. 1 caption): orc_accumulate


@pytest.mark.parametrize("v0,v1", [(60, 200), (220, 35), (128, 128)])
def test_accumulated_frame_of_a_uniform_step(v0, v1):
    """A uniform step with no flow gives every pixel floor(|D| / C) events of
    the step's sign (accumulate mode): the accumulated frame over the whole
    stream is that signed count at every pixel, and frames of disjoint time
    windows add up to it."""
    H, W, C = 6, 9, 13107
    frames = np.stack([np.full((H, W), v0, np.uint8), np.full((H, W), v1, np.uint8)])
    r = oracle.run(frames, zero_flows(frames), times(2, 1000), substeps=5,
                   c_pos_q16=C, c_neg_q16=C)
    lut = py_lut()
    d = int(lut[v1] - lut[v0])
    want = int(np.sign(d)) * (abs(d) // C)
    acc = oracle.accumulate(r["events"], W, H, 0, 1 << 40)
    assert np.all(acc == want)
    parts = np.zeros((H, W), np.int32)
    for t0 in range(0, 1001, 250):
        oracle.accumulate(r["events"], W, H, t0, t0 + 250, parts)
    assert np.array_equal(parts, acc)
    assert not np.any(oracle.accumulate(r["events"], W, H, 1001, 1 << 40))


def test_accumulated_frame_positions_polarity_and_window():
    ev = np.zeros(5, dtype=oracle.EVENT_DTYPE)
    ev["t"] = [10, 10, 20, 30, 40]
    ev["x"] = [3, 3, 0, 6, 2]
    ev["yp"] = [(1 << 1) | 1, (1 << 1) | 1, (4 << 1) | 0, (0 << 1) | 1, (9 << 1) | 1]
    acc = oracle.accumulate(ev, 7, 5, 10, 40)  # t = 40 excluded; (2, 9) outside
    want = np.zeros((5, 7), np.int32)
    want[1, 3] = 2
    want[4, 0] = -1
    want[0, 6] = 1
    assert np.array_equal(acc, want)


# ---------------------------------------------------------------------------
# Per-crossing event times (event_time = T_CROSSING, reading O16): each
# crossing of substep k happens where the straight line between the values
# of substeps k-1 and k (substep 0 = frame i-1) meets the crossed level.


def monotone_ramps(rng, F, H, W, max_step=40):
    """Per-pixel monotone luma sequences (each pixel rises or falls)."""
    v0 = rng.integers(max_step * F // 2, 256 - max_step * F // 2, size=(H, W))
    steps = rng.integers(0, max_step // 2 + 1, size=(F - 1, H, W))
    sign = np.where(rng.random((H, W)) < 0.5, 1, -1)
    seq = np.concatenate([v0[None], v0[None] + sign * np.cumsum(steps, axis=0)])
    assert seq.min() >= 0 and seq.max() <= 255
    return seq.astype(np.uint8)


@pytest.mark.parametrize("N", [1, 2, 4, 8])
@pytest.mark.parametrize("cp,cn", [(40000, 40000), (70001, 123457)])
def test_crossing_times_of_monotone_ramps_follow_the_exact_line(N, cp, cn):
    """Linear intensity, no flow: a pixel's value changes by D_i = 65536 dv
    per frame, and with N a power of two dividing dv 65536 and dt, the
    substep values and times are exact fractions of the frame step, so the
    interpolated path is the straight line through (t_{i-1}, L_{i-1}) and
    (t_i, L_i).  Every level L_0 + j Cp (rising) or L_0 - j Cn (falling) the
    line passes in frame i is crossed at t_{i-1} + floor(dt_i (level -
    L_{i-1}) / D_i), whichever substep it falls in."""
    rng = np.random.default_rng(N * 7 + cp)
    F, H, W = 6, 5, 9
    frames = monotone_ramps(rng, F, H, W)
    t_us = np.concatenate([[0], np.cumsum(rng.integers(1, 4000, size=F - 1) * 8)]).astype(np.int64)
    r = oracle.run(frames, zero_flows(frames), t_us, substeps=N, intensity=oracle.LINEAR,
                   c_pos_q16=cp, c_neg_q16=cn, event_time=oracle.T_CROSSING)
    t, x, y, p = oracle.unpack(r["events"])
    got = {}
    for ti, xi, yi, pi in zip(t.tolist(), x.tolist(), y.tolist(), p.tolist()):
        got.setdefault((xi, yi), []).append((ti, pi))
    L = frames.astype(np.int64) * Q
    for yy in range(H):
        for xx in range(W):
            want = []
            for i in range(1, F):
                a, b = L[i - 1, yy, xx], L[i, yy, xx]
                dt = int(t_us[i] - t_us[i - 1])
                base = L[0, yy, xx]
                if b > a:
                    j = (a - base) // cp + 1
                    while base + j * cp <= b:
                        want.append((int(t_us[i - 1]) + dt * (base + j * cp - a) // (b - a), 1))
                        j += 1
                elif b < a:
                    j = (base - a) // cn + 1
                    while base - j * cn >= b:
                        want.append((int(t_us[i - 1]) + dt * (a - (base - j * cn)) // (a - b), -1))
                        j += 1
            assert got.get((xx, yy), []) == want, (xx, yy)


@pytest.mark.parametrize("C", [2 * Q, 5 * Q + 123])
def test_crossing_times_reset_one_substep(C):
    """Paper mode (strict two-case test, one substep, no flow): an event
    where |L_i - L_{i-1}| > C (the Kaiser difference frame), at the time the
    straight line from L_{i-1} to L_i has moved by C: t_{i-1} +
    floor(dt C / |D|)."""
    rng = np.random.default_rng(C)
    F, H, W = 5, 7, 11
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    t_us = np.concatenate([[0], np.cumsum(rng.integers(1, 30000, size=F - 1))]).astype(np.int64)
    r = oracle.run(frames, zero_flows(frames), t_us, substeps=1, intensity=oracle.LINEAR,
                   ref_mode=oracle.RESET, c_pos_q16=C, c_neg_q16=C,
                   event_time=oracle.T_CROSSING)
    want = []
    for i in range(1, F):
        d = (frames[i].astype(np.int64) - frames[i - 1]) * Q
        dt = int(t_us[i] - t_us[i - 1])
        for yy in range(H):
            for xx in range(W):
                if abs(d[yy, xx]) > C:
                    want.append((int(t_us[i - 1]) + dt * C // abs(int(d[yy, xx])), xx, yy,
                                 1 if d[yy, xx] > 0 else -1))
    t, x, y, p = oracle.unpack(r["events"])
    assert list(zip(t.tolist(), x.tolist(), y.tolist(), p.tolist())) == want


def test_crossing_time_primitive_properties():
    """orc_crossing_time: the level at the end value gives the end time, the
    level at (or behind) the start value the start time; times are monotone in
    the level; falling is rising mirrored; a level halfway along a line of
    even duration gives the midpoint."""
    rng = np.random.default_rng(5)
    for _ in range(300):
        t0 = int(rng.integers(0, 10 ** 6))
        t1 = t0 + int(rng.integers(1, 10 ** 5))
        a = int(rng.integers(-10 ** 6, 10 ** 6))
        b = a + int(rng.integers(1, 10 ** 6))
        assert oracle.crossing_time(t0, t1, a, b, b, True) == t1
        assert oracle.crossing_time(t0, t1, a, b, a, True) == t0
        assert oracle.crossing_time(t0, t1, a, b, a - 5, True) == t0
        lv = sorted(int(v) for v in rng.integers(a, b + 1, size=5))
        ts = [oracle.crossing_time(t0, t1, a, b, v, True) for v in lv]
        assert ts == sorted(ts) and t0 <= ts[0] and ts[-1] <= t1
        for v in lv:
            assert (oracle.crossing_time(t0, t1, a, b, v, True)
                    == oracle.crossing_time(t0, t1, -a, -b, -v, False))
        assert oracle.crossing_time(0, 2 * (t1 - t0), 0, 2 * (b - a), b - a, True) == t1 - t0


@pytest.mark.parametrize("mode", [oracle.DENSE, oracle.SPARSE])
@pytest.mark.parametrize("ref", [oracle.ACCUM, oracle.RESET])
def test_crossing_times_keep_events_and_stay_inside_their_substep(mode, ref):
    """With flow, log intensity and per-pixel noise-free thresholds: the
    per-crossing run emits the same events in the same order as the
    substep-time run (only t differs); each time lies in [t_{k-1}, t_k] of
    the event's substep; a pixel's repeated crossings in one substep have
    non-decreasing times."""
    rng = np.random.default_rng(11 + mode * 2 + ref)
    F, H, W = 5, 10, 13
    frames = np.clip(np.cumsum(rng.integers(-25, 26, size=(F, H, W)), axis=0) + 128, 0,
                     255).astype(np.uint8)
    flows = rng.uniform(-2.5, 2.5, size=(F, H, W, 2)).astype(np.float32)
    t_us = np.concatenate([[0], np.cumsum(rng.integers(2000, 40000, size=F - 1))]).astype(np.int64)
    kw = dict(mode=mode, substeps=0, max_substeps=8, ref_mode=ref, c_pos_q16=9000,
              c_neg_q16=11000, c_act_q16=4000)
    a = oracle.run(frames, flows, t_us, **kw)
    b = oracle.run(frames, flows, t_us, event_time=oracle.T_CROSSING, **kw)
    assert len(a["events"]) == len(b["events"]) > 100
    assert np.array_equal(a["events"]["x"], b["events"]["x"])
    assert np.array_equal(a["events"]["yp"], b["events"]["yp"])
    assert np.array_equal(a["R"], b["R"])
    ta = a["events"]["t"].astype(np.int64)
    tb = b["events"]["t"].astype(np.int64)
    # t_{k-1} of each event from its frame's substep times
    start = 0
    lo = np.zeros_like(ta)
    for i in range(1, F):
        n_i = int(a["ev_per_frame"][i])
        N = int(a["n_per_frame"][i])
        dt = int(t_us[i] - t_us[i - 1])
        tk = [int(t_us[i - 1]) + (k * dt) // N for k in range(N + 1)]
        for e in range(start, start + n_i):
            k = tk.index(int(ta[e]))
            assert k >= 1
            lo[e] = tk[k - 1]
        start += n_i
    assert np.all(tb <= ta) and np.all(tb >= lo)
    assert np.any(tb < ta)
    same = (np.diff(ta) == 0) & (np.diff(b["events"]["x"].astype(np.int64)) == 0) & \
        (np.diff(b["events"]["yp"].astype(np.int64)) == 0)
    assert np.all(np.diff(tb)[same] >= 0)


@pytest.mark.parametrize("case", range(60))
def test_crossing_times_second_restatement_on_random_8x8(case):
    """orc_run with per-crossing times (substep-major C) and exact.simulate
    (pixel-major Python, exact rationals) agree event for event."""
    rng = np.random.default_rng(5000 + case)
    F = int(rng.integers(2, 4))
    H = W = 8
    frames = rng.integers(0, 256, size=(F, H, W), dtype=np.uint8)
    if case % 3 == 0:
        frames = np.clip(np.cumsum(rng.integers(-30, 31, size=(F, H, W)), axis=0) + 128,
                         0, 255).astype(np.uint8)
    flows = rng.uniform(-3, 3, size=(F, H, W, 2)).astype(np.float32)
    N = int(rng.integers(0, 7))
    linear = bool(case % 3 == 1)
    reset = bool(case % 4 == 2)
    sparse = bool(case % 2)
    if linear:
        cp, cn = int(rng.integers(Q, 40 * Q)), int(rng.integers(Q, 40 * Q))
    else:
        cp, cn = int(rng.integers(2000, 40000)), int(rng.integers(2000, 40000))
    cact = int(rng.integers(0, 30000)) if case % 5 == 1 else -1
    t_us = np.cumsum(rng.integers(1, 50000, size=F)).astype(np.int64)
    r = oracle.run(frames, flows, t_us, mode=oracle.SPARSE if sparse else oracle.DENSE,
                   substeps=N, max_substeps=6, intensity=oracle.LINEAR if linear else oracle.LOG,
                   ref_mode=oracle.RESET if reset else oracle.ACCUM, c_pos_q16=cp, c_neg_q16=cn,
                   c_act_q16=cact, event_time=oracle.T_CROSSING)
    fq = [[[(int(np.rint(np.float64(flows[i, y, x, 0]) * Q)),
             int(np.rint(np.float64(flows[i, y, x, 1]) * Q))) for x in range(W)]
           for y in range(H)] for i in range(F)]
    ev, R = exact.simulate([f.tolist() for f in frames], fq, t_us.tolist(), n_sub=N, cp=cp,
                           cn=cn, linear=linear, reset=reset, sparse=sparse, c_act=cact,
                           max_sub=6, crossing=True)
    t, x, y, p = oracle.unpack(r["events"])
    assert list(zip(t.tolist(), x.tolist(), y.tolist(), p.tolist())) == ev


def test_sparse_default_activity_threshold_is_the_smaller_threshold():
    """Sec. III-B with the default activity threshold min(C_pos, C_neg)
    (reading O10): a uniform linear ramp of 2 grey levels per frame with
    C_neg = 1 < 2 < C_pos = 3 levels is active at every pixel and frame, so
    the sparse run equals the dense one: one positive event per pixel when
    the accumulated rise reaches 3 levels (frame 2), none before."""
    F, H, W = 3, 6, 9
    frames = np.stack([np.full((H, W), 100 + 2 * i, np.uint8) for i in range(F)])
    kw = dict(substeps=1, intensity=oracle.LINEAR, c_pos_q16=3 * Q, c_neg_q16=1 * Q)
    d = oracle.run(frames, zero_flows(frames), times(F), mode=oracle.DENSE, **kw)
    s = oracle.run(frames, zero_flows(frames), times(F), mode=oracle.SPARSE, **kw)
    assert list(s["active_per_frame"][1:]) == [H * W, H * W]
    assert np.array_equal(s["events"].view(np.uint64), d["events"].view(np.uint64))
    t, x, y, p = oracle.unpack(s["events"])
    assert len(t) == H * W and np.all(p == 1) and np.all(t == 2 * 1000)


def test_sparse_disregards_slow_drift_below_the_activity_threshold():
    """Sec. III-B: a pixel whose value changes less than the activity
    threshold from one frame to the next is disregarded, however far it has
    drifted from its reference.  A uniform drift of 1 grey level per frame
    with C = 3 levels: the dense method emits one event per pixel every three
    frames, the sparse method none."""
    F, H, W = 7, 4, 5
    frames = np.stack([np.full((H, W), 100 + i, np.uint8) for i in range(F)])
    kw = dict(substeps=2, intensity=oracle.LINEAR, c_pos_q16=3 * Q, c_neg_q16=3 * Q)
    d = oracle.run(frames, zero_flows(frames), times(F), mode=oracle.DENSE, **kw)
    s = oracle.run(frames, zero_flows(frames), times(F), mode=oracle.SPARSE, **kw)
    assert len(d["events"]) == 2 * H * W
    assert len(s["events"]) == 0 and not np.any(s["active_per_frame"])
    assert np.array_equal(s["R"], np.full((H, W), 100 * Q))


def test_sparse_adaptive_substeps_follow_the_active_pixels_only():
    """Sec. III-B with adaptive N (reading O8): the substep count of a sparse
    frame comes from the flow of its active pixels; a larger flow at pixels
    that did not change does not raise it (the dense method takes every
    pixel's flow)."""
    F, H, W = 2, 12, 16
    frames = np.full((F, H, W), 90, np.uint8)
    frames[1, 3:6, 4:8] = 150                       # the only pixels that change
    flows = np.zeros((F, H, W, 2), np.float32)
    flows[1] = (7.0, 0.0)                           # a large flow everywhere ...
    flows[1, 3:6, 4:8] = (2.0, -0.5)                # ... but 2.06 px at the active ones
    kw = dict(substeps=0, max_substeps=16, c_pos_q16=13107, c_neg_q16=13107)
    s = oracle.run(frames, flows, times(F), mode=oracle.SPARSE, **kw)
    d = oracle.run(frames, flows, times(F), mode=oracle.DENSE, **kw)
    assert s["active_per_frame"][1] == 12
    assert s["n_per_frame"][1] == 3 and d["n_per_frame"][1] == 7
