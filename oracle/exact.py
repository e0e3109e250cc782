"""Second, independent restatement of the simulator in pure Python integers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  It is written pixel-major
(each pixel runs all its substeps, then the events are sorted into the
(substep, row, column) output order), unlike the substep-major C oracle, so
that a loop-order or ordering slip in either shows up as a mismatch.  Pure
Python loops: tiny inputs only (8x8 and similar).

Paper: Ziegler et al., arXiv 2209.04634, Sec. III-A (dense interpolation and
the two-case threshold equations), Sec. III-B (sparse activity test) and
Sec. III-C (difference-frame interpolation, ``simulate_diff``).
"""
from __future__ import annotations

import math
from fractions import Fraction


def log_table(linear: bool) -> list[int]:
    if linear:
        return [v << 16 for v in range(256)]
    # round-half-even of 65536 ln(v + 1); Python's round() is half-even
    return [round(65536.0 * math.log(v + 1.0)) for v in range(256)]


def _sample(L, W, H, px, py):
    px = min(max(px, 0), (W - 1) << 16)
    py = min(max(py, 0), (H - 1) << 16)
    ix, iy = px >> 16, py >> 16
    fx, fy = (px & 0xFFFF) >> 4, (py & 0xFFFF) >> 4
    x1, y1 = min(ix + 1, W - 1), min(iy + 1, H - 1)

    def mix(a, b, f):
        return a + ((b - a) * f + 2048) // 4096

    top = mix(L[iy][ix], L[iy][x1], fx)
    bot = mix(L[y1][ix], L[y1][x1], fx)
    return mix(top, bot, fy)


def _crossing(t_a, t_b, i_a, i_b, level):
    """Time at which the straight line from (t_a, i_a) to (t_b, i_b) meets
    `level`, as an exact rational, floored; t_a when the level is not ahead of
    i_a in the direction of travel."""
    if i_b == i_a:
        return t_a
    s = Fraction(level - i_a, i_b - i_a)
    if s <= 0:
        return t_a
    return math.floor(t_a + (t_b - t_a) * s)


def simulate(frames, flows_q16, t_us, *, n_sub, cp, cn, linear=False, reset=False,
             sparse=False, c_act=None, cp_map=None, cn_map=None, max_sub=64, crossing=False):
    """frames: list of HxW lists of ints (luma); flows_q16: list (per frame) of
    HxW lists of (fx, fy) Q16 ints (entry 0 unused).  n_sub: fixed N or 0 for
    adaptive.  crossing: each threshold crossing gets its own time on the
    straight line between consecutive substeps.  Returns (events as
    (t, x, y, p) tuples in output order, R)."""
    lut = log_table(linear)
    H, W = len(frames[0]), len(frames[0][0])
    L0 = [[lut[v] for v in row] for row in frames[0]]
    R = [row[:] for row in L0]
    t0 = t_us[0]
    out = []
    for i in range(1, len(frames)):
        L1 = [[lut[v] for v in row] for row in frames[i]]
        dt = t_us[i] - t_us[i - 1]
        tprev = t_us[i - 1] - t0

        def thr(m, u, y, x):
            return m[y][x] if m is not None else u

        active = [[True] * W for _ in range(H)]
        if sparse:
            for y in range(H):
                for x in range(W):
                    ca = c_act if c_act is not None and c_act >= 0 else \
                        min(thr(cp_map, cp, y, x), thr(cn_map, cn, y, x))
                    active[y][x] = abs(L1[y][x] - L0[y][x]) >= ca
        N = n_sub
        if N == 0:
            m = max([flows_q16[i][y][x][0] ** 2 + flows_q16[i][y][x][1] ** 2
                     for y in range(H) for x in range(W) if active[y][x]], default=0)
            N = 1
            while N < max_sub and N * N * (1 << 32) < m:
                N += 1
        frame_events = []
        for y in range(H):
            for x in range(W):
                if not active[y][x]:
                    continue
                fx, fy = flows_q16[i][y][x]
                r = L0[y][x] if reset else R[y][x]
                c_p, c_n = thr(cp_map, cp, y, x), thr(cn_map, cn, y, x)
                i_last, t_last = L0[y][x], tprev  # substep 0 is frame i-1 itself
                for k in range(1, N + 1):
                    w = (k * 8192 + N) // (2 * N)
                    ox, oy = (fx * k) // N, (fy * k) // N
                    p0x, p0y = (x << 16) - ox, (y << 16) - oy
                    s0 = _sample(L0, W, H, p0x, p0y)
                    s1 = _sample(L1, W, H, p0x + fx, p0y + fy)
                    I = s0 + ((s1 - s0) * w + 2048) // 4096
                    tk = tprev + (k * dt) // N

                    def times(levels):
                        if not crossing:
                            return [tk] * len(levels)
                        return [_crossing(t_last, tk, i_last, I, lv) for lv in levels]

                    d = I - r
                    if reset:
                        if d > c_p:
                            frame_events.append((k, y, x, times([r + c_p]), 1))
                        elif d < -c_n:
                            frame_events.append((k, y, x, times([r - c_n]), -1))
                        r = I
                    else:
                        if d >= c_p:
                            m = d // c_p
                            frame_events.append(
                                (k, y, x, times([r + j * c_p for j in range(1, m + 1)]), 1))
                            r += m * c_p
                        elif -d >= c_n:
                            m = (-d) // c_n
                            frame_events.append(
                                (k, y, x, times([r - j * c_n for j in range(1, m + 1)]), -1))
                            r -= m * c_n
                    i_last, t_last = I, tk
                R[y][x] = r
        frame_events.sort(key=lambda e: (e[0], e[1], e[2]))
        for k, y, x, ts, p in frame_events:
            out.extend((t, x, y, p) for t in ts)
        L0 = L1
    return out, R


def simulate_diff(frames, flows_q16, t_us, *, n_sub, cp, cn, linear=False, cp_map=None,
                  cn_map=None, max_sub=64):
    """Difference-frame interpolation (Sec. III-C), pixel-major: for frame
    i >= 2 each pixel samples the difference frames D_{i-1} = L_{i-1} - L_{i-2}
    and D_i = L_i - L_{i-1} along flows_q16[i] for k = 1..N and emits an event
    where the interpolated difference exceeds C_pos or falls below -C_neg.
    Returns the events as (t, x, y, p) tuples in output order."""
    lut = log_table(linear)
    H, W = len(frames[0]), len(frames[0][0])
    L = [[[lut[v] for v in row] for row in f] for f in frames]
    t0 = t_us[0]
    out = []
    for i in range(2, len(frames)):
        Dp = [[L[i - 1][y][x] - L[i - 2][y][x] for x in range(W)] for y in range(H)]
        Dc = [[L[i][y][x] - L[i - 1][y][x] for x in range(W)] for y in range(H)]
        N = n_sub
        if N == 0:
            m = max(flows_q16[i][y][x][0] ** 2 + flows_q16[i][y][x][1] ** 2
                    for y in range(H) for x in range(W))
            N = 1
            while N < max_sub and N * N * (1 << 32) < m:
                N += 1
        dt, tprev = t_us[i] - t_us[i - 1], t_us[i - 1] - t0
        ev = []
        for y in range(H):
            for x in range(W):
                fx, fy = flows_q16[i][y][x]
                c_p = cp_map[y][x] if cp_map is not None else cp
                c_n = cn_map[y][x] if cn_map is not None else cn
                for k in range(1, N + 1):
                    w = (k * 8192 + N) // (2 * N)
                    p0x, p0y = (x << 16) - (fx * k) // N, (y << 16) - (fy * k) // N
                    s0 = _sample(Dp, W, H, p0x, p0y)
                    s1 = _sample(Dc, W, H, p0x + fx, p0y + fy)
                    I = s0 + ((s1 - s0) * w + 2048) // 4096
                    tk = tprev + (k * dt) // N
                    if I > c_p:
                        ev.append((k, y, x, tk, 1))
                    elif I < -c_n:
                        ev.append((k, y, x, tk, -1))
        ev.sort(key=lambda e: (e[0], e[1], e[2]))
        out.extend((tk, x, y, p) for k, y, x, tk, p in ev)
    return out
