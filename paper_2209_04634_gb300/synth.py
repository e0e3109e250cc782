"""Seeded synthetic workloads (frames, flow, timestamps, threshold maps).

This module draws inputs only: it holds none of the simulator's arithmetic
(no log table, no interpolation, no threshold test).  Both the CUDA path and
the CPU oracle consume exactly the arrays it returns.

Randomness comes from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) keyed by (seed, counter), so
every stream of numbers is a pure function of its seed.  Normal deviates use
the Box-Muller transform.

Workloads (stand-ins for the paper's recordings, which are not available):
  * ``blob_translation``  240x180 luma, 64 Gaussian blobs on mid-grey moving
    with a constant flow (3.2, -1.7) px/frame; 8 substeps; C = 0.2 (log).
  * ``warped_texture``    640x480 luma, blob + sinusoid texture advected by a
    smooth flow field of 4 windowed affine/rotation parts (max 8 px/frame,
    magnitude oscillating over time), adaptive substeps, C = 0.2 with
    per-pixel Gaussian threshold noise (sigma 0.03).  Shape of the paper's
    high events-per-frame run (Sec. IV-A: 640x480 driving sequence).
  * ``moving_rectangles`` 1280x720 RGB, static textured background plus 6
    textured rectangles bouncing at 2-12 px/frame with occlusions, 60 fps,
    10 substeps, C = 0.15.  Shape of the paper's low events-per-frame run
    (Sec. IV-A: 1280x720 table-tennis sequence, static background).
  * ``mixed_streams``     many streams of the three sizes, warped-texture
    content, one seed per stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser of a uint64 counter array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


class Rng:
    """Counter-based uniform / normal source keyed by a 64-bit seed."""

    def __init__(self, seed: int):
        self.key = np.uint64(splitmix64(np.uint64(seed & _M64)))
        self.ctr = 0

    def _bits(self, n: int) -> np.ndarray:
        c = np.arange(self.ctr, self.ctr + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return splitmix64(c ^ self.key)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self._bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Sequence:
    """One camera stream: frames, flow and simulator settings."""
    name: str
    frames: np.ndarray                 # (F, H, W) or (F, H, W, 3) uint8
    flows: np.ndarray                  # (F, H, W, 2) float32; index i: frame i-1 -> i
    t_us: np.ndarray                   # (F,) int64
    substeps: int                      # > 0 fixed, 0 adaptive
    max_substeps: int = 64
    c_pos: float = 0.2
    c_neg: float = 0.2
    cpos_map: np.ndarray | None = None  # (H, W) uint16 Q16
    cneg_map: np.ndarray | None = None
    info: dict = field(default_factory=dict)

    @property
    def height(self) -> int:
        return int(self.frames.shape[1])

    @property
    def width(self) -> int:
        return int(self.frames.shape[2])

    @property
    def channels(self) -> int:
        return 3 if self.frames.ndim == 4 else 1

    def head(self, n: int) -> "Sequence":
        """The first n frames of the sequence (same settings)."""
        return Sequence(self.name, self.frames[:n], self.flows[:n], self.t_us[:n],
                        self.substeps, self.max_substeps, self.c_pos, self.c_neg,
                        self.cpos_map, self.cneg_map, dict(self.info))


# ----------------------------------------------------------------------------
# textures

@dataclass
class Texture:
    blobs: np.ndarray      # (nb, 4): cx, cy, sigma, amplitude
    waves: np.ndarray      # (ns, 4): theta, period, amplitude, phase
    base: float = 128.0

    def eval(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        out = np.full(np.broadcast(X, Y).shape, self.base, dtype=np.float64)
        for cx, cy, s, a in self.blobs:
            r2 = (X - cx) ** 2 + (Y - cy) ** 2
            out += a * np.exp(-r2 / (2.0 * s * s))
        for th, per, a, ph in self.waves:
            out += a * np.sin(2.0 * np.pi * (X * np.cos(th) + Y * np.sin(th)) / per + ph)
        return out


def random_texture(rng: Rng, n_blobs: int, n_waves: int, W: int, H: int,
                   sigma=(3.0, 15.0), amp=(20.0, 200.0)) -> Texture:
    cx = rng.uniform(n_blobs, -0.5 * W, 1.5 * W)
    cy = rng.uniform(n_blobs, -0.5 * H, 1.5 * H)
    s = rng.uniform(n_blobs, *sigma)
    a = rng.uniform(n_blobs, *amp) * np.where(rng.uniform(n_blobs) < 0.5, -1.0, 1.0)
    th = rng.uniform(n_waves, 0.0, np.pi)
    per = rng.uniform(n_waves, 8.0, 64.0)
    wa = rng.uniform(n_waves, 10.0, 40.0)
    ph = rng.uniform(n_waves, 0.0, 2 * np.pi)
    return Texture(np.stack([cx, cy, s, a], 1), np.stack([th, per, wa, ph], 1))


def to_u8(v: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


# ----------------------------------------------------------------------------
# workloads

def blob_translation(seed: int = 3209, frames: int = 20, width: int = 240,
                     height: int = 180, flow=(3.2, -1.7), fps: float = 30.0,
                     substeps: int = 8) -> Sequence:
    """Constant-flow translation of a 64-blob texture on mid-grey."""
    rng = Rng(seed)
    tex = random_texture(rng, 64, 0, width, height)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    fr = np.empty((frames, height, width), dtype=np.uint8)
    for j in range(frames):
        fr[j] = to_u8(tex.eval(xx - j * flow[0], yy - j * flow[1]))
    fl = np.zeros((frames, height, width, 2), dtype=np.float32)
    fl[1:, :, :, 0] = flow[0]
    fl[1:, :, :, 1] = flow[1]
    t = np.rint(np.arange(frames) * 1e6 / fps).astype(np.int64)
    return Sequence("blob_translation", fr, fl, t, substeps, 64, 0.2, 0.2,
                    info={"seed": seed, "fps": fps})


def smooth_flow_field(rng: Rng, W: int, H: int, max_flow: float) -> np.ndarray:
    """Sum of 4 Gaussian-windowed affine/rotation parts, scaled to max_flow."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    F = np.zeros((H, W, 2), dtype=np.float64)
    for _ in range(4):
        cx, cy = rng.uniform(1, 0, W)[0], rng.uniform(1, 0, H)[0]
        a = rng.uniform(4, -0.02, 0.02)
        om = rng.uniform(1, -0.02, 0.02)[0]
        b = rng.uniform(2, -1.0, 1.0)
        g = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * 150.0 ** 2))
        dx, dy = xx - cx, yy - cy
        F[..., 0] += g * (a[0] * dx + (a[1] - om) * dy + b[0])
        F[..., 1] += g * ((a[2] + om) * dx + a[3] * dy + b[1])
    m = np.sqrt((F ** 2).sum(-1)).max()
    return F * (max_flow / max(m, 1e-12))


def threshold_map(rng: Rng, W: int, H: int, c: float, sigma: float,
                  c_min: float = 0.01) -> np.ndarray:
    """Per-pixel Q16 threshold max(c_min, c + sigma z), z ~ N(0, 1)."""
    z = rng.normal(W * H).reshape(H, W)
    v = np.maximum(c_min, c + sigma * z)
    return np.clip(np.rint(v * 65536.0), 1, 65535).astype(np.uint16)


def warped_texture(seed: int = 4209, frames: int = 100, width: int = 640,
                   height: int = 480, max_flow: float = 8.0, fps: float = 20.0,
                   c: float = 0.2, c_sigma: float = 0.03, max_substeps: int = 8,
                   period: float = 50.0) -> Sequence:
    """Blob + sinusoid texture advected by a smooth stationary flow field whose
    magnitude oscillates in time (so the adaptive substep count varies)."""
    rng = Rng(seed)
    tex = random_texture(rng, 32, 3, width, height)
    F = smooth_flow_field(rng, width, height, max_flow)
    phase = rng.uniform(1, 0, 2 * np.pi)[0]
    s = np.sin(2 * np.pi * np.arange(frames) / period + phase)
    s[0] = 0.0
    D = np.cumsum(s)  # displacement along F, in units of F, of frame j
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    fr = np.empty((frames, height, width), dtype=np.uint8)
    fl = np.zeros((frames, height, width, 2), dtype=np.float32)
    for j in range(frames):
        fr[j] = to_u8(tex.eval(xx - D[j] * F[..., 0], yy - D[j] * F[..., 1]))
        if j > 0:
            fl[j] = (s[j] * F).astype(np.float32)
    t = np.rint(np.arange(frames) * 1e6 / fps).astype(np.int64)
    cp = threshold_map(rng, width, height, c, c_sigma)
    cn = threshold_map(rng, width, height, c, c_sigma)
    return Sequence("warped_texture", fr, fl, t, 0, max_substeps, c, c, cp, cn,
                    info={"seed": seed, "fps": fps})


def moving_rectangles(seed: int = 5209, frames: int = 300, width: int = 1280,
                      height: int = 720, fps: float = 60.0, substeps: int = 10,
                      c: float = 0.15, n_rects: int = 6, side=(80, 240)) -> Sequence:
    """Static RGB background plus textured rectangles bouncing with occlusion.
    Flow at a pixel is the velocity of the top-most rectangle covering it in
    the target frame, else zero."""
    rng = Rng(seed)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    bg = np.stack([random_texture(rng, 32, 3, width, height, amp=(10.0, 60.0)).eval(xx, yy)
                   for _ in range(3)], -1)
    bg = to_u8(bg)
    rects = []
    for _ in range(n_rects):
        w = int(rng.uniform(1, side[0], side[1] + 1)[0])
        h = int(rng.uniform(1, side[0], side[1] + 1)[0])
        ry, rx = np.mgrid[0:h, 0:w].astype(np.float64)
        tex = np.stack([random_texture(rng, 12, 4, w, h, sigma=(3.0, 10.0)).eval(rx, ry)
                        for _ in range(3)], -1)
        speed = rng.uniform(1, 2.0, 12.0)[0]
        ang = rng.uniform(1, 0, 2 * np.pi)[0]
        pos = np.array([rng.uniform(1, 0, width - w)[0], rng.uniform(1, 0, height - h)[0]])
        rects.append({"w": w, "h": h, "tex": to_u8(tex),
                      "v": np.array([speed * np.cos(ang), speed * np.sin(ang)]), "p": pos})
    fr = np.empty((frames, height, width, 3), dtype=np.uint8)
    fl = np.zeros((frames, height, width, 2), dtype=np.float32)
    for j in range(frames):
        if j > 0:
            for r in rects:  # advance and bounce off the borders
                r["p"] = r["p"] + r["v"]
                for a, lim in ((0, width - r["w"]), (1, height - r["h"])):
                    if r["p"][a] < 0 or r["p"][a] > lim:
                        r["v"][a] = -r["v"][a]
                        r["p"][a] = min(max(r["p"][a], 0.0), float(lim))
        f = bg.copy()
        for r in rects:  # fixed z-order: later rectangles on top
            x0, y0 = int(np.rint(r["p"][0])), int(np.rint(r["p"][1]))
            f[y0:y0 + r["h"], x0:x0 + r["w"]] = r["tex"]
            if j > 0:
                fl[j, y0:y0 + r["h"], x0:x0 + r["w"]] = r["v"].astype(np.float32)
        fr[j] = f
    t = np.rint(np.arange(frames) * 1e6 / fps).astype(np.int64)
    return Sequence("moving_rectangles", fr, fl, t, substeps, 64, c, c,
                    info={"seed": seed, "fps": fps})


def mixed_streams(seed: int = 6209, frames: int = 50,
                  sizes=((240, 180, 32), (640, 480, 24), (1280, 720, 8)),
                  max_substeps: int = 8) -> list[Sequence]:
    """Many independent warped-texture streams of mixed resolutions."""
    out = []
    sid = 0
    for (w, h, count) in sizes:
        for _ in range(count):
            out.append(warped_texture(seed=seed + sid, frames=frames, width=w, height=h,
                                      max_substeps=max_substeps))
            out[-1].name = f"stream{sid}_{w}x{h}"
            sid += 1
    return out


def shifted_streams(seed: int = 6209, unique_frames: int = 6,
                    sizes=((240, 180, 32), (640, 480, 24), (1280, 720, 8)),
                    max_substeps: int = 8) -> list[Sequence]:
    """Many independent streams of mixed resolutions, cheap to generate: one
    warped-texture sequence of `unique_frames` frames per resolution, and
    each stream a distinct cyclic shift of it (frames, flow and threshold
    maps shifted together, so every stream is a valid warped texture of its
    own).  Play them to any length with `pingpong`."""
    out = []
    sid = 0
    for k, (w, h, count) in enumerate(sizes):
        base = warped_texture(seed=seed + 1000 * k, frames=unique_frames, width=w, height=h,
                              max_substeps=max_substeps)
        off = Rng(seed + 7 * k + 1).uniform(2 * count, 0.0, 1.0)
        for j in range(count):
            dy, dx = int(off[2 * j] * h), int(off[2 * j + 1] * w)
            s = Sequence(f"stream{sid}_{w}x{h}", np.roll(base.frames, (dy, dx), axis=(1, 2)),
                         np.roll(base.flows, (dy, dx), axis=(1, 2)), base.t_us.copy(),
                         base.substeps, base.max_substeps, base.c_pos, base.c_neg,
                         np.roll(base.cpos_map, (dy, dx), axis=(0, 1)),
                         np.roll(base.cneg_map, (dy, dx), axis=(0, 1)),
                         info={"seed": seed + 1000 * k, "shift": (dy, dx)})
            out.append(s)
            sid += 1
    return out


def pingpong(step: int, n: int) -> tuple[int, int, int]:
    """Frame played at `step` (>= 1) when n frames are replayed forward and
    backward, the frame before it, and the sign of the stored flow to use:
    (b, a, +1) uses flows[b] (a = b - 1); (b, a, -1) uses -flows[a]
    (a = b + 1), the exact reverse of a warped-texture step."""
    period = 2 * (n - 1)

    def at(t):
        p = t % period
        return p if p < n else period - p

    a, b = at(step - 1), at(step)
    return (b, a, 1) if b == a + 1 else (b, a, -1)
