"""Python side of the serving loop (``sim_serve_run`` in the C ABI).

Builds the device-resident content pools (one warped-texture sequence per
stream size, replayed forward and backward) and marshals the loop's
configuration and results.  The loop itself, the admission and the batching
are native (csrc/serve.cu); the simulation runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import evsim, synth

SIM_SERVE_GROUP, SIM_SERVE_PER_STREAM = 0, 1
POLICIES = {"group": SIM_SERVE_GROUP, "per_stream": SIM_SERVE_PER_STREAM}

# stream sizes and frame rates of the serving workload
SIZES = ((240, 180), (346, 260), (640, 480), (1280, 720), (1920, 1080))
FPS = (30, 60, 120)


class sim_serve_pool(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("frames", ctypes.c_int32),
        ("substeps", ctypes.c_int32), ("max_substeps", ctypes.c_int32),
        ("c_pos_q16", ctypes.c_int32), ("c_neg_q16", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("frame", ctypes.POINTER(ctypes.c_void_p)), ("flow", ctypes.POINTER(ctypes.c_void_p)),
        ("flow_back", ctypes.POINTER(ctypes.c_void_p)),
        ("c_pos_map", ctypes.c_void_p), ("c_neg_map", ctypes.c_void_p),
    ]


class sim_serve_stream(ctypes.Structure):
    _fields_ = [
        ("sid", ctypes.c_int32), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("fps", ctypes.c_int32), ("pool", ctypes.c_int32), ("phase", ctypes.c_int32),
        ("frames", ctypes.c_int32), ("status", ctypes.c_int32), ("events", ctypes.c_int64),
        ("digest", ctypes.c_uint64),
    ]


class sim_serve_config(ctypes.Structure):
    _fields_ = [
        ("policy", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("horizon_s", ctypes.c_double), ("warmup_s", ctypes.c_double),
        ("rate_per_s", ctypes.c_double), ("dur_min_s", ctypes.c_double),
        ("dur_max_s", ctypes.c_double), ("warm_start", ctypes.c_int32),
        ("n_pools", ctypes.c_int32), ("pools", ctypes.POINTER(sim_serve_pool)),
        ("n_fps", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("fps", ctypes.POINTER(ctypes.c_int32)), ("seed", ctypes.c_uint64),
        ("max_streams", ctypes.c_int32), ("frames_per_step", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_int64), ("events_per_pixel", ctypes.c_int64),
        ("latency_ms", ctypes.POINTER(ctypes.c_double)), ("latency_cap", ctypes.c_int64),
        ("streams", ctypes.POINTER(sim_serve_stream)), ("streams_cap", ctypes.c_int32),
        ("reserved2", ctypes.c_int32),
    ]


class sim_serve_result(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "arrived", "admitted", "never_admitted", "peak_streams", "frames_released",
        "frames_completed", "frames_failed", "events", "pixel_substeps", "steps",
        "kernel_launches")] + [(n, ctypes.c_double) for n in (
            "wall_s", "gpix_substeps_per_s", "events_per_s", "lat_p50_ms", "lat_p90_ms",
            "lat_p99_ms", "lat_max_ms", "lat_mean_ms", "admit_wait_p50_ms",
            "admit_wait_p99_ms")] + [
        ("latencies", ctypes.c_int64), ("streams_written", ctypes.c_int32),
        ("reserved", ctypes.c_int32)]


DIGEST_M = 0x9E3779B97F4A7C15


def digest(events: np.ndarray) -> int:
    """The serving loop's event-stream digest: Horner's rule over the events
    as 64-bit words, h = h * M + e (mod 2^64)."""
    w = np.ascontiguousarray(events).view(np.uint64)
    n = w.size
    if n == 0:
        return 0
    pw = np.empty(n, np.uint64)
    pw[-1] = 1
    if n > 1:
        pw[:-1] = np.uint64(DIGEST_M)
        pw[:-1] = np.cumprod(pw[:-1][::-1], dtype=np.uint64)[::-1]
    with np.errstate(over="ignore"):
        return int(np.sum(w * pw, dtype=np.uint64))


class Pools:
    """Device-resident content of the serving workload: for each size, a
    warped-texture sequence of `frames` frames (luma), its flows and the
    reversed flows, and the per-pixel threshold maps."""

    def __init__(self, sizes=SIZES, frames: int = 6, seed: int = 8209, max_substeps: int = 8):
        import torch
        self.seqs, self._keep = [], []
        arr = (sim_serve_pool * len(sizes))()
        for i, (w, h) in enumerate(sizes):
            s = synth.warped_texture(seed=seed + 1000 * i, frames=frames, width=w, height=h,
                                     max_substeps=max_substeps)
            fr = torch.from_numpy(s.frames).cuda()
            fl = torch.from_numpy(s.flows).cuda()
            rfl = -fl
            ptr = lambda t: (ctypes.c_void_p * frames)(*[int(t[u].data_ptr()) for u in range(frames)])
            pf, pfl, prf = ptr(fr), ptr(fl), ptr(rfl)
            cp = np.ascontiguousarray(s.cpos_map, dtype=np.uint16)
            cn = np.ascontiguousarray(s.cneg_map, dtype=np.uint16)
            p = arr[i]
            p.width, p.height, p.frames = w, h, frames
            p.substeps, p.max_substeps = s.substeps, s.max_substeps
            p.c_pos_q16, p.c_neg_q16 = evsim.q16(s.c_pos), evsim.q16(s.c_neg)
            p.frame = ctypes.cast(pf, ctypes.POINTER(ctypes.c_void_p))
            p.flow = ctypes.cast(pfl, ctypes.POINTER(ctypes.c_void_p))
            p.flow_back = ctypes.cast(prf, ctypes.POINTER(ctypes.c_void_p))
            p.c_pos_map, p.c_neg_map = cp.ctypes.data, cn.ctypes.data
            self._keep += [fr, fl, rfl, pf, pfl, prf, cp, cn]
            self.seqs.append(s)
        self.arr = arr
        self.sizes = tuple(sizes)
        self.frames = frames

    def stream_frames(self, pool: int, phase: int, n: int):
        """Frames 0..n-1 of a stream (content index, flow source) exactly as the
        serving loop feeds them: (frames (n,H,W), flows (n,H,W,2))."""
        s = self.seqs[pool]
        U = self.frames
        period = 2 * (U - 1)

        def at(t):
            p = t % period
            return p if p < U else period - p

        fr = np.stack([s.frames[at(j + phase)] for j in range(n)])
        fl = np.zeros((n,) + s.flows.shape[1:], np.float32)
        for j in range(1, n):
            b, a = at(j + phase), at(j - 1 + phase)
            fl[j] = s.flows[b] if b == a + 1 else -s.flows[a]
        return fr, fl


def run(pools: Pools, policy: str = "group", *, mode: int = evsim.SIM_DENSE,
        horizon_s: float = 15.0, warmup_s: float = 2.0, rate_per_s: float = 4.0,
        dur_s=(10.0, 60.0), fps=FPS, seed: int = 9209, warm_start: bool = True,
        max_streams: int = 512, frames_per_step: int = 2, hbm_budget_bytes: int = 8 << 30,
        events_per_pixel: int = 2, streams_cap: int = 4096, keep_latencies: bool = False):
    """One serving run; returns (result dict, per-stream records)."""
    lib = evsim.load()
    cfg = sim_serve_config()
    cfg.policy = POLICIES[policy]
    cfg.mode = mode
    cfg.horizon_s, cfg.warmup_s, cfg.rate_per_s = horizon_s, warmup_s, rate_per_s
    cfg.dur_min_s, cfg.dur_max_s = dur_s
    cfg.warm_start = 1 if warm_start else 0
    cfg.n_pools = len(pools.sizes)
    cfg.pools = ctypes.cast(pools.arr, ctypes.POINTER(sim_serve_pool))
    fps_arr = (ctypes.c_int32 * len(fps))(*fps)
    cfg.n_fps = len(fps)
    cfg.fps = ctypes.cast(fps_arr, ctypes.POINTER(ctypes.c_int32))
    cfg.seed = seed
    cfg.max_streams = max_streams
    cfg.frames_per_step = frames_per_step
    cfg.hbm_budget_bytes = hbm_budget_bytes
    cfg.events_per_pixel = events_per_pixel
    lat = None
    if keep_latencies:
        lat = (ctypes.c_double * 4_000_000)()
        cfg.latency_ms = ctypes.cast(lat, ctypes.POINTER(ctypes.c_double))
        cfg.latency_cap = 4_000_000
    recs = (sim_serve_stream * streams_cap)()
    cfg.streams = ctypes.cast(recs, ctypes.POINTER(sim_serve_stream))
    cfg.streams_cap = streams_cap
    res = sim_serve_result()
    evsim.check(lib.sim_serve_run(ctypes.addressof(cfg), ctypes.addressof(res)), "sim_serve_run")
    out = {name: getattr(res, name) for name, _ in sim_serve_result._fields_
           if not name.startswith("reserved")}
    if lat is not None:
        out["latency_ms"] = np.ctypeslib.as_array(lat)[: min(res.latencies, 4_000_000)].copy()
    streams = [{n: getattr(recs[i], n) for n, _ in sim_serve_stream._fields_}
               for i in range(res.streams_written)]
    return out, streams
