"""Thin ctypes binding of the evsim C ABI (include/evsim.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library ``_build/libevsim.so``.  Loading fails loudly when that library is
missing; there is no CPU fallback.

The functions keep the C names (``sim_create``, ``sim_push_frame``,
``sim_pop_events`` ...).  ``Simulator`` wraps one handle for convenience and
accepts numpy arrays (host) or torch CUDA tensors (device).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SIM_OK, SIM_MORE = 0, 1
SIM_ERR_ARG, SIM_ERR_CUDA, SIM_ERR_OOM, SIM_ERR_TIME = -1, -2, -3, -4
SIM_ERR_TIME_RANGE, SIM_ERR_EVENT_OVERFLOW, SIM_ERR_DEVICE_TIMEOUT = -5, -6, -7
SIM_ERR_STATE, SIM_ERR_ADMIT, SIM_ERR_NO_DEVICE = -8, -9, -10
SIM_ERR_TOO_LARGE = -11
SIM_MAX_GROUP = 1024
SIM_STATIC_SCRATCH_BYTES = 32 << 20
SIM_LUMA8, SIM_RGB8 = 1, 3
SIM_DENSE, SIM_SPARSE, SIM_DIFF = 0, 1, 2
SIM_LOG, SIM_LINEAR = 0, 1
SIM_REF_ACCUM, SIM_REF_RESET = 0, 1
SIM_HOST, SIM_DEVICE = 0, 1
CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy
SIM_MAX_BATCH = 1024
SIM_TILE_AUTO, SIM_TILE_TUNE, SIM_TILE_ROWS = 0, -1, 1
SIM_HOST_STAGE, SIM_HOST_MAPPED = 0, 1
SIM_TIME_SUBSTEP, SIM_TIME_CROSSING = 0, 1
SIM_K_INIT, SIM_K_FLOWMAX, SIM_K_DENSE, SIM_K_MASK, SIM_K_SPARSE, SIM_K_ORDER, SIM_K_COPY = range(7)
KERNEL_NAMES = ["init", "flowmax", "dense", "mask", "sparse", "order", "copy"]

EVENT_DTYPE = np.dtype([("t", "<u4"), ("x", "<u2"), ("yp", "<u2")])


class sim_config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("pixel_format", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("substeps", ctypes.c_int32), ("max_substeps", ctypes.c_int32),
        ("intensity", ctypes.c_int32), ("ref_mode", ctypes.c_int32),
        ("c_pos_q16", ctypes.c_int32), ("c_neg_q16", ctypes.c_int32),
        ("c_act_q16", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("c_pos_map", ctypes.c_void_p), ("c_neg_map", ctypes.c_void_p),
        ("event_capacity", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
        ("tile_height", ctypes.c_int32), ("event_time", ctypes.c_int32),
        ("host_inputs", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class sim_stats(ctypes.Structure):
    _fields_ = [
        ("frames_pushed", ctypes.c_int64), ("frames_committed", ctypes.c_int64),
        ("events_pending", ctypes.c_int64), ("events_popped", ctypes.c_int64),
        ("last_active", ctypes.c_int64), ("last_batch_events", ctypes.c_int64),
        ("flow_clamped", ctypes.c_int64), ("last_substeps", ctypes.c_int32),
        ("max_batch", ctypes.c_int32), ("pixel_substeps", ctypes.c_int64),
        ("active_substeps", ctypes.c_int64),
        ("tile_height", ctypes.c_int32), ("block_order", ctypes.c_int32),
        ("active_pixels", ctypes.c_int64),
    ]


class simb_config(ctypes.Structure):
    _fields_ = [
        ("max_streams", ctypes.c_int32), ("frames_per_step", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_int64), ("use_graphs", ctypes.c_int32),
        ("reserved", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
        ("delivery_events", ctypes.c_int64),
    ]


class simb_delivery(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_int32), ("status", ctypes.c_int32), ("first", ctypes.c_int64),
        ("count", ctypes.c_int64), ("frames_committed", ctypes.c_int64),
        ("pixel_substeps", ctypes.c_int64),
    ]


DELIVERY_DTYPE = np.dtype([("id", "<i4"), ("status", "<i4"), ("first", "<i8"),
                           ("count", "<i8"), ("frames_committed", "<i8"),
                           ("pixel_substeps", "<i8")])


class simb_stats(ctypes.Structure):
    _fields_ = [
        ("members", ctypes.c_int32), ("tile_classes", ctypes.c_int32),
        ("bytes_used", ctypes.c_int64), ("budget", ctypes.c_int64),
        ("steps", ctypes.c_int64), ("frames_stepped", ctypes.c_int64),
        ("graph_captures", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64), ("admit_refused", ctypes.c_int64),
    ]


class sim_flow_config(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pixel_format", ctypes.c_int32),
        ("levels", ctypes.c_int32), ("radius", ctypes.c_int32), ("iterations", ctypes.c_int32),
        ("min_eig", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
    ]


# (name, restype, argtypes) of every function that include/evsim.h declares
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = [
    ("sim_threshold_q16", _I32, [ctypes.c_double]),
    ("sim_config_default", ctypes.c_int, [ctypes.POINTER(sim_config), _I32, _I32]),
    ("sim_create", ctypes.c_int, [ctypes.POINTER(sim_config), ctypes.POINTER(_VP)]),
    ("sim_push_frame", ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _I32]),
    ("sim_push_frames", ctypes.c_int, [_VP, _I32, ctypes.POINTER(_VP), _I64,
                                       ctypes.POINTER(_VP), ctypes.POINTER(_I64), _I32]),
    ("sim_pop_events", ctypes.c_int, [_VP, _VP, _I64, ctypes.POINTER(_I64), _I32]),
    ("sim_sync", ctypes.c_int, [_VP]),
    ("sim_get_stats", ctypes.c_int, [_VP, ctypes.POINTER(sim_stats)]),
    ("sim_get_reference", ctypes.c_int, [_VP, _VP]),
    ("sim_set_profiling", ctypes.c_int, [_VP, _I32]),
    ("sim_kernel_time", ctypes.c_int, [_VP, _I32, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(_I64), _I32]),
    ("sim_reset", ctypes.c_int, [_VP]),
    ("sim_destroy", ctypes.c_int, [_VP]),
    ("sim_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("sim_version", ctypes.c_char_p, []),
    ("sim_last_cuda_error", ctypes.c_char_p, []),
    ("sim_autotune", ctypes.c_int, [ctypes.POINTER(sim_config), _I32, ctypes.POINTER(_I32),
                                    ctypes.POINTER(ctypes.c_double)]),
    ("sim_autotune_sample", ctypes.c_int, [ctypes.POINTER(sim_config), _I32, ctypes.POINTER(_VP),
                                           _I64, ctypes.POINTER(_VP), ctypes.POINTER(_I64), _I32,
                                           ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_double)]),
    ("sim_autotune_save", ctypes.c_int, [ctypes.c_char_p]),
    ("sim_accumulate", ctypes.c_int, [_VP, _I64, _I32, _I32, _I64, _I64, _VP, _VP]),
    ("sim_state_size", ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    ("sim_get_state", ctypes.c_int, [_VP, _VP, _I64]),
    ("sim_set_state", ctypes.c_int, [_VP, _VP, _I64]),
    ("sim_autotune_load", ctypes.c_int, [ctypes.c_char_p]),
    ("simb_config_default", ctypes.c_int, [ctypes.POINTER(simb_config)]),
    ("simb_create", ctypes.c_int, [ctypes.POINTER(simb_config), ctypes.POINTER(_VP)]),
    ("simb_state_bytes", ctypes.c_int, [_VP, ctypes.POINTER(sim_config), ctypes.POINTER(_I64)]),
    ("simb_admit", ctypes.c_int, [_VP, ctypes.POINTER(sim_config), ctypes.POINTER(_I32)]),
    ("simb_push", ctypes.c_int, [_VP, _I32, _VP, _I64, _VP, _I64, _I32]),
    ("simb_step", ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    ("simb_step_deliver", ctypes.c_int, [_VP, ctypes.POINTER(_I64)]),
    ("simb_collect", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.POINTER(simb_delivery)),
                                    ctypes.POINTER(_I32), ctypes.POINTER(_VP),
                                    ctypes.POINTER(_I64)]),
    ("simb_delivery_ready", ctypes.c_int, [_VP]),
    ("simb_pop", ctypes.c_int, [_VP, _I32, _VP, _I64, ctypes.POINTER(_I64), _I32]),
    ("simb_stream_stats", ctypes.c_int, [_VP, _I32, ctypes.POINTER(sim_stats)]),
    ("simb_evict", ctypes.c_int, [_VP, _I32]),
    ("simb_sync", ctypes.c_int, [_VP]),
    ("simb_get_stats", ctypes.c_int, [_VP, ctypes.POINTER(simb_stats)]),
    ("simb_destroy", ctypes.c_int, [_VP]),
    ("sim_serve_run", ctypes.c_int, [_VP, _VP]),
    ("sim_selftest_bounded_wait", ctypes.c_int, [_I32, _I32, _I32, ctypes.POINTER(_I32)]),
    ("sim_flow_config_default", ctypes.c_int, [ctypes.POINTER(sim_flow_config), _I32, _I32]),
    ("sim_flow_create", ctypes.c_int, [ctypes.POINTER(sim_flow_config), ctypes.POINTER(_VP)]),
    ("sim_flow_compute", ctypes.c_int, [_VP, _VP, _I64, _VP, _I64, _VP]),
    ("sim_flow_destroy", ctypes.c_int, [_VP]),
    ("sim_step_pair_static", ctypes.c_int, [ctypes.POINTER(sim_config), _VP, _I64, _VP, _I64, _VP,
                                            _I64, _I64, _VP, _VP, _VP, _I64,
                                            ctypes.POINTER(_I64)]),
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libevsim.so (raises if it has not been built); the EVSIM_LIBRARY
    environment variable may name another build of it (the bounds-checked
    debug build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or os.environ.get("EVSIM_LIBRARY") or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError(f"evsim CUDA library not built ({p}); run "
                                   "paper_2209_04634_gb300.build.build() first")
            lib = ctypes.CDLL(p)
            for name, res, args in SIGNATURES:
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


class SimError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code in (SIM_ERR_CUDA, SIM_ERR_OOM, SIM_ERR_NO_DEVICE):
            detail = " [" + load().sim_last_cuda_error().decode() + "]"
        super().__init__(f"{what}: {strerror(code)} ({code}){detail}")


def strerror(code: int) -> str:
    return load().sim_strerror(code).decode()


def check(code: int, what: str) -> int:
    if code < 0:
        raise SimError(code, what)
    return code


def q16(c: float) -> int:
    """Threshold in log (or 8-bit) units -> Q16 integer (sim_threshold_q16)."""
    return check(int(load().sim_threshold_q16(float(c))), "sim_threshold_q16")


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


class Simulator:
    """One simulator handle.

    Frames: (H, W) or (H, W, 3) uint8; flow: (H, W, 2) float32.  numpy arrays
    are pushed as host memory, torch CUDA tensors as device memory (they must
    stay alive until the stream passes the push; pop() and sync() wait)."""

    def __init__(self, width: int, height: int, *, pixel_format: int = SIM_LUMA8,
                 mode: int = SIM_DENSE, substeps: int = 8, max_substeps: int = 16,
                 intensity: int = SIM_LOG, ref_mode: int = SIM_REF_ACCUM,
                 c_pos_q16: int = 13107, c_neg_q16: int = 13107, c_act_q16: int = -1,
                 c_pos_map=None, c_neg_map=None, event_capacity: int = 0, stream=None,
                 max_batch: int = 0, tile_height: int = SIM_TILE_AUTO,
                 event_time: int = SIM_TIME_SUBSTEP, host_inputs: int = SIM_HOST_STAGE):
        lib = load()
        cfg = sim_config()
        check(lib.sim_config_default(ctypes.byref(cfg), width, height), "sim_config_default")
        cfg.pixel_format = pixel_format
        cfg.mode = mode
        cfg.substeps = substeps
        cfg.max_substeps = max_substeps
        cfg.intensity = intensity
        cfg.ref_mode = ref_mode
        cfg.c_pos_q16 = c_pos_q16
        cfg.c_neg_q16 = c_neg_q16
        cfg.c_act_q16 = c_act_q16
        self._maps = None
        if c_pos_map is not None:
            cp = np.ascontiguousarray(c_pos_map, dtype=np.uint16)
            cn = np.ascontiguousarray(c_neg_map, dtype=np.uint16)
            self._maps = (cp, cn)
            cfg.c_pos_map = cp.ctypes.data
            cfg.c_neg_map = cn.ctypes.data
        cfg.event_capacity = event_capacity
        cfg.max_batch = max_batch
        cfg.tile_height = tile_height
        cfg.event_time = event_time
        cfg.host_inputs = host_inputs
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream))
            # handle 0 is the legacy default stream (torch's default stream):
            # name it explicitly, since a null handle asks for a library stream
            cfg.cuda_stream = handle if handle else CUDA_STREAM_LEGACY
        h = ctypes.c_void_p()
        check(lib.sim_create(ctypes.byref(cfg), ctypes.byref(h)), "sim_create")
        self._maps = None
        self.h = h
        self.width, self.height, self.channels = width, height, pixel_format
        self._lib = lib

    def push(self, frame, flow, t_us: int, pitch: int | None = None) -> None:
        dev = _is_device(frame)
        if not dev:
            frame = np.ascontiguousarray(frame, dtype=np.uint8)
            if flow is not None:
                flow = np.ascontiguousarray(flow, dtype=np.float32)
        if pitch is None:
            pitch = self.width * self.channels
        fp = 0 if flow is None else _ptr(flow)
        check(self._lib.sim_push_frame(self.h, _ptr(frame), pitch, fp or None, int(t_us),
                                       SIM_DEVICE if dev else SIM_HOST), "sim_push_frame")

    def push_many(self, frames, flows, t_us, pitch: int | None = None) -> None:
        """Push frames[0..F) with flows[i] (i -> frame i-1 to i) in one call.
        frames/flows: torch CUDA tensors (device batch) or numpy arrays (host
        batch); flows[0] is ignored for a stream's first frame."""
        F = len(t_us)
        dev = _is_device(frames)
        if not dev:
            frames = np.ascontiguousarray(frames, dtype=np.uint8)
            flows = np.ascontiguousarray(flows, dtype=np.float32)
            fb, lb = frames.strides[0], flows.strides[0]
        else:
            fb, lb = frames.stride(0) * frames.element_size(), flows.stride(0) * flows.element_size()
        f0, l0 = _ptr(frames), _ptr(flows)
        fp = (ctypes.c_void_p * F)(*[f0 + i * fb for i in range(F)])
        lp = (ctypes.c_void_p * F)(*[l0 + i * lb for i in range(F)])
        ts = (ctypes.c_int64 * F)(*[int(t) for t in t_us])
        if pitch is None:
            pitch = self.width * self.channels
        check(self._lib.sim_push_frames(self.h, F, fp, pitch, lp, ts,
                                        SIM_DEVICE if dev else SIM_HOST), "sim_push_frames")

    def pop(self, cap: int | None = None) -> np.ndarray:
        """All pending events (or up to cap) as a structured numpy array."""
        chunks = []
        while True:
            st = self.stats()
            want = st.events_pending if cap is None else min(cap, st.events_pending)
            out = np.empty(max(int(want), 1), dtype=EVENT_DTYPE)
            n = ctypes.c_int64(0)
            rc = self._lib.sim_pop_events(self.h, out.ctypes.data, int(want), ctypes.byref(n), SIM_HOST)
            check(rc, "sim_pop_events")
            chunks.append(out[: n.value])
            if rc != SIM_MORE or cap is not None:
                break
        return np.concatenate(chunks) if len(chunks) > 1 else chunks[0]

    def pop_into(self, out, cap: int) -> tuple[int, int]:
        """Pop into a caller buffer (numpy: host; torch CUDA tensor: device).
        Returns (count, return code)."""
        n = ctypes.c_int64(0)
        rc = self._lib.sim_pop_events(self.h, _ptr(out), int(cap), ctypes.byref(n),
                                      SIM_DEVICE if _is_device(out) else SIM_HOST)
        check(rc, "sim_pop_events")
        return int(n.value), rc

    def sync(self) -> int:
        return check(self._lib.sim_sync(self.h), "sim_sync")

    def stats(self) -> sim_stats:
        st = sim_stats()
        check(self._lib.sim_get_stats(self.h, ctypes.byref(st)), "sim_get_stats")
        return st

    def reference(self) -> np.ndarray:
        R = np.empty((self.height, self.width), dtype=np.int32)
        check(self._lib.sim_get_reference(self.h, R.ctypes.data), "sim_get_reference")
        return R

    def set_profiling(self, on: bool) -> None:
        check(self._lib.sim_set_profiling(self.h, 1 if on else 0), "sim_set_profiling")

    def kernel_time(self, kind: int, reset: bool = False) -> tuple[float, int]:
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        check(self._lib.sim_kernel_time(self.h, kind, ctypes.byref(ms), ctypes.byref(n),
                                        1 if reset else 0), "sim_kernel_time")
        return float(ms.value), int(n.value)

    def get_state(self) -> bytes:
        """Checkpoint of the stream's simulation state (sim_get_state)."""
        n = ctypes.c_int64(0)
        check(self._lib.sim_state_size(self.h, ctypes.byref(n)), "sim_state_size")
        buf = ctypes.create_string_buffer(int(n.value))
        check(self._lib.sim_get_state(self.h, buf, n.value), "sim_get_state")
        return buf.raw

    def set_state(self, state: bytes) -> None:
        """Restore a checkpoint taken from a handle of the same configuration."""
        buf = ctypes.create_string_buffer(state, len(state))
        check(self._lib.sim_set_state(self.h, buf, len(state)), "sim_set_state")

    def reset(self) -> None:
        check(self._lib.sim_reset(self.h), "sim_reset")

    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def make_config(width: int, height: int, *, pixel_format: int = SIM_LUMA8,
                mode: int = SIM_DENSE, substeps: int = 8, max_substeps: int = 16,
                intensity: int = SIM_LOG, ref_mode: int = SIM_REF_ACCUM,
                c_pos_q16: int = 13107, c_neg_q16: int = 13107, c_act_q16: int = -1,
                c_pos_map=None, c_neg_map=None, event_capacity: int = 0,
                tile_height: int = SIM_TILE_AUTO, event_time: int = SIM_TIME_SUBSTEP):
    """A sim_config (plus the threshold-map arrays it points to, which must
    outlive the call that reads it)."""
    cfg = sim_config()
    check(load().sim_config_default(ctypes.byref(cfg), width, height), "sim_config_default")
    cfg.pixel_format = pixel_format
    cfg.mode = mode
    cfg.substeps = substeps
    cfg.max_substeps = max_substeps
    cfg.intensity = intensity
    cfg.ref_mode = ref_mode
    cfg.c_pos_q16 = c_pos_q16
    cfg.c_neg_q16 = c_neg_q16
    cfg.c_act_q16 = c_act_q16
    keep = None
    if c_pos_map is not None:
        cp = np.ascontiguousarray(c_pos_map, dtype=np.uint16)
        cn = np.ascontiguousarray(c_neg_map, dtype=np.uint16)
        keep = (cp, cn)
        cfg.c_pos_map = cp.ctypes.data
        cfg.c_neg_map = cn.ctypes.data
    cfg.event_capacity = event_capacity
    cfg.tile_height = tile_height
    cfg.event_time = event_time
    return cfg, keep


def autotune(width: int, height: int, frames: int = 8, **kw) -> tuple[int, float, float, float]:
    """sim_autotune for a configuration (make_config keywords): returns the
    chosen tile height (16, 8 or SIM_TILE_ROWS) and the per-frame kernel
    times (us) of heights 16 and 8 and of the row kernel."""
    cfg, keep = make_config(width, height, **kw)
    th = ctypes.c_int32(0)
    us = (ctypes.c_double * 3)()
    check(load().sim_autotune(ctypes.byref(cfg), frames, ctypes.byref(th), us), "sim_autotune")
    del keep
    return int(th.value), float(us[0]), float(us[1]), float(us[2])


def autotune_sample(width: int, height: int, frames, flows, t_us,
                    **kw) -> tuple[int, float, float, float]:
    """sim_autotune_sample on a sample of a stream: frames (F, H, W[, 3]) uint8
    and flows (F, H, W, 2) float32, numpy (host) or torch CUDA tensors
    (device), t_us (F,) int64; make_config keywords for the rest."""
    cfg, keep = make_config(width, height, **kw)
    F = len(frames)
    dev = _is_device(frames)
    if not dev:
        frames = np.ascontiguousarray(frames, dtype=np.uint8)
        flows = np.ascontiguousarray(flows, dtype=np.float32)
    fr = (ctypes.c_void_p * F)(*[_ptr(frames[i]) for i in range(F)])
    fl = (ctypes.c_void_p * F)(*[_ptr(flows[i]) for i in range(F)])
    t = (ctypes.c_int64 * F)(*[int(v) for v in t_us])
    pitch = width * (3 if getattr(frames, "ndim", len(frames.shape)) == 4 else 1)
    th = ctypes.c_int32(0)
    us = (ctypes.c_double * 3)()
    check(load().sim_autotune_sample(ctypes.byref(cfg), F, fr, pitch, fl, t,
                                     SIM_DEVICE if dev else SIM_HOST, ctypes.byref(th), us),
          "sim_autotune_sample")
    del keep
    return int(th.value), float(us[0]), float(us[1]), float(us[2])


def accumulate(events, n: int, width: int, height: int, t_begin: int, t_end: int, frame,
               stream=None) -> None:
    """sim_accumulate: add the polarities of events[0..n) (a device buffer of
    sim_event records, e.g. filled by Simulator.pop_into) with
    t_begin <= t < t_end into frame (a device int32 tensor of height x width)."""
    s = 0 if stream is None else int(getattr(stream, "cuda_stream", stream))
    check(load().sim_accumulate(_ptr(events), int(n), width, height, int(t_begin), int(t_end),
                                _ptr(frame), s or None), "sim_accumulate")


def autotune_save(path: str) -> None:
    check(load().sim_autotune_save(path.encode()), "sim_autotune_save")


def autotune_load(path: str) -> None:
    check(load().sim_autotune_load(path.encode()), "sim_autotune_load")


class Group:
    """A multi-stream group (simb_*): admit streams, push frames to members,
    advance all of them with step(), pop each member's events."""

    def __init__(self, max_streams: int = 64, frames_per_step: int = 4,
                 hbm_budget_bytes: int = 0, use_graphs: bool = True, stream=None,
                 delivery_events: int = 0):
        lib = load()
        cfg = simb_config()
        check(lib.simb_config_default(ctypes.byref(cfg)), "simb_config_default")
        cfg.max_streams = max_streams
        cfg.frames_per_step = frames_per_step
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.delivery_events = delivery_events
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream))
            cfg.cuda_stream = handle if handle else CUDA_STREAM_LEGACY
        h = ctypes.c_void_p()
        check(lib.simb_create(ctypes.byref(cfg), ctypes.byref(h)), "simb_create")
        self.h = h
        self._lib = lib
        self.shapes = {}

    def state_bytes(self, width: int, height: int, **kw) -> int:
        cfg, _keep = make_config(width, height, **kw)
        out = ctypes.c_int64(0)
        check(self._lib.simb_state_bytes(self.h, ctypes.byref(cfg), ctypes.byref(out)),
              "simb_state_bytes")
        return int(out.value)

    def admit(self, width: int, height: int, **kw) -> int | None:
        """Member id, or None when admission is refused."""
        cfg, _keep = make_config(width, height, **kw)
        out = ctypes.c_int32(-1)
        rc = self._lib.simb_admit(self.h, ctypes.byref(cfg), ctypes.byref(out))
        if rc == SIM_ERR_ADMIT:
            return None
        check(rc, "simb_admit")
        self.shapes[int(out.value)] = (width, height, kw.get("pixel_format", SIM_LUMA8))
        return int(out.value)

    def push(self, sid: int, frame, flow, t_us: int, pitch: int | None = None) -> None:
        dev = _is_device(frame)
        if not dev:
            frame = np.ascontiguousarray(frame, dtype=np.uint8)
            if flow is not None:
                flow = np.ascontiguousarray(flow, dtype=np.float32)
        w, _, ch = self.shapes[sid]
        if pitch is None:
            pitch = w * ch
        fp = 0 if flow is None else _ptr(flow)
        check(self._lib.simb_push(self.h, sid, _ptr(frame), pitch, fp or None, int(t_us),
                                  SIM_DEVICE if dev else SIM_HOST), "simb_push")

    def step(self) -> int:
        n = ctypes.c_int64(0)
        check(self._lib.simb_step(self.h, ctypes.byref(n)), "simb_step")
        return int(n.value)

    def step_deliver(self) -> int:
        """Step and deliver every member's committed events to host memory
        (asynchronous; collect() returns them)."""
        n = ctypes.c_int64(0)
        check(self._lib.simb_step_deliver(self.h, ctypes.byref(n)), "simb_step_deliver")
        return int(n.value)

    def collect(self, copy: bool = True):
        """Wait for the oldest delivery: (table, events).  table: structured
        array (id, status, first, count, frames_committed) per member; events:
        EVENT_DTYPE array.  With copy=False both are views of library memory,
        valid until the next step_deliver()."""
        tab = ctypes.POINTER(simb_delivery)()
        n = ctypes.c_int32(0)
        ev = ctypes.c_void_p()
        ne = ctypes.c_int64(0)
        check(self._lib.simb_collect(self.h, ctypes.byref(tab), ctypes.byref(n), ctypes.byref(ev),
                                     ctypes.byref(ne)), "simb_collect")
        nt, nev = int(n.value), int(ne.value)
        if nt:
            buf = (ctypes.c_char * (nt * DELIVERY_DTYPE.itemsize)).from_address(
                ctypes.addressof(tab.contents))
            table = np.frombuffer(buf, dtype=DELIVERY_DTYPE)
        else:
            table = np.zeros(0, dtype=DELIVERY_DTYPE)
        if nev:
            ebuf = (ctypes.c_char * (nev * 8)).from_address(ev.value)
            events = np.frombuffer(ebuf, dtype=EVENT_DTYPE)
        else:
            events = np.zeros(0, dtype=EVENT_DTYPE)
        if copy:
            table, events = table.copy(), events.copy()
        return table, events

    def pop(self, sid: int, cap: int | None = None) -> np.ndarray:
        st = self.stream_stats(sid)
        cap = max(int(st.events_pending), 1) if cap is None else cap
        out = np.empty(cap, dtype=EVENT_DTYPE)
        n = ctypes.c_int64(0)
        check(self._lib.simb_pop(self.h, sid, out.ctypes.data, cap, ctypes.byref(n), SIM_HOST),
              "simb_pop")
        return out[: n.value]

    def pop_into(self, sid: int, out, cap: int) -> tuple[int, int]:
        """Pop into a caller buffer (numpy: host; torch CUDA tensor: device);
        returns (return code, events)."""
        n = ctypes.c_int64(0)
        rc = self._lib.simb_pop(self.h, sid, _ptr(out), cap, ctypes.byref(n),
                                SIM_DEVICE if _is_device(out) else SIM_HOST)
        check(rc, "simb_pop")
        return rc, int(n.value)

    def stream_stats(self, sid: int) -> sim_stats:
        st = sim_stats()
        check(self._lib.simb_stream_stats(self.h, sid, ctypes.byref(st)), "simb_stream_stats")
        return st

    def evict(self, sid: int) -> None:
        check(self._lib.simb_evict(self.h, sid), "simb_evict")
        self.shapes.pop(sid, None)

    def sync(self) -> None:
        check(self._lib.simb_sync(self.h), "simb_sync")

    def stats(self) -> simb_stats:
        st = simb_stats()
        check(self._lib.simb_get_stats(self.h, ctypes.byref(st)), "simb_get_stats")
        return st

    def close(self) -> None:
        if getattr(self, "h", None):
            self._lib.simb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def seq_options(seq, **kw) -> dict:
    """Simulator / Group.admit options for a synth.Sequence."""
    args = dict(pixel_format=SIM_RGB8 if seq.channels == 3 else SIM_LUMA8,
                substeps=seq.substeps, max_substeps=seq.max_substeps,
                c_pos_q16=q16(seq.c_pos), c_neg_q16=q16(seq.c_neg),
                c_pos_map=seq.cpos_map, c_neg_map=seq.cneg_map)
    args.update(kw)
    return args


def simulator_for(seq, mode: int = SIM_DENSE, **kw) -> Simulator:
    """A Simulator configured for a synth.Sequence."""
    args = dict(pixel_format=SIM_RGB8 if seq.channels == 3 else SIM_LUMA8, mode=mode,
                substeps=seq.substeps, max_substeps=seq.max_substeps,
                c_pos_q16=q16(seq.c_pos), c_neg_q16=q16(seq.c_neg),
                c_pos_map=seq.cpos_map, c_neg_map=seq.cneg_map)
    args.update(kw)
    return Simulator(seq.width, seq.height, **args)


def step_pair_static(prev_frame, frame, flow, t_prev_us: int, t_us: int, ref_in, ref_out,
                     events, *, pixel_format: int = SIM_LUMA8, mode: int = SIM_DENSE,
                     substeps: int = 8, max_substeps: int = 16, intensity: int = SIM_LOG,
                     ref_mode: int = SIM_REF_ACCUM, c_pos_q16: int = 13107,
                     c_neg_q16: int = 13107, c_act_q16: int = -1, stream=None) -> int:
    """``sim_step_pair_static`` on torch CUDA tensors (the caller allocates
    every buffer; the library call allocates nothing).  prev_frame / frame:
    (H, W) or (H, W, 3) uint8, contiguous; flow: (H, W, 2) float32; ref_in /
    ref_out: (H, W) int32 or None; events: uint8 tensor of 8 * capacity bytes.
    Returns the number of events written."""
    lib = load()
    H, W = int(frame.shape[0]), int(frame.shape[1])
    cfg = sim_config()
    check(lib.sim_config_default(ctypes.byref(cfg), W, H), "sim_config_default")
    cfg.pixel_format = pixel_format
    cfg.mode = mode
    cfg.substeps = substeps
    cfg.max_substeps = max_substeps
    cfg.intensity = intensity
    cfg.ref_mode = ref_mode
    cfg.c_pos_q16 = c_pos_q16
    cfg.c_neg_q16 = c_neg_q16
    cfg.c_act_q16 = c_act_q16
    if stream is not None:
        handle = int(getattr(stream, "cuda_stream", stream))
        cfg.cuda_stream = handle if handle else CUDA_STREAM_LEGACY
    n = ctypes.c_int64(0)
    pitch = W * pixel_format
    check(lib.sim_step_pair_static(
        ctypes.byref(cfg), _ptr(prev_frame), pitch, _ptr(frame), pitch, _ptr(flow),
        int(t_prev_us), int(t_us), None if ref_in is None else _ptr(ref_in),
        None if ref_out is None else _ptr(ref_out), _ptr(events), events.numel() // 8,
        ctypes.byref(n)), "sim_step_pair_static")
    return int(n.value)


class Flow:
    """sim_flow_* handle: pyramidal Lucas-Kanade flow between consecutive
    frames on the device.  compute(prev, cur, out) takes torch CUDA uint8
    frames ((H, W) or (H, W, 3), contiguous) and writes the flow into out, a
    float32 CUDA tensor of shape (H, W, 2), asynchronously on the handle's
    stream."""

    def __init__(self, width: int, height: int, *, pixel_format: int = SIM_LUMA8,
                 levels: int = 3, radius: int = 3, iterations: int = 3,
                 min_eig: float = 64.0, stream=None):
        self._lib = load()
        cfg = sim_flow_config()
        check(self._lib.sim_flow_config_default(ctypes.byref(cfg), width, height),
              "sim_flow_config_default")
        cfg.pixel_format = pixel_format
        cfg.levels = levels
        cfg.radius = radius
        cfg.iterations = iterations
        cfg.min_eig = float(min_eig)
        if stream is not None:
            handle = int(getattr(stream, "cuda_stream", stream))
            cfg.cuda_stream = handle if handle else CUDA_STREAM_LEGACY
        self.width, self.height, self.pixel_format = width, height, pixel_format
        h = ctypes.c_void_p()
        check(self._lib.sim_flow_create(ctypes.byref(cfg), ctypes.byref(h)), "sim_flow_create")
        self.h = h

    def compute(self, prev, cur, out) -> None:
        pitch = self.width * self.pixel_format
        check(self._lib.sim_flow_compute(self.h, _ptr(prev), pitch, _ptr(cur), pitch, _ptr(out)),
              "sim_flow_compute")

    def close(self) -> None:
        if self.h:
            check(self._lib.sim_flow_destroy(self.h), "sim_flow_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
