"""Plain CPU oracle of the flow-interpolation event simulator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never imports, links or calls
it, and the two share no code: this package holds its own C source
(``evsim_oracle.c``), its own LUT, its own fixed-point helpers.

``run()`` is a ctypes wrapper of ``orc_run`` (the whole per-stream method of
Sec. III-A / III-B of Ziegler et al., arXiv 2209.04634, as restated in
``evsim_oracle.c``; ``event_time=T_CROSSING`` gives each threshold crossing
its own time inside its interpolation step, ``orc_crossing_time``); ``run_diff()`` wraps ``orc_run_diff`` (the
difference-frame interpolation of Sec. III-C); ``flow_lk()`` wraps
``orc_flow_lk`` (the pyramidal Lucas-Kanade flow the paper's sparse and
difference simulators take their flow from).  ``exact.py`` is a second, pixel-major restatement in
pure Python integers for tiny inputs.

Parity status of each function is pinned by ``tests/test_oracle_pins.py``
(closed forms, invariants, the Kaiser difference-frame special case,
exhaustive 1x1 enumeration, exact integer translations, plane images).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "evsim_oracle.c")
_lock = threading.Lock()
_lib = None

EVENT_DTYPE = np.dtype([("t", "<u4"), ("x", "<u2"), ("yp", "<u2")])

DENSE, SPARSE = 0, 1
LOG, LINEAR = 0, 1
ACCUM, RESET = 0, 1
T_SUBSTEP, T_CROSSING = 0, 1


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32),
        ("height", ctypes.c_int32),
        ("channels", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("substeps", ctypes.c_int32),
        ("max_substeps", ctypes.c_int32),
        ("intensity", ctypes.c_int32),
        ("ref_mode", ctypes.c_int32),
        ("c_pos_q16", ctypes.c_int32),
        ("c_neg_q16", ctypes.c_int32),
        ("c_act_q16", ctypes.c_int32),
        ("event_time", ctypes.c_int32),
        ("row_begin", ctypes.c_int32),
        ("row_end", ctypes.c_int32),
    ]


class LkConfig(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("min_eig", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_SO) >= os.path.getmtime(os.path.join(_HERE, "evsim_oracle.h"))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def use_library(path: str | None) -> None:
    """Point the wrapper at another build of the oracle source (the mutation
    tests load deliberately broken copies); None restores the default."""
    global _lib, _override
    with _lock:
        _override = path
        _lib = None


_override = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_override or build())
            lib.orc_lut.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
            lib.orc_luma.argtypes = [ctypes.c_int32] * 3
            lib.orc_luma.restype = ctypes.c_int32
            lib.orc_flow_q16.argtypes = [ctypes.c_float, ctypes.POINTER(ctypes.c_int32)]
            lib.orc_flow_q16.restype = ctypes.c_int32
            lib.orc_bilinear.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_int64]
            lib.orc_bilinear.restype = ctypes.c_int32
            lib.orc_adaptive_substeps.argtypes = [ctypes.c_int64, ctypes.c_int32]
            lib.orc_adaptive_substeps.restype = ctypes.c_int32
            lib.orc_crossing_time.argtypes = [ctypes.c_int64] * 5 + [ctypes.c_int32]
            lib.orc_crossing_time.restype = ctypes.c_int64
            vp = ctypes.c_void_p
            lib.orc_run.argtypes = [ctypes.POINTER(OrcConfig), ctypes.c_int32, vp, vp, vp,
                                    vp, vp, vp, ctypes.c_int64, vp, vp, vp, vp, vp]
            lib.orc_run.restype = ctypes.c_int64
            lib.orc_run_diff.argtypes = [ctypes.POINTER(OrcConfig), ctypes.c_int32, vp, vp, vp,
                                         vp, vp, vp, ctypes.c_int64, vp, vp, vp]
            lib.orc_run_diff.restype = ctypes.c_int64
            lib.orc_accumulate.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int64, ctypes.c_int64, vp]
            lib.orc_accumulate.restype = None
            lib.orc_flow_lk.argtypes = [ctypes.POINTER(LkConfig), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, vp, vp, vp]
            lib.orc_flow_lk.restype = ctypes.c_int
            _lib = lib
    return _lib


def lut(intensity: int = LOG) -> np.ndarray:
    out = (ctypes.c_int32 * 256)()
    _load().orc_lut(intensity, out)
    return np.frombuffer(out, dtype=np.int32).copy()


def luma(r: int, g: int, b: int) -> int:
    return int(_load().orc_luma(r, g, b))


def flow_q16(f: float) -> tuple[int, bool]:
    cl = ctypes.c_int32(0)
    v = _load().orc_flow_q16(ctypes.c_float(f), ctypes.byref(cl))
    return int(v), bool(cl.value)


def bilinear(L: np.ndarray, px: int, py: int) -> int:
    L = np.ascontiguousarray(L, dtype=np.int32)
    H, W = L.shape
    return int(_load().orc_bilinear(L.ctypes.data, W, H, px, py))


def adaptive_substeps(max_f2: int, max_substeps: int) -> int:
    return int(_load().orc_adaptive_substeps(max_f2, max_substeps))


def crossing_time(t_prev: int, t_cur: int, i_prev: int, i_cur: int, level: int,
                  rising: bool) -> int:
    """orc_crossing_time: the time at which a value moving linearly from i_prev
    (at t_prev) to i_cur (at t_cur) reaches `level` (floor; t_prev for a level
    at or behind i_prev)."""
    return int(_load().orc_crossing_time(t_prev, t_cur, i_prev, i_cur, level, int(rising)))


def q16(c: float) -> int:
    """Host conversion of a threshold in log (or 8-bit) units to Q16."""
    return int(round(abs(float(c)) * 65536.0))


def run(frames: np.ndarray, flows: np.ndarray | None, t_us, *, mode: int = DENSE,
        substeps: int = 8, max_substeps: int = 64, intensity: int = LOG,
        ref_mode: int = ACCUM, c_pos_q16: int = 13107, c_neg_q16: int = 13107,
        c_act_q16: int = -1, cpos_map: np.ndarray | None = None,
        cneg_map: np.ndarray | None = None, cap: int | None = None,
        event_time: int = T_SUBSTEP, rows: tuple[int, int] | None = None) -> dict:
    """Run the oracle over a whole sequence.

    frames: (F, H, W) uint8 luma or (F, H, W, 3) uint8 RGB.
    flows : (F, H, W, 2) float32, index i holds the flow of frame i-1 -> i
            (entry 0 unused); may be None when F == 1.
    rows  : (begin, end): simulate only these rows (a band of run_bands);
            the other rows' R entries are not meaningful.
    Returns a dict with 'events' (structured array, EVENT_DTYPE), 'R' (H, W)
    int32, 'n_per_frame', 'ev_per_frame', 'active_per_frame', 'clamped'.
    """
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    F = frames.shape[0]
    H, W = frames.shape[1], frames.shape[2]
    ch = 3 if frames.ndim == 4 else 1
    t = np.ascontiguousarray(np.asarray(t_us, dtype=np.int64))
    assert t.shape == (F,)
    if flows is not None:
        flows = np.ascontiguousarray(flows, dtype=np.float32)
        assert flows.shape == (F, H, W, 2), flows.shape
    cfg = OrcConfig(W, H, ch, mode, substeps, max_substeps, intensity, ref_mode,
                    c_pos_q16, c_neg_q16, c_act_q16, event_time,
                    rows[0] if rows else 0, rows[1] if rows else 0)
    maps = []
    for m in (cpos_map, cneg_map):
        if m is None:
            maps.append(None)
        else:
            m = np.ascontiguousarray(m, dtype=np.uint16)
            assert m.shape == (H, W)
            maps.append(m)
    R = np.zeros((H, W), dtype=np.int32)
    npf = np.zeros(F, dtype=np.int32)
    epf = np.zeros(F, dtype=np.int64)
    apf = np.zeros(F, dtype=np.int64)
    clamped = ctypes.c_int64(0)
    if cap is None:
        cap = 1 << 16
    lib = _load()

    def call(capacity):
        ev = np.zeros(max(capacity, 1), dtype=EVENT_DTYPE)
        n = lib.orc_run(ctypes.byref(cfg), F, frames.ctypes.data,
                        None if flows is None else flows.ctypes.data, t.ctypes.data,
                        None if maps[0] is None else maps[0].ctypes.data,
                        None if maps[1] is None else maps[1].ctypes.data,
                        ev.ctypes.data, capacity, R.ctypes.data, npf.ctypes.data,
                        epf.ctypes.data, apf.ctypes.data, ctypes.byref(clamped))
        return n, ev

    n, ev = call(cap)
    if n > cap:
        n, ev = call(int(n))
    if n < 0:
        raise ValueError(f"oracle rejected the input (code {n})")
    return {"events": ev[:n].copy(), "R": R, "n_per_frame": npf, "ev_per_frame": epf,
            "active_per_frame": apf, "clamped": int(clamped.value)}


def run_bands(frames: np.ndarray, flows: np.ndarray | None, t_us, *, threads: int,
              substeps: int = 8, max_substeps: int = 64, **kw) -> dict:
    """``run`` split into `threads` row bands run concurrently (the C call
    releases the interpreter lock), merged into the single run's output: the
    events of every (frame, substep) in band order, the reference by rows,
    the per-frame counts summed.  The merge orders events by time, so it
    needs substep times that strictly increase, i.e. every frame interval at
    least N_max microseconds (checked); per-crossing times are refused."""
    import concurrent.futures as cf
    if kw.get("event_time", T_SUBSTEP) != T_SUBSTEP:
        raise ValueError("run_bands merges substep times only")
    t = np.asarray(t_us, dtype=np.int64)
    nmax = substeps if substeps > 0 else max_substeps
    if len(t) > 1 and int(np.diff(t).min()) < nmax:
        raise ValueError("run_bands needs frame intervals of at least N_max microseconds")
    H = frames.shape[1]
    threads = max(1, min(int(threads), H))
    edges = [H * j // threads for j in range(threads + 1)]
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda j: run(frames, flows, t_us, substeps=substeps,
                                          max_substeps=max_substeps,
                                          rows=(edges[j], edges[j + 1]), **kw),
                            range(threads)))
    ev = np.concatenate([p["events"] for p in parts])
    ev = ev[np.argsort(ev["t"], kind="stable")]
    R = parts[0]["R"].copy()
    for j, p in enumerate(parts):
        R[edges[j]:edges[j + 1]] = p["R"][edges[j]:edges[j + 1]]
    return {"events": ev, "R": R, "n_per_frame": parts[0]["n_per_frame"],
            "ev_per_frame": sum(p["ev_per_frame"] for p in parts),
            "active_per_frame": sum(p["active_per_frame"] for p in parts),
            "clamped": sum(p["clamped"] for p in parts), "threads": threads}


def run_diff(frames: np.ndarray, flows: np.ndarray | None, t_us, *, substeps: int = 8,
             max_substeps: int = 64, intensity: int = LOG, c_pos_q16: int = 13107,
             c_neg_q16: int = 13107, cpos_map: np.ndarray | None = None,
             cneg_map: np.ndarray | None = None, cap: int | None = None) -> dict:
    """Run the difference-frame interpolation oracle (orc_run_diff, Sec. III-C)
    over a whole sequence; flows[i] is the flow between difference frames i-1
    and i.  Returns 'events', 'n_per_frame', 'ev_per_frame', 'clamped'."""
    frames = np.ascontiguousarray(frames, dtype=np.uint8)
    F = frames.shape[0]
    H, W = frames.shape[1], frames.shape[2]
    ch = 3 if frames.ndim == 4 else 1
    t = np.ascontiguousarray(np.asarray(t_us, dtype=np.int64))
    if flows is not None:
        flows = np.ascontiguousarray(flows, dtype=np.float32)
        assert flows.shape == (F, H, W, 2), flows.shape
    cfg = OrcConfig(W, H, ch, 0, substeps, max_substeps, intensity, RESET,
                    c_pos_q16, c_neg_q16, -1, T_SUBSTEP)
    maps = [None if m is None else np.ascontiguousarray(m, dtype=np.uint16)
            for m in (cpos_map, cneg_map)]
    npf = np.zeros(F, dtype=np.int32)
    epf = np.zeros(F, dtype=np.int64)
    clamped = ctypes.c_int64(0)
    lib = _load()

    def call(capacity):
        ev = np.zeros(max(capacity, 1), dtype=EVENT_DTYPE)
        n = lib.orc_run_diff(ctypes.byref(cfg), F, frames.ctypes.data,
                             None if flows is None else flows.ctypes.data, t.ctypes.data,
                             None if maps[0] is None else maps[0].ctypes.data,
                             None if maps[1] is None else maps[1].ctypes.data,
                             ev.ctypes.data, capacity, npf.ctypes.data, epf.ctypes.data,
                             ctypes.byref(clamped))
        return n, ev

    n, ev = call(cap if cap is not None else 1 << 16)
    if n > len(ev):
        n, ev = call(int(n))
    if n < 0:
        raise ValueError(f"oracle rejected the input (code {n})")
    return {"events": ev[:n].copy(), "n_per_frame": npf, "ev_per_frame": epf,
            "clamped": int(clamped.value)}


def flow_lk(f0: np.ndarray, f1: np.ndarray, *, levels: int = 3, radius: int = 3,
            iterations: int = 3, min_eig: float = 64.0) -> np.ndarray:
    """orc_flow_lk: pyramidal Lucas-Kanade flow from f0 to f1 ((H, W) or
    (H, W, 3) uint8); returns (H, W, 2) int32, Q16 px."""
    f0 = np.ascontiguousarray(f0, dtype=np.uint8)
    f1 = np.ascontiguousarray(f1, dtype=np.uint8)
    assert f0.shape == f1.shape
    H, W = f0.shape[:2]
    ch = 3 if f0.ndim == 3 else 1
    out = np.zeros((H, W, 2), dtype=np.int32)
    cfg = LkConfig(levels, radius, iterations, 0, float(min_eig))
    rc = _load().orc_flow_lk(ctypes.byref(cfg), W, H, ch, f0.ctypes.data, f1.ctypes.data,
                             out.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle rejected the input (code {rc})")
    return out


def accumulate(events: np.ndarray, W: int, H: int, t_begin: int, t_end: int,
               frame: np.ndarray | None = None) -> np.ndarray:
    """orc_accumulate: the accumulated event frame of the events with
    t_begin <= t < t_end, added to `frame` (a new zero frame if None)."""
    ev = np.ascontiguousarray(events, dtype=EVENT_DTYPE)
    out = np.zeros((H, W), dtype=np.int32) if frame is None else frame
    assert out.dtype == np.int32 and out.flags.c_contiguous and out.shape == (H, W)
    _load().orc_accumulate(ev.ctypes.data if ev.size else None, len(ev), W, H, int(t_begin),
                           int(t_end), out.ctypes.data)
    return out


def unpack(events: np.ndarray):
    """Split packed events into (t, x, y, p) arrays with p in {+1, -1}."""
    t = events["t"].astype(np.int64)
    x = events["x"].astype(np.int64)
    y = (events["yp"] >> 1).astype(np.int64)
    p = np.where(events["yp"] & 1, 1, -1).astype(np.int64)
    return t, x, y, p
