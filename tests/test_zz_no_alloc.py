"""sim_step_pair_static: the allocation-free frame-pair entry point.

Some callers cannot allocate device memory while they run: code whose device
memory belongs to another framework's caching allocator, frame-rate loops
with a no-allocation rule after start-up, plug-ins handed their buffers by a
host application.  For them the library offers one frame pair per call with
all scratch in a fixed device array.

Checks, through the C ABI: on two calls in a row the events and the reference
equal the CPU oracle's and the handle API's; device memory does not shrink
across calls; an event overflow leaves an in-place reference untouched and the
same call then succeeds; separate ref_in / ref_out leave ref_in untouched; a
1920 x 1080 problem near the array's limit is exact.  This file is collected
last so that it also runs after every other GPU test in the same process; it
passes when run alone as well."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import evsim, synth


CASES = {
    # name: (sequence factory, simulator options)
    "dense_accum_fixed": (lambda: synth.blob_translation(frames=3),
                          dict(mode=evsim.SIM_DENSE)),
    "sparse_accum_adaptive": (lambda: synth.warped_texture(frames=3),
                              dict(mode=evsim.SIM_SPARSE, substeps=0, max_substeps=8)),
    "dense_reset_rgb": (lambda: synth.moving_rectangles(frames=3),
                        dict(mode=evsim.SIM_DENSE, ref_mode=evsim.SIM_REF_RESET)),
    "sparse_linear_adaptive": (lambda: synth.blob_translation(frames=3),
                               dict(mode=evsim.SIM_SPARSE, substeps=0, max_substeps=8,
                                    intensity=evsim.SIM_LINEAR, c_pos_q16=10 << 16,
                                    c_neg_q16=12 << 16)),
}


def _options(seq, opts):
    o = dict(pixel_format=evsim.SIM_RGB8 if seq.channels == 3 else evsim.SIM_LUMA8,
             substeps=seq.substeps, max_substeps=seq.max_substeps,
             c_pos_q16=oracle.q16(seq.c_pos), c_neg_q16=oracle.q16(seq.c_neg))
    o.update(opts)
    return o


def _oracle(seq, o, frames=3):
    """The oracle's events per frame (frames 1 .. frames-1) and final reference."""
    r = oracle.run(seq.frames[:frames], seq.flows[:frames], seq.t_us[:frames],
                   mode=oracle.SPARSE if o["mode"] == evsim.SIM_SPARSE else oracle.DENSE,
                   substeps=o["substeps"], max_substeps=o["max_substeps"],
                   intensity=oracle.LINEAR if o.get("intensity") == evsim.SIM_LINEAR
                   else oracle.LOG,
                   ref_mode=oracle.RESET if o.get("ref_mode") == evsim.SIM_REF_RESET
                   else oracle.ACCUM,
                   c_pos_q16=o["c_pos_q16"], c_neg_q16=o["c_neg_q16"])
    ends = np.cumsum(r["ev_per_frame"])
    per = [r["events"][(ends[i - 1] if i else 0):ends[i]] for i in range(frames)]
    return per[1:], r["R"]


def _config(W, H, o, stream):
    lib = evsim.load()
    cfg = evsim.sim_config()
    assert lib.sim_config_default(ctypes.byref(cfg), W, H) == 0
    for k, v in o.items():
        setattr(cfg, k, v)
    handle = int(getattr(stream, "cuda_stream", 0) or 0)
    cfg.cuda_stream = handle if handle else evsim.CUDA_STREAM_LEGACY
    return cfg


def _step(cfg, prev, cur, flow, t0, t1, ref_in, ref_out, events, cap):
    """One sim_step_pair_static call through the C ABI; returns (rc, n)."""
    lib = evsim.load()
    n = ctypes.c_int64(-1)
    pitch = cfg.width * cfg.pixel_format
    ptr = (lambda t: None if t is None else t.data_ptr())
    rc = lib.sim_step_pair_static(ctypes.byref(cfg), prev.data_ptr(), pitch, cur.data_ptr(),
                                  pitch, flow.data_ptr(), int(t0), int(t1), ptr(ref_in),
                                  ptr(ref_out), events.data_ptr(), int(cap), ctypes.byref(n))
    return rc, n.value


def _events(buf, n):
    return buf[:8 * n].cpu().numpy().view(evsim.EVENT_DTYPE).copy()


def _same(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(CASES))
def test_static_pair_matches_oracle_and_handle_on_two_calls(name):
    import torch
    make, opts = CASES[name]
    seq = make()
    o = _options(seq, opts)
    H, W = seq.height, seq.width
    frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
    flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    t = [int(v - seq.t_us[0]) for v in seq.t_us]
    stream = torch.cuda.current_stream()
    accum = o.get("ref_mode", evsim.SIM_REF_ACCUM) == evsim.SIM_REF_ACCUM
    cfg = _config(W, H, o, stream)

    # the allocation-free entry point: two calls in a row (a stream start,
    # then an in-place update); the caller owns every buffer
    cap = 4 * W * H
    ev_buf = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    ref = torch.empty((H, W), dtype=torch.int32, device="cuda") if accum else None
    got = []
    for i in (1, 2):
        rc, n = _step(cfg, frames[i - 1], frames[i], flows[i], t[i - 1], t[i],
                      ref if i > 1 else None, ref, ev_buf, cap)
        assert rc == evsim.SIM_OK, (i, rc, evsim.strerror(rc))
        got.append(_events(ev_buf, n))
    ref_static = ref.cpu().numpy() if accum else None

    # the oracle on the same frames
    want, R = _oracle(seq, o)
    for i in range(2):
        assert len(want[i]) > 0
        assert len(got[i]) == len(want[i]), (i, len(got[i]), len(want[i]))
        assert _same(got[i], want[i]), i
    if accum:
        assert np.array_equal(ref_static, R.reshape(H, W))

    # the handle API on the same frames
    sim = evsim.Simulator(W, H, stream=stream, **o)
    sim.push(frames[0], None, t[0])
    for i in (1, 2):
        sim.push(frames[i], flows[i], t[i])
        assert _same(sim.pop(), got[i - 1]), i
    if accum:
        assert np.array_equal(sim.reference().reshape(H, W), ref_static)
    sim.close()


@pytest.mark.gpu
def test_static_pair_allocates_nothing_and_keeps_separate_reference_input():
    import torch
    seq = synth.warped_texture(frames=3)
    o = _options(seq, dict(mode=evsim.SIM_DENSE, substeps=0, max_substeps=8))
    H, W = seq.height, seq.width
    frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
    flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    t = [int(v - seq.t_us[0]) for v in seq.t_us]
    stream = torch.cuda.current_stream()
    cfg = _config(W, H, o, stream)
    want, R = _oracle(seq, o)
    cap = 4 * W * H
    ev_buf = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    r1 = torch.empty((H, W), dtype=torch.int32, device="cuda")
    r2 = torch.empty((H, W), dtype=torch.int32, device="cuda")
    rc, n = _step(cfg, frames[0], frames[1], flows[1], t[0], t[1], None, r1, ev_buf, cap)
    assert rc == evsim.SIM_OK and _same(_events(ev_buf, n), want[0])
    r1_before = r1.clone()
    torch.cuda.synchronize()
    free = []
    for _ in range(3):  # separate reference buffers: r1 is read, r2 written
        rc, n = _step(cfg, frames[1], frames[2], flows[2], t[1], t[2], r1, r2, ev_buf, cap)
        assert rc == evsim.SIM_OK
        assert _same(_events(ev_buf, n), want[1])
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[0] == free[1] == free[2], free  # no device memory taken by the calls
    assert torch.equal(r1, r1_before)
    assert np.array_equal(r2.cpu().numpy(), R.reshape(H, W))


@pytest.mark.gpu
@pytest.mark.parametrize("start", [False, True])
def test_static_pair_overflow_keeps_the_reference_and_can_be_repeated(start):
    import torch
    seq = synth.blob_translation(frames=3)
    o = _options(seq, dict(mode=evsim.SIM_DENSE))
    H, W = seq.height, seq.width
    frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
    flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    t = [int(v - seq.t_us[0]) for v in seq.t_us]
    cfg = _config(W, H, o, torch.cuda.current_stream())
    want, R = _oracle(seq, o)
    cap = 4 * W * H
    ev_buf = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    ref = torch.empty((H, W), dtype=torch.int32, device="cuda")
    if start:  # a stream-starting step (ref_in = NULL) that overflows
        i, ref_in = 1, None
        ref.fill_(-7)
    else:      # an in-place step that overflows
        rc, n = _step(cfg, frames[0], frames[1], flows[1], t[0], t[1], None, ref, ev_buf, cap)
        assert rc == evsim.SIM_OK
        i, ref_in = 2, ref
    before = ref.clone()
    small = len(want[i - 1]) // 2
    rc, n = _step(cfg, frames[i - 1], frames[i], flows[i], t[i - 1], t[i], ref_in, ref, ev_buf,
                  small)
    assert rc == evsim.SIM_ERR_EVENT_OVERFLOW and n == 0
    assert torch.equal(ref, before)  # the caller's reference is as it was
    rc, n = _step(cfg, frames[i - 1], frames[i], flows[i], t[i - 1], t[i], ref_in, ref, ev_buf,
                  cap)
    assert rc == evsim.SIM_OK
    assert _same(_events(ev_buf, n), want[i - 1])
    if not start:
        assert np.array_equal(ref.cpu().numpy(), R.reshape(H, W))


@pytest.mark.gpu
def test_static_pair_near_its_scratch_limit():
    # 1920 x 1080 at N = 36 with separate reference buffers: the largest N
    # the 32 MiB array holds at this size (N = 37 is refused, see below)
    import torch
    seq = synth.warped_texture(frames=2, width=1920, height=1080, max_flow=6.0)
    o = _options(seq, dict(mode=evsim.SIM_DENSE, substeps=36, max_substeps=36))
    H, W = seq.height, seq.width
    frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
    flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    t = [int(v - seq.t_us[0]) for v in seq.t_us]
    cfg = _config(W, H, o, torch.cuda.current_stream())
    want, R = _oracle(seq, o, frames=2)
    cap = 2 * W * H
    ev_buf = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    r0 = torch.from_numpy(oracle.lut(oracle.LOG)[seq.frames[0]]).cuda()
    r1 = torch.empty((H, W), dtype=torch.int32, device="cuda")
    rc, n = _step(cfg, frames[0], frames[1], flows[1], t[0], t[1], r0, r1, ev_buf, cap)
    assert rc == evsim.SIM_OK, evsim.strerror(rc)
    assert n == len(want[0]) > 0
    assert _same(_events(ev_buf, n), want[0])
    assert np.array_equal(r1.cpu().numpy(), R.reshape(H, W))


def _call(lib, cfg, *, flow=64, events=64, cap=16, ref=128, ref_in=None):
    n = ctypes.c_int64(-1)
    rc = lib.sim_step_pair_static(ctypes.byref(cfg), 16, cfg.width, 32, cfg.width, flow, 0, 1000,
                                  ref_in, ref, events, cap, ctypes.byref(n))
    return rc, n.value


def _cfg(lib, W, H):
    cfg = evsim.sim_config()
    assert lib.sim_config_default(ctypes.byref(cfg), W, H) == 0
    return cfg


def test_static_pair_rejects_problems_beyond_its_scratch():
    # checked before any device work: runs without a GPU (the pointers are
    # never dereferenced)
    lib = evsim.load()
    rc, n = _call(lib, _cfg(lib, 8192, 8192))
    assert rc == evsim.SIM_ERR_TOO_LARGE and n == 0
    assert b"scratch" in lib.sim_strerror(rc)
    cfg = _cfg(lib, 1920, 1080)
    cfg.substeps = 37
    assert _call(lib, cfg, ref_in=256)[0] == evsim.SIM_ERR_TOO_LARGE
    cfg = _cfg(lib, 3840, 2160)
    cfg.substeps = 6
    assert _call(lib, cfg, ref_in=256)[0] == evsim.SIM_ERR_TOO_LARGE
    # an in-place or stream-starting accumulate step also holds the new
    # reference (4 W H bytes) in the array
    cfg = _cfg(lib, 1920, 1080)
    cfg.substeps = 26
    assert _call(lib, cfg, ref_in=128)[0] == evsim.SIM_ERR_TOO_LARGE   # in place
    assert _call(lib, cfg, ref_in=None)[0] == evsim.SIM_ERR_TOO_LARGE  # stream start
    cfg = _cfg(lib, 3840, 2160)
    cfg.substeps = 1
    assert _call(lib, cfg, ref_in=128)[0] == evsim.SIM_ERR_TOO_LARGE
    # reset mode keeps no reference: the larger limit applies
    cfg = _cfg(lib, 1920, 1080)
    cfg.substeps = 37
    cfg.ref_mode = evsim.SIM_REF_RESET
    assert _call(lib, cfg)[0] == evsim.SIM_ERR_TOO_LARGE


def test_static_pair_argument_checks():
    lib = evsim.load()
    cfg = _cfg(lib, 64, 32)
    cp = np.full(64 * 32, 13107, np.uint16)
    cfg.c_pos_map = cp.ctypes.data
    cfg.c_neg_map = cp.ctypes.data
    assert _call(lib, cfg)[0] == evsim.SIM_ERR_ARG      # maps: handle API only
    cfg = _cfg(lib, 64, 32)
    cfg.event_time = evsim.SIM_TIME_CROSSING
    assert _call(lib, cfg)[0] == evsim.SIM_ERR_ARG      # per-crossing times: handle API only
    cfg = _cfg(lib, 64, 32)
    assert _call(lib, cfg, flow=68)[0] == evsim.SIM_ERR_ARG    # flow not 8-byte aligned
    assert _call(lib, cfg, events=0)[0] == evsim.SIM_ERR_ARG   # no event buffer
    assert _call(lib, cfg, ref=None)[0] == evsim.SIM_ERR_ARG   # accumulate: ref_out needed
    cfg.c_pos_q16 = 5                                          # below the accumulate bound
    assert _call(lib, cfg)[0] == evsim.SIM_ERR_ARG
    cfg = _cfg(lib, 64, 32)
    n = ctypes.c_int64(-1)
    assert lib.sim_step_pair_static(ctypes.byref(cfg), 16, 64, 32, 64, 64, 5, 5, None, 128, 64,
                                    16, ctypes.byref(n)) == evsim.SIM_ERR_TIME
    assert lib.sim_step_pair_static(ctypes.byref(cfg), 16, 64, 32, 64, 64, 0, 1 << 32, None, 128,
                                    64, 16, ctypes.byref(n)) == evsim.SIM_ERR_TIME_RANGE
