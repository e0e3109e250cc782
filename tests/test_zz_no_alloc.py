"""sim_step_pair_static: the allocation-free frame-pair entry point.

It must give exactly the events (and, in accumulate mode, the reference) of
the handle API (sim_create / sim_push_frame / sim_pop_events) fed the same
frames, on two calls in a row that share its fixed scratch array.  This file
is collected last so that it also runs after every other GPU test in the same
process; it passes when run alone as well."""
import ctypes

import numpy as np
import pytest

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
             c_pos_q16=evsim.q16(seq.c_pos), c_neg_q16=evsim.q16(seq.c_neg))
    o.update(opts)
    return o


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(CASES))
def test_static_pair_matches_handle_on_two_calls(name):
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

    # the allocation-free entry point: two calls in a row; the caller owns
    # every buffer
    cap = 4 * W * H
    ev_buf = torch.empty(8 * cap, dtype=torch.uint8, device="cuda")
    ref = torch.empty((H, W), dtype=torch.int32, device="cuda") if accum else None
    got = []
    for i in (1, 2):
        n = evsim.step_pair_static(frames[i - 1], frames[i], flows[i], t[i - 1], t[i],
                                   ref if i > 1 else None, ref, ev_buf, stream=stream, **o)
        got.append(ev_buf[:8 * n].cpu().numpy().view(evsim.EVENT_DTYPE).copy())
    ref_static = ref.cpu().numpy() if accum else None

    # the handle API on the same frames
    sim = evsim.Simulator(W, H, stream=stream, **o)
    want = []
    sim.push(frames[0], None, t[0])
    for i in (1, 2):
        sim.push(frames[i], flows[i], t[i])
        want.append(sim.pop())
    ref_handle = sim.reference() if accum else None
    sim.close()

    for i in range(2):
        assert len(want[i]) > 0
        assert len(got[i]) == len(want[i]), (i, len(got[i]), len(want[i]))
        assert np.array_equal(got[i], want[i]), i
    if accum:
        assert np.array_equal(ref_static, ref_handle.reshape(H, W))


def _call(lib, cfg, *, flow=64, events=64, cap=16, ref=128):
    n = ctypes.c_int64(-1)
    rc = lib.sim_step_pair_static(ctypes.byref(cfg), 16, cfg.width, 32, cfg.width, flow, 0, 1000,
                                  None, ref, events, cap, ctypes.byref(n))
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
    assert _call(lib, cfg)[0] == evsim.SIM_ERR_TOO_LARGE
    cfg = _cfg(lib, 3840, 2160)
    cfg.substeps = 6
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
