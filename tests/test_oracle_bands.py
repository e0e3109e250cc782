"""The oracle split into row bands run on several host threads (the all-core
CPU baseline) reproduces the single run exactly: same events in the same
order, same reference, same per-frame counts."""
import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import synth


def _same(a, b):
    return a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))


@pytest.mark.parametrize("threads", [1, 2, 3, 7])
@pytest.mark.parametrize("case", ["dense_fixed", "sparse_adaptive_maps", "reset_rgb",
                                  "sparse_fixed_rgb"])
def test_row_bands_equal_the_single_run(case, threads):
    if case == "dense_fixed":
        s = synth.blob_translation(frames=4, width=96, height=50)
        kw = dict(mode=oracle.DENSE, substeps=8)
    elif case == "sparse_adaptive_maps":
        s = synth.warped_texture(frames=4, width=120, height=72)
        kw = dict(mode=oracle.SPARSE, substeps=0, max_substeps=8, cpos_map=s.cpos_map,
                  cneg_map=s.cneg_map)
    elif case == "reset_rgb":
        s = synth.moving_rectangles(frames=4, width=160, height=90, side=(20, 50))
        kw = dict(mode=oracle.DENSE, substeps=10, ref_mode=oracle.RESET)
    else:
        s = synth.moving_rectangles(frames=4, width=160, height=90, side=(20, 50))
        kw = dict(mode=oracle.SPARSE, substeps=10)
    kw.update(c_pos_q16=oracle.q16(s.c_pos), c_neg_q16=oracle.q16(s.c_neg))
    one = oracle.run(s.frames, s.flows, s.t_us, **kw)
    many = oracle.run_bands(s.frames, s.flows, s.t_us, threads=threads, **kw)
    assert len(one["events"]) > 0
    assert _same(many["events"], one["events"])
    if kw.get("ref_mode", oracle.ACCUM) == oracle.ACCUM:
        assert np.array_equal(many["R"], one["R"])
    for k in ("n_per_frame", "ev_per_frame", "active_per_frame"):
        assert np.array_equal(many[k], one[k]), k
    assert many["clamped"] == one["clamped"]


def test_row_bands_refuse_what_they_cannot_merge():
    s = synth.blob_translation(frames=3, width=32, height=16)
    with pytest.raises(ValueError):
        oracle.run_bands(s.frames, s.flows, s.t_us, threads=2, event_time=oracle.T_CROSSING)
    t = np.array([0, 5, 10], np.int64)  # intervals shorter than N = 8 us
    with pytest.raises(ValueError):
        oracle.run_bands(s.frames, s.flows, t, threads=2, substeps=8)
