"""Parity of the difference-frame interpolation method (Sec. III-C, SIM_DIFF)
of the CUDA path with the CPU oracle (orc_run_diff): bit-exact event streams
on ragged shapes, flows beyond the shared-memory halo, adaptive substeps,
threshold maps, linear intensity, RGB and pitched frames, and batches that
split the three-frame history across pushes."""
import numpy as np
import pytest

from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import assert_same_events, gpu_run, oracle_run
from .test_gpu_parity import random_seq

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

DIFF = evsim.SIM_DIFF


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


def check(seq, what, **kw):
    g = gpu_run(seq, DIFF, **kw)
    okw = {k: v for k, v in kw.items() if k in ("intensity", "substeps", "c_pos_q16",
                                                 "c_neg_q16", "use_maps")}
    o = oracle_run(seq, DIFF, **okw)
    assert_same_events(g["events"], o["events"], what)
    if not kw.get("batch"):
        F = seq.frames.shape[0]
        assert list(g["ev_per_frame"][1:]) == list(o["ev_per_frame"][1:F]), what
        assert list(g["n_per_frame"][2:]) == list(o["n_per_frame"][2:F]), what
    return g, o


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (17, 65), (16, 64), (33, 130),
                                 (70, 9)])
def test_diff_ragged_shapes(H, W):
    seq = random_seq(H, W, F=5, seed=7 * H + W)
    check(seq, f"diff {W}x{H}", use_maps=False)


@pytest.mark.parametrize("amp", [2.0, 15.5, 40.0])
def test_diff_flows_beyond_the_halo(amp):
    seq = random_seq(60, 150, F=4, flow_amp=amp, seed=int(amp * 3))
    check(seq, f"diff flow amplitude {amp}", use_maps=False)


def test_diff_adaptive_substeps_maps_and_linear():
    seq = synth.warped_texture(frames=6, width=130, height=70)
    g, o = check(seq, "diff warped texture (maps, adaptive N)")
    assert o["ev_per_frame"][2:].sum() > 0
    check(seq, "diff linear", use_maps=False, intensity=evsim.SIM_LINEAR,
          c_pos_q16=10 * 65536, c_neg_q16=10 * 65536, substeps=4)


def test_diff_rgb_and_host_frames():
    seq = synth.moving_rectangles(frames=5, width=200, height=120, side=(20, 50))
    check(seq, "diff rgb")
    g = gpu_run(seq, DIFF, device_inputs=False)
    assert_same_events(g["events"], oracle_run(seq, DIFF)["events"], "diff rgb host")


@pytest.mark.parametrize("batch", [1, 2, 3, 7])
def test_diff_batches_carry_the_two_frame_history(batch):
    """Pushes of 1, 2, 3 and 7 frames: the frames before each batch (i-1 and
    i-2) come from the stream's two frame rings."""
    seq = random_seq(40, 100, F=9, seed=batch, substeps=3)
    check(seq, f"diff batches of {batch}", use_maps=False, batch=batch)


def test_diff_first_two_frames_emit_nothing():
    seq = random_seq(20, 30, F=3, seed=11, substeps=2)
    g = gpu_run(seq, DIFF, use_maps=False)
    assert list(g["ev_per_frame"][:2]) == [0, 0]
    assert g["ev_per_frame"][2] > 0


def test_diff_is_single_handle_only():
    g = evsim.Group(max_streams=2, frames_per_step=1)
    with pytest.raises(evsim.SimError):
        g.admit(64, 32, mode=DIFF)
    g.close()
