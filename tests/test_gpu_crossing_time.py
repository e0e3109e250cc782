"""Per-crossing event times (SIM_TIME_CROSSING) on the CUDA path against the
oracle (orc_run with ORC_T_CROSSING): bit-exact events, order and
reference, through the C ABI, for dense and sparse, both reference modes,
both intensity tables, threshold maps, fixed and adaptive N, flows beyond
the shared halo, rows of multi-crossings, ragged shapes, batches and host
inputs."""
import numpy as np
import pytest

from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import assert_same_events, gpu_run, oracle_run
from .test_gpu_parity import random_seq

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

XT = evsim.SIM_TIME_CROSSING


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


def check(seq, mode, what, **kw):
    g = gpu_run(seq, mode, event_time=XT, **kw)
    okw = {k: v for k, v in kw.items() if k in ("intensity", "ref_mode", "c_act_q16", "substeps",
                                                 "c_pos_q16", "c_neg_q16", "use_maps")}
    o = oracle_run(seq, mode, event_time=XT, **okw)
    assert_same_events(g["events"], o["events"], what)
    if kw.get("ref_mode", evsim.SIM_REF_ACCUM) == evsim.SIM_REF_ACCUM:
        assert np.array_equal(g["R"], o["R"]), f"{what}: reference differs"
    assert g["stats"].tile_height == 16
    return g, o


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_warped_texture(mode):
    seq = synth.warped_texture(frames=8, width=200, height=150)
    g, o = check(seq, mode, "warped texture")
    # the same events as with substep times, each no later than its substep
    s = gpu_run(seq, mode)
    assert np.array_equal(g["events"]["x"], s["events"]["x"])
    assert np.array_equal(g["events"]["yp"], s["events"]["yp"])
    assert np.all(g["events"]["t"] <= s["events"]["t"])
    assert np.any(g["events"]["t"] < s["events"]["t"])


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_warped_texture_640x480_head(mode):
    seq = synth.warped_texture(frames=6)
    check(seq, mode, "warped texture 640x480, 6 frames")


@pytest.mark.parametrize("intensity", [evsim.SIM_LOG, evsim.SIM_LINEAR])
@pytest.mark.parametrize("ref", [evsim.SIM_REF_ACCUM, evsim.SIM_REF_RESET])
@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_mode_matrix(intensity, ref, mode):
    seq = random_seq(45, 77, F=4, seed=100 + intensity * 4 + ref * 2 + mode)
    c = 700 if intensity == evsim.SIM_LINEAR else 9000
    if intensity == evsim.SIM_LINEAR and ref == evsim.SIM_REF_ACCUM:
        c = 3 * 65536
    check(seq, mode, "mode matrix", intensity=intensity, ref_mode=ref, c_pos_q16=c,
          c_neg_q16=c + 1, use_maps=False)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_threshold_maps_and_adaptive_substeps(mode):
    seq = synth.warped_texture(frames=5, width=130, height=70)
    check(seq, mode, "maps, adaptive N")


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (17, 65), (33, 130), (70, 9)])
@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_ragged_shapes(H, W, mode):
    seq = random_seq(H, W, F=4, seed=7 * H + W)
    check(seq, mode, f"{W}x{H}", use_maps=False, tile_height=8)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("amp", [15.5, 40.0])
def test_large_flow_beyond_the_shared_halo(mode, amp):
    seq = random_seq(60, 150, F=3, flow_amp=amp, seed=int(amp) + 1)
    check(seq, mode, f"flow amplitude {amp}", use_maps=False)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("N", [1, 4, 40])
def test_rows_of_multi_crossings(mode, N):
    """Many crossings of one pixel in one substep get increasing times inside
    the substep; N = 40 runs the substep loop past 32."""
    H, W, F = 24, 100, 4
    fr = np.full((F, H, W), 20, np.uint8)
    fr[1] = 240
    fr[2] = 240
    fr[2, 5, 7] = 100
    fr[3] = 240
    fr[3, 10:13, 30:36] = 15
    flows = np.zeros((F, H, W, 2), np.float32)
    t = np.arange(F, dtype=np.int64) * 10007
    seq = synth.Sequence("multi", fr, flows, t, N, 64, 0.2, 0.2)
    g, o = check(seq, mode, "multi-crossing rows", use_maps=False, substeps=N)
    if N == 1:
        ev = g["events"]
        first = ev[(ev["x"] == 0) & (ev["yp"] >> 1 == 0)]
        assert len(first) >= 12 and np.all(np.diff(first["t"][:12].astype(np.int64)) > 0)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("batch,device", [(3, True), (5, False)])
def test_batched_pushes(mode, batch, device):
    seq = synth.warped_texture(frames=9, width=150, height=90)
    g = gpu_run(seq, mode, batch=batch, device_inputs=device, event_time=XT)
    o = oracle_run(seq, mode, event_time=XT)
    assert_same_events(g["events"], o["events"], f"batches of {batch}")
    assert np.array_equal(g["R"], o["R"])


def test_sparse_tiles_without_active_pixels():
    """A sparse frame whose tiles are mostly inactive (only a small square
    changes) publishes empty segments for the inactive tiles."""
    F, H, W = 4, 70, 200
    fr = np.full((F, H, W), 90, np.uint8)
    for i in range(1, F):
        fr[i, 20:30, 100:110] = 90 + 40 * i
    flows = np.zeros((F, H, W, 2), np.float32)
    flows[:, 20:30, 100:110, 0] = 1.5
    t = np.arange(F, dtype=np.int64) * 30000
    seq = synth.Sequence("square", fr, flows, t, 0, 8, 0.2, 0.2)
    g, o = check(seq, evsim.SIM_SPARSE, "square", use_maps=False, substeps=0)
    assert len(o["events"]) > 100


def test_group_refuses_crossing_times():
    cfg, keep = evsim.make_config(64, 48, event_time=XT)
    lib = evsim.load()
    import ctypes
    gc = evsim.simb_config()
    assert lib.simb_config_default(ctypes.byref(gc)) == 0
    g = ctypes.c_void_p()
    assert lib.simb_create(ctypes.byref(gc), ctypes.byref(g)) == 0
    try:
        mid = ctypes.c_int32(-1)
        assert lib.simb_admit(g, ctypes.byref(cfg), ctypes.byref(mid)) == evsim.SIM_ERR_ARG
    finally:
        lib.simb_destroy(g)
