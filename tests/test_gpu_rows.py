"""Parity of the row kernel (sim_config.tile_height = SIM_TILE_ROWS) with the
CPU oracle: bit-exact events, references and per-frame counts, dense and
sparse, on the three workloads, every mode combination, ragged shapes, far
and invalid flows, multi-crossing rows, N above 32, threshold maps, batches,
overflow; and the exact skip of quiet pixels (zero flow, both end values
inside the threshold band) at its bound and one unit either side and in
quiet, moving and mixed rows, for the row kernel and both tile shapes (the
dense tile kernel skips rows whose pixels are all quiet)."""
import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import assert_same_events, gpu_run, oracle_run
from .test_gpu_parity import check_parity, random_seq

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROWS = evsim.SIM_TILE_ROWS
MODES = [evsim.SIM_DENSE, evsim.SIM_SPARSE]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


def rows_parity(seq, mode, what, th=ROWS, **kw):
    g, o = check_parity(seq, mode, what + f" (tile height {th})", tile_height=th, **kw)
    assert g["stats"].tile_height == th
    return g, o


@pytest.mark.parametrize("mode", MODES)
def test_blob_translation_full(mode):
    rows_parity(synth.blob_translation(), mode, "blob translation")


@pytest.mark.parametrize("mode", MODES)
def test_warped_texture_full_size(mode):
    rows_parity(synth.warped_texture(), mode, "warped texture 640x480x100", pop_every=10)


@pytest.mark.parametrize("mode", MODES)
def test_moving_rectangles_full_size_head(mode):
    rows_parity(synth.moving_rectangles(frames=16), mode, "moving rectangles 1280x720 head")


@pytest.mark.parametrize("mode", MODES)
def test_moving_rectangles_small(mode):
    seq = synth.moving_rectangles(frames=40, width=320, height=180, side=(24, 70))
    rows_parity(seq, mode, "moving rectangles 320x180")


@pytest.mark.parametrize("intensity", [evsim.SIM_LOG, evsim.SIM_LINEAR])
@pytest.mark.parametrize("ref", [evsim.SIM_REF_ACCUM, evsim.SIM_REF_RESET])
@pytest.mark.parametrize("mode", MODES)
def test_mode_matrix(intensity, ref, mode):
    seq = synth.warped_texture(frames=8, width=200, height=150)
    c = (3 << 16) if intensity == evsim.SIM_LINEAR else None
    rows_parity(seq, mode, "mode matrix", intensity=intensity, ref_mode=ref, use_maps=False,
                c_pos_q16=c, c_neg_q16=c)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (17, 65), (15, 63), (16, 64),
                                 (3, 130), (70, 200)])
@pytest.mark.parametrize("mode", MODES)
def test_ragged_shapes(H, W, mode):
    seq = random_seq(H, W, F=5, seed=H * 1000 + W)
    rows_parity(seq, mode, f"{W}x{H}", use_maps=False)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("amp", [15.5, 40.0])
def test_far_flows(mode, amp):
    seq = random_seq(48, 150, F=4, flow_amp=amp, seed=int(amp), substeps=6)
    rows_parity(seq, mode, f"flow amplitude {amp}", use_maps=False)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("batch", [0, 3])
def test_rows_of_multi_crossings(mode, batch):
    # one substep and large steps: many pixels cross several thresholds
    seq = random_seq(40, 130, F=5, seed=7, substeps=1)
    g = gpu_run(seq, mode, use_maps=False, substeps=1, batch=batch, tile_height=ROWS,
                c_pos_q16=20000, c_neg_q16=15000)
    o = oracle_run(seq, mode, use_maps=False, substeps=1, c_pos_q16=20000, c_neg_q16=15000)
    assert_same_events(g["events"], o["events"], "multi-crossing rows")
    assert np.array_equal(g["R"], o["R"])


@pytest.mark.parametrize("mode", MODES)
def test_more_than_32_substeps(mode):
    seq = random_seq(33, 100, F=4, seed=11, substeps=40, max_substeps=40)
    rows_parity(seq, mode, "N = 40", use_maps=False, substeps=40)


@pytest.mark.parametrize("mode", MODES)
def test_adaptive_substeps_and_maps(mode):
    seq = synth.warped_texture(frames=12, width=256, height=96)
    rows_parity(seq, mode, "adaptive N with threshold maps")


@pytest.mark.parametrize("mode", MODES)
def test_nan_and_clamped_flow(mode):
    seq = random_seq(20, 70, F=3, seed=5)
    seq.flows[1, 3, 4] = (np.nan, 2.0)
    seq.flows[1, 7, 9] = (5000.0, -3.0)
    seq.flows[2, 0, 0] = (-1e9, np.inf)
    seq.flows[2, 19, 69] = (np.nan, np.nan)
    rows_parity(seq, mode, "NaN / clamped flow", use_maps=False, substeps=4)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("batch,device", [(7, True), (1, True), (5, False), (40, True)])
def test_batched_pushes(mode, batch, device):
    seq = synth.warped_texture(frames=41, width=160, height=120)
    g = gpu_run(seq, mode, batch=batch, device_inputs=device, tile_height=ROWS)
    o = oracle_run(seq, mode)
    assert_same_events(g["events"], o["events"], f"batches of {batch}")
    assert np.array_equal(g["R"], o["R"])


@pytest.mark.parametrize("mode", MODES)
def test_batches_split_at_the_device_batch_cap(mode):
    seq = synth.warped_texture(frames=23, width=130, height=70)
    g = gpu_run(seq, mode, batch=22, max_batch=4, tile_height=ROWS)
    o = oracle_run(seq, mode)
    assert_same_events(g["events"], o["events"], "batch cap 4")
    assert np.array_equal(g["R"], o["R"])


@pytest.mark.parametrize("mode", MODES)
def test_batch_overflow_commits_nothing(mode):
    seq = synth.warped_texture(frames=6, width=128, height=64)
    o = oracle_run(seq, mode)
    sim = evsim.simulator_for(seq, mode, tile_height=ROWS, event_capacity=len(o["events"]) // 2)
    frames = torch.from_numpy(seq.frames).cuda()
    flows = torch.from_numpy(seq.flows).cuda()
    sim.push(frames[0], None, int(seq.t_us[0]))
    R0 = sim.reference()
    sim.push_many(frames[1:], flows[1:], seq.t_us[1:])
    with pytest.raises(evsim.SimError) as ei:
        sim.pop()
    assert ei.value.code == evsim.SIM_ERR_EVENT_OVERFLOW
    assert sim.stats().frames_committed == 1
    assert np.array_equal(sim.reference(), R0)
    sim.close()


def _plateau(v0, v1, H=8, W=70, F=3):
    """Frames: uniform v0, then v1 on the left half and v0 on the right, then
    back; zero flow everywhere except one moving pixel in row 5."""
    fr = np.full((F, H, W), v0, np.uint8)
    fr[1, :, : W // 2] = v1
    flows = np.zeros((F, H, W, 2), np.float32)
    flows[1:, 5, 40] = (2.5, -1.0)
    fr[1, 5, 40] = 200
    t = np.arange(F, dtype=np.int64) * 10_000
    return synth.Sequence("plateau", fr, flows, t, 6, 8, 0.2, 0.2)


@pytest.mark.parametrize("th", [ROWS, 16, 8])
@pytest.mark.parametrize("intensity", [evsim.SIM_LOG, evsim.SIM_LINEAR])
@pytest.mark.parametrize("ref", [evsim.SIM_REF_ACCUM, evsim.SIM_REF_RESET])
@pytest.mark.parametrize("delta", [-1, 0, 1])
@pytest.mark.parametrize("mode", MODES)
def test_quiet_pixel_skip_at_its_bound(intensity, ref, delta, mode, th):
    # zero-flow pixels whose change is the threshold, one unit below or one
    # unit above: the skip must decide exactly as the simulation would
    lut = oracle.lut(oracle.LINEAR if intensity == evsim.SIM_LINEAR else oracle.LOG)
    v0, v1 = 100, 117
    D = int(lut[v1]) - int(lut[v0])
    big = 1 << 29  # beyond any change of the 8-bit range
    for rising in (True, False):
        s = _plateau(v0, v1) if rising else _plateau(v1, v0)
        cp, cn = (D + delta, big) if rising else (big, D + delta)
        # activity threshold 0: every pixel is active, so the skip decides alone
        rows_parity(s, mode, f"skip bound {delta:+d} ({'rising' if rising else 'falling'})",
                    th=th, intensity=intensity, ref_mode=ref, use_maps=False, c_pos_q16=cp,
                    c_neg_q16=cn, c_act_q16=0)


@pytest.mark.parametrize("th", [ROWS, 16, 8])
@pytest.mark.parametrize("mode", MODES)
def test_quiet_moving_and_mixed_rows(mode, th):
    # static rows (skipped), rows with one moving pixel, rows half static
    rng = np.random.default_rng(3)
    H, W, F = 24, 200, 6
    fr = np.repeat(rng.integers(40, 220, size=(1, H, W), dtype=np.uint8), F, axis=0)
    flows = np.zeros((F, H, W, 2), np.float32)
    for i in range(1, F):
        fr[i, 8:12] = np.roll(fr[i - 1, 8:12], 3, axis=1)     # moving rows
        flows[i, 8:12] = (3.0, 0.0)
        fr[i, 16, 100:] = np.roll(fr[i - 1, 16, 100:], 2)    # half a row moving
        flows[i, 16, 100:] = (2.0, 0.0)
        fr[i, 20, 7] = (int(fr[i - 1, 20, 7]) + 60) % 256     # one pixel changing in place
    t = np.arange(F, dtype=np.int64) * 16_667
    seq = synth.Sequence("mixed", fr, flows, t, 10, 10, 0.15, 0.15)
    g, _ = rows_parity(seq, mode, "quiet, moving and mixed rows", th=th, use_maps=False)
    # a second batch after a batch of quiet frames (the kept halo is rebuilt)
    g2 = gpu_run(seq, mode, use_maps=False, batch=3, tile_height=th)
    assert_same_events(g2["events"], g["events"], "quiet rows across batches")
    assert len(g["events"]) > 0


def test_tile_and_row_kernels_agree_on_the_workload_heads():
    for seq in (synth.moving_rectangles(frames=8), synth.warped_texture(frames=10)):
        for mode in MODES:
            a = gpu_run(seq, mode, batch=seq.frames.shape[0], tile_height=16)
            b = gpu_run(seq, mode, batch=seq.frames.shape[0], tile_height=ROWS)
            assert_same_events(b["events"], a["events"], "row vs tile kernel")
            assert np.array_equal(a["R"], b["R"])
