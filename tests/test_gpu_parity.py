"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: the same events in the same order, the same committed reference,
the same substep counts, on seeded synthetic inputs of the workloads' shapes,
at sizes that span several tiles with ragged tails, and at the full sizes the
benchmark runs (whole streams where the oracle finishes in seconds; the first
frames plus invariants that hold at any size otherwise)."""
import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import assert_same_events, gpu_run, oracle_run

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


def check_parity(seq, mode, what, **kw):
    g = gpu_run(seq, mode, **kw)
    okw = {k: v for k, v in kw.items() if k in ("intensity", "ref_mode", "c_act_q16", "substeps",
                                                 "c_pos_q16", "c_neg_q16", "use_maps")}
    o = oracle_run(seq, mode, **okw)
    assert_same_events(g["events"], o["events"], what)
    if g["R"] is not None and kw.get("ref_mode", evsim.SIM_REF_ACCUM) == evsim.SIM_REF_ACCUM:
        assert np.array_equal(g["R"], o["R"]), f"{what}: reference differs"
    if kw.get("pop_every", 1) == 1:
        F = seq.frames.shape[0]
        assert list(g["n_per_frame"][1:]) == list(o["n_per_frame"][1:F]), what
        assert list(g["ev_per_frame"][1:]) == list(o["ev_per_frame"][1:F]), what
        if mode == evsim.SIM_SPARSE:
            assert list(g["active_per_frame"][1:]) == list(o["active_per_frame"][1:F]), what
    return g, o


def random_seq(H, W, F=4, flow_amp=3.0, seed=0, rgb=False, substeps=5, max_substeps=8):
    rng = np.random.default_rng(seed)
    shape = (F, H, W, 3) if rgb else (F, H, W)
    base = rng.integers(0, 256, size=shape, dtype=np.uint8)
    # smooth half of the content so sub-threshold structure and interpolation matter
    sm = np.clip(np.cumsum(rng.integers(-12, 13, size=shape), axis=2) + 128, 0, 255).astype(np.uint8)
    frames = np.where(rng.random(shape) < 0.5, base, sm).astype(np.uint8)
    flows = rng.uniform(-flow_amp, flow_amp, size=(F, H, W, 2)).astype(np.float32)
    flows[0] = 0
    t = np.cumsum(rng.integers(1000, 40000, size=F)).astype(np.int64)
    return synth.Sequence("random", frames, flows, t, substeps, max_substeps, 0.2, 0.2)


# ---------------------------------------------------------------------------
# the workloads

def test_blob_translation_dense_full():
    seq = synth.blob_translation()  # 240x180, 20 frames, N = 8, C = 0.2
    check_parity(seq, evsim.SIM_DENSE, "blob translation dense")


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_warped_texture_small(mode):
    seq = synth.warped_texture(frames=8, width=200, height=150)
    check_parity(seq, mode, "warped texture small")


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_warped_texture_full_size(mode):
    seq = synth.warped_texture()  # 640x480, 100 frames, adaptive N <= 8, noisy thresholds
    check_parity(seq, mode, "warped texture 640x480x100", pop_every=1)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_moving_rectangles_small(mode):
    seq = synth.moving_rectangles(frames=10, width=320, height=180, side=(20, 60))
    check_parity(seq, mode, "moving rectangles small")


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_moving_rectangles_full_size_head(mode):
    seq = synth.moving_rectangles(frames=24)  # 1280x720 RGB, N = 10, C = 0.15
    check_parity(seq, mode, "moving rectangles 1280x720 (24 frames)")


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_moving_rectangles_full_length_invariants(mode):
    """All 300 frames at 1280x720: properties that hold at any size."""
    seq = synth.moving_rectangles()
    g = gpu_run(seq, mode, pop_every=25)
    ev = g["events"]
    t, x, y, p = oracle.unpack(ev)
    key = t * (1 << 32) + y * (1 << 16) + x
    assert np.all(np.diff(key) >= 0), "events out of (time, row, column) order"
    lut = oracle.lut(oracle.LOG).astype(np.int64)
    w = seq.frames.astype(np.int64)
    luma0 = (77 * w[0, ..., 0] + 150 * w[0, ..., 1] + 29 * w[0, ..., 2] + 128) >> 8
    lumaL = (77 * w[-1, ..., 0] + 150 * w[-1, ..., 1] + 29 * w[-1, ..., 2] + 128) >> 8
    C = oracle.q16(seq.c_pos)
    pos = np.zeros(luma0.shape, np.int64)
    neg = np.zeros(luma0.shape, np.int64)
    np.add.at(pos, (y[p > 0], x[p > 0]), 1)
    np.add.at(neg, (y[p < 0], x[p < 0]), 1)
    assert np.array_equal(g["R"].astype(np.int64), lut[luma0] + C * pos - C * neg)
    if mode == evsim.SIM_DENSE:
        D = lut[lumaL] - g["R"]
        assert np.all(D < C) and np.all(D > -C)
    assert g["stats"].frames_committed == seq.frames.shape[0]
    assert t.max() == seq.t_us[-1] - seq.t_us[0]


# ---------------------------------------------------------------------------
# modes and edge cases

@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("C", [2, 10, 20])
def test_paper_mode_linear_reset(mode, C):
    """Linear differences of consecutive interpolated frames, Table I settings
    (C = 2 / 10 / 20 in 8-bit units, 10 interpolated frames)."""
    seq = synth.warped_texture(frames=6, width=150, height=100)
    check_parity(seq, mode, f"paper mode C={C}", intensity=evsim.SIM_LINEAR,
                 ref_mode=evsim.SIM_REF_RESET, substeps=10, c_pos_q16=C * 65536,
                 c_neg_q16=C * 65536, use_maps=False)


@pytest.mark.parametrize("intensity", [evsim.SIM_LOG, evsim.SIM_LINEAR])
@pytest.mark.parametrize("ref", [evsim.SIM_REF_ACCUM, evsim.SIM_REF_RESET])
@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_mode_matrix(intensity, ref, mode):
    seq = random_seq(45, 77, F=4, seed=intensity * 4 + ref * 2 + mode)
    c = 700 if intensity == evsim.SIM_LINEAR else 9000
    if intensity == evsim.SIM_LINEAR and ref == evsim.SIM_REF_ACCUM:
        c = 3 * 65536
    check_parity(seq, mode, "mode matrix", intensity=intensity, ref_mode=ref, c_pos_q16=c,
                 c_neg_q16=c + 1, use_maps=False)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (17, 65), (15, 63), (16, 64),
                                 (33, 130), (3, 200), (70, 9), (9, 70), (8, 64)])
@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("th", [16, 8])
def test_ragged_shapes(H, W, mode, th):
    seq = random_seq(H, W, F=4, seed=H * 1000 + W)
    check_parity(seq, mode, f"{W}x{H} tiles 64x{th}", use_maps=False, tile_height=th)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("amp", [15.5, 40.0])
@pytest.mark.parametrize("th", [16, 8])
def test_large_flow_beyond_the_shared_halo(mode, amp, th):
    """Flows beyond the shared-memory halo take the global-memory taps."""
    seq = random_seq(60, 150, F=3, flow_amp=amp, seed=int(amp))
    check_parity(seq, mode, f"flow amplitude {amp}", use_maps=False, tile_height=th)


def test_mixed_tiles_small_and_large_flow():
    seq = random_seq(64, 192, F=3, flow_amp=2.0, seed=77)
    seq.flows[:, :, 128:, :] *= 12.0  # right third of the frame moves far
    check_parity(seq, evsim.SIM_DENSE, "mixed tiles", use_maps=False)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("batch", [0, 3])
@pytest.mark.parametrize("th", [16, 8])
def test_rows_of_multi_crossings(mode, batch, th):
    """Pixels that cross several thresholds in one substep: whole rows of
    them (rows of 16 or more events, which dense tiles publish as per-pixel
    counts) and a single such pixel in a row (its events are staged), both in
    the oracle's order (substep, row, column, repeats adjacent)."""
    H, W, F = 40, 150, 4
    fr = np.full((F, H, W), 20, np.uint8)
    fr[1] = 240                          # ~12 thresholds per pixel in one substep
    fr[2] = 240
    fr[2, 5, 7] = 100                    # one pixel: 4 thresholds down
    fr[3] = 240
    fr[3, 30:33, 64:70] = 15             # a small block: rows of 36 events
    flows = np.zeros((F, H, W, 2), np.float32)
    t = np.arange(F, dtype=np.int64) * 10000
    seq = synth.Sequence("multi", fr, flows, t, 1, 8, 0.2, 0.2)
    if batch:
        g = gpu_run(seq, mode, use_maps=False, substeps=1, batch=batch, tile_height=th)
        o = oracle_run(seq, mode, use_maps=False, substeps=1)
        assert_same_events(g["events"], o["events"], "multi-crossing rows (batched)")
        assert np.array_equal(g["R"], o["R"])
    else:
        g, o = check_parity(seq, mode, "multi-crossing rows", use_maps=False, substeps=1,
                            tile_height=th)
    assert o["ev_per_frame"][1] >= 12 * H * W


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_nan_and_clamped_flow(mode):
    seq = random_seq(40, 70, F=3, seed=5)
    seq.flows[1, 3, 4] = (np.nan, 2.0)
    seq.flows[1, 10, 11] = (5000.0, -1e9)
    seq.flows[2, 20, 30] = (np.inf, -np.inf)
    seq.flows[2, 0, 0] = (-1024.0, 1024.0)
    g, o = check_parity(seq, mode, "nan/clamp", use_maps=False, substeps=4)
    if mode == evsim.SIM_DENSE:
        assert g["stats"].flow_clamped == o["clamped"] == 4


def test_adaptive_substeps_track_the_flow():
    seq = random_seq(30, 40, F=6, flow_amp=0.0, seed=9, substeps=0, max_substeps=12)
    for i, m in enumerate([0, 0.3, 2.0, 5.5, 11.2, 30.0]):
        seq.flows[i, 7, 9] = (m, -m / 2)
    g, o = check_parity(seq, evsim.SIM_DENSE, "adaptive N", use_maps=False)
    assert list(g["n_per_frame"][1:]) == [1, 3, 7, 12, 12]


def test_threshold_maps():
    seq = synth.warped_texture(frames=5, width=96, height=80, c_sigma=0.05)
    check_parity(seq, evsim.SIM_DENSE, "maps")
    check_parity(seq, evsim.SIM_SPARSE, "maps sparse")


def test_sparse_with_zero_activity_threshold_equals_dense():
    seq = synth.warped_texture(frames=5, width=130, height=70)
    d = gpu_run(seq, evsim.SIM_DENSE)
    s = gpu_run(seq, evsim.SIM_SPARSE, c_act_q16=0)
    assert_same_events(s["events"], d["events"], "sparse(C_act=0) vs dense")
    assert np.array_equal(s["R"], d["R"])


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_host_inputs_equal_device_inputs(mode):
    seq = synth.moving_rectangles(frames=5, width=200, height=120, side=(20, 50))
    a = gpu_run(seq, mode, device_inputs=False)
    b = gpu_run(seq, mode, device_inputs=True)
    assert_same_events(a["events"], b["events"], "host vs device inputs")


def test_pitched_frames():
    seq = random_seq(33, 50, F=3, seed=3)
    o = oracle_run(seq, evsim.SIM_DENSE, use_maps=False)
    pitch = 64
    padded = np.zeros((3, 33, pitch), np.uint8)
    padded[:, :, :50] = seq.frames
    padded[:, :, 50:] = 255  # garbage past the row must be ignored
    sim = evsim.simulator_for(seq, evsim.SIM_DENSE, c_pos_map=None, c_neg_map=None)
    for i in range(3):
        sim.push(padded[i], seq.flows[i] if i else None, int(seq.t_us[i]), pitch=pitch)
    assert_same_events(sim.pop(), o["events"], "pitched host frames")
    sim.close()


def test_pop_in_pieces():
    seq = synth.blob_translation(frames=4)
    o = oracle_run(seq)
    sim = evsim.simulator_for(seq)
    for i in range(4):
        sim.push(seq.frames[i], seq.flows[i] if i else None, int(seq.t_us[i]))
    parts = []
    while True:
        out = np.empty(1000, dtype=evsim.EVENT_DTYPE)
        n, rc = sim.pop_into(out, 1000)
        parts.append(out[:n])
        if rc != evsim.SIM_MORE:
            break
    assert len(parts) > 3
    assert_same_events(np.concatenate(parts), o["events"], "pieces")
    assert sim.stats().events_pending == 0
    sim.close()


def test_event_overflow_is_transactional():
    """A frame whose events do not fit is not committed; the error surfaces at
    the next pop; re-pushing after popping reproduces the oracle exactly."""
    seq = synth.blob_translation(frames=6)
    o = oracle_run(seq)
    per = o["ev_per_frame"]
    cap = int(per[1] + per[2] + per[3] // 2)  # frame 3 cannot fit after frames 1, 2
    sim = evsim.simulator_for(seq, event_capacity=cap)
    for i in range(5):
        sim.push(seq.frames[i], seq.flows[i] if i else None, int(seq.t_us[i]))
    with pytest.raises(evsim.SimError) as ei:
        sim.sync()
    assert ei.value.code == evsim.SIM_ERR_EVENT_OVERFLOW
    st = sim.stats()
    assert st.frames_committed == 3  # frames 0, 1, 2
    got = [sim.pop()]  # the committed events are still there
    assert len(got[0]) == per[1] + per[2]
    for i in range(3, 6):
        sim.push(seq.frames[i], seq.flows[i], int(seq.t_us[i]))
        got.append(sim.pop())
    assert_same_events(np.concatenate(got), o["events"], "after overflow")
    assert np.array_equal(sim.reference(), o["R"])
    sim.close()


def test_timestamp_errors():
    seq = synth.blob_translation(frames=3)
    sim = evsim.simulator_for(seq)
    sim.push(seq.frames[0], None, 100)
    with pytest.raises(evsim.SimError) as e1:
        sim.push(seq.frames[1], seq.flows[1], 100)
    assert e1.value.code == evsim.SIM_ERR_TIME
    with pytest.raises(evsim.SimError) as e2:
        sim.push(seq.frames[1], seq.flows[1], 100 + (1 << 32))
    assert e2.value.code == evsim.SIM_ERR_TIME_RANGE
    with pytest.raises(evsim.SimError):
        sim.push(seq.frames[1], None, 200)
    sim.push(seq.frames[1], seq.flows[1], 200)
    assert sim.stats().frames_committed == 2
    sim.close()


def test_two_handles_on_two_streams_are_independent():
    a_seq = synth.warped_texture(frames=5, width=120, height=90, seed=11)
    b_seq = synth.moving_rectangles(frames=5, width=160, height=90, side=(20, 40), seed=12)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = evsim.simulator_for(a_seq, evsim.SIM_SPARSE, stream=s1)
    b = evsim.simulator_for(b_seq, evsim.SIM_DENSE, stream=s2)
    ea, eb = [], []
    for i in range(5):
        a.push(a_seq.frames[i], a_seq.flows[i] if i else None, int(a_seq.t_us[i]))
        b.push(b_seq.frames[i], b_seq.flows[i] if i else None, int(b_seq.t_us[i]))
    ea.append(a.pop())
    eb.append(b.pop())
    assert_same_events(np.concatenate(ea), oracle_run(a_seq, evsim.SIM_SPARSE)["events"], "stream a")
    assert_same_events(np.concatenate(eb), oracle_run(b_seq, evsim.SIM_DENSE)["events"], "stream b")
    a.close()
    b.close()


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("batch,device", [(7, True), (1, True), (5, False), (40, True)])
def test_batched_pushes(mode, batch, device):
    """sim_push_frames (device batches carried through by persistent blocks,
    staged host batches) gives the same stream as the oracle."""
    seq = synth.warped_texture(frames=23, width=160, height=120, seed=21)
    g = gpu_run(seq, mode, batch=batch, device_inputs=device)
    o = oracle_run(seq, mode)
    assert_same_events(g["events"], o["events"], f"batch {batch}")
    assert np.array_equal(g["R"], o["R"])


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_batches_split_at_the_device_batch_cap(mode):
    """A push of 9 frames on a handle whose device batch holds 4 frames runs
    as batches of 4, 4, 1 (+ the first frame) and still equals the oracle."""
    seq = synth.moving_rectangles(frames=10, width=256, height=144, side=(20, 60), seed=8)
    g = gpu_run(seq, mode, batch=10, max_batch=4)
    assert g["stats"].max_batch == 4
    assert_same_events(g["events"], oracle_run(seq, mode)["events"], "split batches")


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_batch_overflow_commits_nothing_of_the_batch(mode):
    seq = synth.blob_translation(frames=7)
    o = oracle_run(seq, mode)
    per = o["ev_per_frame"]
    cap = int(per[1:4].sum() + per[4:6].sum() // 2)  # frames 1-3 fit, 1-6 do not
    sim = evsim.simulator_for(seq, mode, event_capacity=cap)
    sim.push_many(seq.frames[:4], seq.flows[:4], seq.t_us[:4])
    sim.push_many(seq.frames[4:7], seq.flows[4:7], seq.t_us[4:7])
    with pytest.raises(evsim.SimError) as ei:
        sim.sync()
    assert ei.value.code == evsim.SIM_ERR_EVENT_OVERFLOW
    assert sim.stats().frames_committed == 4
    got = [sim.pop()]
    sim.push_many(seq.frames[4:7], seq.flows[4:7], seq.t_us[4:7])
    got.append(sim.pop())
    assert_same_events(np.concatenate(got), o["events"], "after a failed batch")
    assert np.array_equal(sim.reference(), o["R"])
    sim.close()


def test_batch_rejects_bad_timestamps_before_enqueueing():
    seq = synth.blob_translation(frames=5)
    sim = evsim.simulator_for(seq)
    t = seq.t_us.copy()
    t[3] = t[2]
    with pytest.raises(evsim.SimError) as e:
        sim.push_many(seq.frames, seq.flows, t)
    assert e.value.code == evsim.SIM_ERR_TIME
    assert sim.stats().frames_pushed == 0
    sim.push_many(seq.frames, seq.flows, seq.t_us)
    assert_same_events(sim.pop(), oracle_run(seq)["events"], "after rejected batch")
    sim.close()


def test_overflow_reported_by_pop_keeps_committed_events():
    seq = synth.blob_translation(frames=5)
    o = oracle_run(seq)
    per = o["ev_per_frame"]
    cap = int(per[1] + per[2] // 2)
    sim = evsim.simulator_for(seq, event_capacity=cap)
    for i in range(4):
        sim.push(seq.frames[i], seq.flows[i] if i else None, int(seq.t_us[i]))
    out = np.empty(cap, dtype=evsim.EVENT_DTYPE)
    n = evsim.ctypes.c_int64(-1)
    rc = sim._lib.sim_pop_events(sim.h, out.ctypes.data, cap, evsim.ctypes.byref(n), evsim.SIM_HOST)
    assert rc == evsim.SIM_ERR_EVENT_OVERFLOW and n.value == 0
    first = sim.pop()
    assert len(first) == per[1]
    assert_same_events(first, o["events"][:per[1]], "committed before the overflow")
    sim.close()


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_tile_shapes_agree_on_the_workloads(mode):
    """Both tile shapes of the batch kernel give the oracle's events on heads of
    the 640x480 and 1280x720 workloads, pushed as one batch."""
    for seq in (synth.warped_texture(frames=6), synth.moving_rectangles(frames=4)):
        o = oracle_run(seq, mode)
        for th in (16, 8):
            g = gpu_run(seq, mode, batch=seq.frames.shape[0], tile_height=th)
            assert g["stats"].tile_height == th
            assert_same_events(g["events"], o["events"], f"{seq.name} tiles 64x{th}")
            assert np.array_equal(g["R"], o["R"])


def test_autotune_chooses_a_shape_that_sim_create_uses():
    th, us16, us8, us_rows = evsim.autotune(240, 180, frames=6, substeps=0, max_substeps=8)
    assert th in (8, 16, evsim.SIM_TILE_ROWS) and us16 > 0 and us8 > 0 and us_rows > 0
    sim = evsim.Simulator(240, 180, substeps=0, max_substeps=8)  # SIM_TILE_AUTO
    assert sim.stats().tile_height == th
    sim.close()
    sim = evsim.Simulator(240, 180, substeps=0, max_substeps=8, tile_height=16)
    assert sim.stats().tile_height == 16
    sim.close()
    # a configuration the table does not hold: tuned at create (SIM_TILE_TUNE)
    sim = evsim.Simulator(200, 100, substeps=3, tile_height=evsim.SIM_TILE_TUNE)
    assert sim.stats().tile_height in (8, 16, evsim.SIM_TILE_ROWS)
    sim.close()


@pytest.mark.parametrize("device", [True, False])
def test_autotune_on_a_sample_of_the_stream(device):
    seq = synth.warped_texture(frames=6, width=200, height=96)
    fr, fl = seq.frames, seq.flows
    if device:
        fr, fl = torch.from_numpy(fr).cuda(), torch.from_numpy(fl).cuda()
    opts = evsim.seq_options(seq, mode=evsim.SIM_SPARSE)
    th, us16, us8, us_rows = evsim.autotune_sample(seq.width, seq.height, fr, fl, seq.t_us,
                                                   **opts)
    assert th in (8, 16, evsim.SIM_TILE_ROWS) and us16 > 0 and us8 > 0 and us_rows > 0
    sim = evsim.simulator_for(seq, evsim.SIM_SPARSE)  # SIM_TILE_AUTO: the table's entry
    assert sim.stats().tile_height == th
    sim.close()
    # the sample's own events are unaffected: a stream run afterwards matches the oracle
    g = gpu_run(seq, evsim.SIM_SPARSE)
    assert_same_events(g["events"], oracle_run(seq, evsim.SIM_SPARSE)["events"], "after tuning")


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_block_orders_give_the_oracle_events(order, mode, tmp_path):
    """The serpentine and the balanced block orders (set through an autotuner
    table) only reschedule the tiles: the events stay the oracle's, over
    several batches (the balanced order plans each batch from samples of its
    own flows)."""
    seq = random_seq(90, 200, F=7, seed=31 + order, substeps=3)
    f = tmp_path / "table.txt"
    f.write_text(f"200 90 1 {mode} 3 0 0 0 0 16 {order} 1.0 1.0 0.0\n")
    evsim.autotune_load(str(f))
    g = gpu_run(seq, mode, use_maps=False, batch=2)
    assert g["stats"].block_order == order and g["stats"].tile_height == 16
    o = oracle_run(seq, mode, use_maps=False)
    assert_same_events(g["events"], o["events"], f"block order {order}")
    assert np.array_equal(g["R"], o["R"])


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
def test_pinned_host_inputs_read_in_place_equal_the_oracle(mode):
    """Host frames and flows in pinned memory are read by the kernels through
    their device mapping (SIM_HOST_MAPPED) or staged (SIM_HOST_STAGE): both
    give the oracle's events; pageable arrays are staged either way."""
    seq = synth.warped_texture(frames=12, width=200, height=120)
    fr = torch.from_numpy(seq.frames).pin_memory()
    fl = torch.from_numpy(seq.flows).pin_memory()
    o = oracle_run(seq, mode)
    for how in (evsim.SIM_HOST_MAPPED, evsim.SIM_HOST_STAGE):
        for frames, flows in ((fr.numpy(), fl.numpy()), (seq.frames, seq.flows)):
            sim = evsim.simulator_for(seq, mode, host_inputs=how)
            sim.push(frames[0], None, int(seq.t_us[0]))
            sim.push_many(frames[1:], flows[1:], seq.t_us[1:])
            assert_same_events(sim.pop(), o["events"], f"host inputs {how}")
            assert np.array_equal(sim.reference(), o["R"])
            sim.close()
