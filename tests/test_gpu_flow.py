"""Parity of the device Lucas-Kanade flow (sim_flow_*) with the CPU oracle
(orc_flow_lk): the same float flow, bit for bit, on the workloads' frames,
ragged sizes, RGB frames, every parameter range, untrackable content and
flows that feed the simulator (whose events then equal the oracle's
simulator fed the oracle's flow)."""
import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import assert_same_events

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


def gpu_flow(f0, f1, **kw):
    H, W = f0.shape[:2]
    ch = 3 if f0.ndim == 3 else 1
    fl = evsim.Flow(W, H, pixel_format=ch, **kw)
    a = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(f1)).cuda()
    out = torch.full((H, W, 2), float("nan"), dtype=torch.float32, device="cuda")
    fl.compute(a, b, out)
    torch.cuda.synchronize()
    fl.close()
    return out.cpu().numpy()


def want_flow(f0, f1, **kw):
    q = oracle.flow_lk(f0, f1, **kw)
    return q.astype(np.float32) / np.float32(65536.0)


def check(f0, f1, what, **kw):
    g = gpu_flow(f0, f1, **kw)
    w = want_flow(f0, f1, **kw)
    bad = np.argwhere(g.view(np.uint32) != w.view(np.uint32))
    assert bad.size == 0, f"{what}: {len(bad)} flow components differ, first {bad[:3].tolist()}"
    return g


def test_warped_texture_pairs():
    s = synth.warped_texture(frames=6)
    for i in range(1, 6):
        g = check(s.frames[i - 1], s.frames[i], f"warped texture pair {i}")
    assert np.abs(g).max() > 1.0


def test_moving_rectangles_rgb_full_size():
    s = synth.moving_rectangles(frames=3)
    check(s.frames[1], s.frames[2], "moving rectangles 1280x720 RGB")


def test_blob_translation():
    s = synth.blob_translation(frames=3)
    check(s.frames[0], s.frames[1], "blob translation", levels=2, radius=2, iterations=4)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 37), (37, 1), (17, 65), (8, 32), (9, 33),
                                 (100, 3), (70, 200)])
def test_ragged_sizes(H, W):
    rng = np.random.default_rng(H * 1000 + W)
    f0 = rng.integers(0, 256, (H, W), dtype=np.uint8)
    f1 = np.roll(f0, 1, axis=1)
    check(f0, f1, f"{W}x{H}", min_eig=1.0)


@pytest.mark.parametrize("levels", [1, 2, 4, 6])
@pytest.mark.parametrize("radius", [1, 3, 7])
@pytest.mark.parametrize("iterations", [1, 5])
def test_parameter_ranges(levels, radius, iterations):
    s = synth.warped_texture(frames=2, width=150, height=110, max_flow=6.0)
    check(s.frames[0], s.frames[1], f"L={levels} r={radius} K={iterations}", levels=levels,
          radius=radius, iterations=iterations)


def test_untrackable_content_and_thresholds():
    f = np.full((40, 64), 77, np.uint8)
    g = check(f, f.copy(), "uniform")
    assert not g.any()
    s = synth.warped_texture(frames=2, width=96, height=64)
    for me in (0.0, 1.0, 1e4, 1e12):
        check(s.frames[0], s.frames[1], f"min_eig {me}", min_eig=me)


def test_flow_feeds_the_simulator():
    """Frames -> device flow -> simulator: the events equal the oracle's
    simulator run on the oracle's flow."""
    s = synth.warped_texture(frames=8, width=200, height=120)
    H, W = s.height, s.width
    frames = torch.from_numpy(s.frames).cuda()
    flows = torch.zeros((len(s.t_us), H, W, 2), dtype=torch.float32, device="cuda")
    fl = evsim.Flow(W, H)
    for i in range(1, len(s.t_us)):
        fl.compute(frames[i - 1], frames[i], flows[i])
    torch.cuda.synchronize()
    fl.close()
    want_fl = np.zeros_like(s.flows)
    for i in range(1, len(s.t_us)):
        want_fl[i] = want_flow(s.frames[i - 1], s.frames[i])
    assert np.array_equal(flows.cpu().numpy().view(np.uint32), want_fl.view(np.uint32))
    for mode, omode in ((evsim.SIM_DENSE, oracle.DENSE), (evsim.SIM_SPARSE, oracle.SPARSE)):
        sim = evsim.simulator_for(s, mode, c_pos_map=None, c_neg_map=None)
        sim.push_many(frames, flows, s.t_us)
        got = sim.pop()
        R = sim.reference()
        sim.close()
        o = oracle.run(s.frames, want_fl, s.t_us, mode=omode, substeps=s.substeps,
                       max_substeps=s.max_substeps, c_pos_q16=oracle.q16(s.c_pos),
                       c_neg_q16=oracle.q16(s.c_neg))
        assert len(got) > 0
        assert_same_events(got, o["events"], "simulator on the device flow")
        assert np.array_equal(R, o["R"])
