"""Accumulated event frames on the GPU (sim_accumulate) equal the oracle's
(orc_accumulate) for every frame window of a simulated stream."""
import numpy as np
import pytest

import oracle
from paper_2209_04634_gb300 import build, evsim, synth

from .helpers import oracle_run

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    evsim.load()


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE, evsim.SIM_DIFF])
def test_accumulated_frames_per_frame_window(mode):
    seq = synth.warped_texture(frames=6, width=150, height=90)
    H, W = seq.height, seq.width
    sim = evsim.simulator_for(seq, mode)
    sim.push_many(torch.from_numpy(seq.frames).cuda(), torch.from_numpy(seq.flows).cuda(),
                  seq.t_us)
    cap = 1 << 22
    buf = torch.empty(cap * 8, dtype=torch.uint8, device="cuda")
    n, rc = sim.pop_into(buf, cap)
    assert rc == evsim.SIM_OK and n > 0
    sim.close()
    want_ev = oracle_run(seq, mode)["events"]
    assert len(want_ev) == n
    t = seq.t_us - seq.t_us[0]
    frame = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    total = np.zeros((H, W), np.int32)
    for i in range(1, len(t)):
        frame.zero_()
        evsim.accumulate(buf, n, W, H, int(t[i - 1]) + 1, int(t[i]) + 1, frame)
        want = oracle.accumulate(want_ev, W, H, int(t[i - 1]) + 1, int(t[i]) + 1)
        assert np.array_equal(frame.cpu().numpy(), want), i
        total += want
    frame.zero_()
    evsim.accumulate(buf, n, W, H, 0, 1 << 40, frame)
    assert np.array_equal(frame.cpu().numpy(), total)


def test_accumulate_skips_events_outside_the_frame_and_window():
    ev = np.zeros(4, dtype=oracle.EVENT_DTYPE)
    ev["t"] = [5, 5, 6, 99]
    ev["x"] = [1, 40, 2, 1]
    ev["yp"] = [(2 << 1) | 1, (0 << 1) | 1, (50 << 1) | 0, (2 << 1) | 0]
    d = torch.from_numpy(ev.view(np.uint8).copy()).cuda()
    frame = torch.zeros((8, 16), dtype=torch.int32, device="cuda")
    evsim.accumulate(d, 4, 16, 8, 0, 99, frame)
    want = oracle.accumulate(ev, 16, 8, 0, 99)
    assert np.array_equal(frame.cpu().numpy(), want)
    assert want.sum() == 1
