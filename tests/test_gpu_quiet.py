"""Streams with quiet stretches: frames that repeat the previous one with
zero flow emit nothing (every tile takes the quiet path and flags its rows
empty), and a batch in which no row of any frame is busy leaves the order
pass without a live segment.  Such batches must still commit (reference,
frame ring and cursor move on), so the frames after them match the oracle.
Compared bit-exact with the CPU oracle, one frame per push and in batches,
dense and sparse, 64x16 and 64x8 tiles."""
import numpy as np
import pytest

from .helpers import assert_same_events, gpu_run, oracle_run
from paper_2209_04634_gb300 import evsim, synth

pytestmark = pytest.mark.gpu


def quiet_stretch_sequence() -> synth.Sequence:
    """A moving texture, then five repeats of its last frame with zero flow,
    then the texture moving again."""
    base = synth.warped_texture(frames=9, width=200, height=72, seed=5)
    F = base.frames.shape[0]
    keep = [0, 1, 2, 3, 3, 3, 3, 3, 3, 4, 5, 6, 7, 8]
    frames = np.ascontiguousarray(base.frames[keep])
    flows = np.zeros((len(keep),) + base.flows.shape[1:], np.float32)
    for j in range(1, len(keep)):
        if keep[j] != keep[j - 1]:
            flows[j] = base.flows[keep[j]]
    t = np.arange(len(keep), dtype=np.int64) * 33333 + 1000
    assert keep[-1] == F - 1
    return synth.Sequence("quiet_stretch", frames, flows, t, base.substeps, base.max_substeps,
                          base.c_pos, base.c_neg, base.cpos_map, base.cneg_map)


@pytest.mark.parametrize("mode", [evsim.SIM_DENSE, evsim.SIM_SPARSE])
@pytest.mark.parametrize("batch", [1, 3, 0])
@pytest.mark.parametrize("tile_height", [16, 8])
def test_quiet_stretch(mode, batch, tile_height):
    seq = quiet_stretch_sequence()
    g = gpu_run(seq, mode, batch=batch, tile_height=tile_height)
    o = oracle_run(seq, mode)
    assert_same_events(g["events"], o["events"], f"batch {batch}, 64x{tile_height}")
    # the stretch is quiet: the repeated frames' intervals hold no event
    t = o["events"]["t"].astype(np.int64)
    assert not ((t > seq.t_us[3]) & (t <= seq.t_us[8])).any()
    assert (t > seq.t_us[8]).any()
