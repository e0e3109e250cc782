"""Checkpoint and restore of a stream (sim_get_state / sim_set_state): a
stream saved after some frames and restored into a fresh handle of the same
configuration continues bit-exactly - the events of the two halves are the
CPU oracle's events of the whole sequence (and those of the uninterrupted
GPU run), and the reference ends equal to the oracle's."""
import numpy as np
import pytest

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


def _options(seq, mode, ref, maps):
    kw = dict(ref_mode=ref)
    if not maps:
        kw.update(c_pos_map=None, c_neg_map=None)
    return kw


def _push(sim, seq, frames, flows, lo, hi):
    for i in range(lo, hi):
        sim.push(frames[i], flows[i] if i else None, int(seq.t_us[i]))
    return sim.pop()


CASES = [(evsim.SIM_DENSE, evsim.SIM_REF_ACCUM, True),
         (evsim.SIM_SPARSE, evsim.SIM_REF_ACCUM, True),
         (evsim.SIM_DENSE, evsim.SIM_REF_RESET, False),
         (evsim.SIM_DIFF, evsim.SIM_REF_RESET, False)]


@pytest.mark.parametrize("mode,ref,maps", CASES)
@pytest.mark.parametrize("split", [0, 1, 4])
def test_restored_stream_continues_bit_exactly(mode, ref, maps, split):
    seq = synth.warped_texture(frames=7, width=130, height=70)
    frames = torch.from_numpy(seq.frames).cuda()
    flows = torch.from_numpy(seq.flows).cuda()
    full = gpu_run(seq, mode, ref_mode=ref, use_maps=maps)
    want = oracle_run(seq, mode, ref_mode=ref, use_maps=maps)
    a = evsim.simulator_for(seq, mode, **_options(seq, mode, ref, maps))
    ev_a = _push(a, seq, frames, flows, 0, split + 1)
    state = a.get_state()
    a.close()
    b = evsim.simulator_for(seq, mode, **_options(seq, mode, ref, maps))
    b.set_state(state)
    ev_b = _push(b, seq, frames, flows, split + 1, seq.frames.shape[0])
    spliced = np.concatenate([ev_a, ev_b])
    assert len(want["events"]) > 0
    assert_same_events(spliced, want["events"], f"split after {split} vs the oracle")
    assert_same_events(spliced, full["events"], f"split after {split} vs the GPU run")
    st = b.stats()
    assert st.frames_committed == seq.frames.shape[0]
    assert st.pixel_substeps == full["stats"].pixel_substeps
    if ref == evsim.SIM_REF_ACCUM and mode != evsim.SIM_DIFF:
        assert np.array_equal(b.reference(), want["R"])
    b.close()


def test_state_of_a_fresh_handle_and_mismatched_restores():
    seq = synth.warped_texture(frames=4, width=70, height=40)
    a = evsim.simulator_for(seq, evsim.SIM_DENSE)
    empty = a.get_state()
    b = evsim.simulator_for(seq, evsim.SIM_DENSE)
    b.set_state(empty)  # nothing pushed yet: b starts the stream itself
    frames = torch.from_numpy(seq.frames).cuda()
    flows = torch.from_numpy(seq.flows).cuda()
    ev = _push(b, seq, frames, flows, 0, 4)
    assert_same_events(ev, oracle_run(seq, evsim.SIM_DENSE)["events"], "fresh state")
    c = evsim.simulator_for(seq, evsim.SIM_SPARSE)
    with pytest.raises(evsim.SimError):
        c.set_state(empty)  # another mode
    d = evsim.Simulator(71, 40)
    with pytest.raises(evsim.SimError):
        d.set_state(empty)  # another size
    with pytest.raises(evsim.SimError):
        b.set_state(empty[:-1])  # truncated
    for h in (a, b, c, d):
        h.close()
