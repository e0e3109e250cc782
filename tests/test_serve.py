"""Serving loop (sim_serve_run): under both policies every stream's delivered
event stream equals the stream run alone through a single-stream handle
(same frames, same timestamps), while streams arrive, are admitted by memory
budget, overlap on the device and leave."""
import numpy as np
import pytest

from paper_2209_04634_gb300 import evsim, serve


def _alone(pools, rec, mode):
    seq = pools.seqs[rec["pool"]]
    fr, fl = pools.stream_frames(rec["pool"], rec["phase"], rec["frames"])
    t = np.array([round(j * 1e6 / rec["fps"]) for j in range(rec["frames"])], np.int64)
    sim = evsim.Simulator(seq.width, seq.height, mode=mode, substeps=seq.substeps,
                          max_substeps=seq.max_substeps, c_pos_q16=evsim.q16(seq.c_pos),
                          c_neg_q16=evsim.q16(seq.c_neg), c_pos_map=seq.cpos_map,
                          c_neg_map=seq.cneg_map, max_batch=64,
                          event_capacity=64 * seq.width * seq.height)
    sim.push_many(fr, fl, t)
    ev = sim.pop()
    sim.close()
    return ev


@pytest.mark.gpu
@pytest.mark.parametrize("policy,mode", [("group", evsim.SIM_DENSE), ("group", evsim.SIM_SPARSE),
                                         ("per_stream", evsim.SIM_DENSE)])
def test_served_streams_equal_streams_alone(policy, mode):
    pools = serve.Pools(sizes=((240, 180), (320, 240), (200, 150)), frames=5)
    res, streams = serve.run(pools, policy, mode=mode, horizon_s=2.5, warmup_s=0.2,
                             rate_per_s=8.0, dur_s=(0.3, 1.5), fps=(30, 60, 120), seed=11,
                             max_streams=32, frames_per_step=2, hbm_budget_bytes=1 << 30,
                             events_per_pixel=8)
    assert res["frames_failed"] == 0
    assert res["frames_completed"] == res["frames_released"] > 0
    assert res["admitted"] >= 8 and res["streams_written"] == res["admitted"]
    assert res["peak_streams"] >= 4  # streams overlapped on the device
    assert 0 < res["lat_p50_ms"] <= res["lat_p99_ms"]
    for rec in streams:
        assert rec["status"] == 0
        ev = _alone(pools, rec, mode)
        assert len(ev) == rec["events"], rec
        assert serve.digest(ev) == rec["digest"], rec


@pytest.mark.gpu
def test_serving_admission_waits_for_memory():
    pools = serve.Pools(sizes=((320, 240),), frames=4)
    need = evsim.Group(max_streams=1, frames_per_step=2).state_bytes(
        320, 240, substeps=0, max_substeps=8, event_capacity=2 * 320 * 240,
        c_pos_map=pools.seqs[0].cpos_map, c_neg_map=pools.seqs[0].cneg_map)
    res, streams = serve.run(pools, "group", horizon_s=2.0, warmup_s=0.0, rate_per_s=10.0,
                             dur_s=(0.2, 0.6), fps=(60,), seed=5, warm_start=False,
                             max_streams=16, frames_per_step=2, hbm_budget_bytes=2 * need,
                             events_per_pixel=2)
    assert res["peak_streams"] <= 2          # the budget holds two streams
    assert res["admit_wait_p99_ms"] > 0      # later arrivals waited for memory
    assert res["frames_failed"] == 0


def test_digest_matches_horner_rule():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2 ** 63, size=257, dtype=np.uint64)
    h = 0
    for v in w:
        h = (h * serve.DIGEST_M + int(v)) % (1 << 64)
    assert serve.digest(w) == h
    assert serve.digest(np.zeros(0, np.uint64)) == 0
