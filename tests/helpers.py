"""Shared helpers of the GPU tests: run a synthetic sequence through the CUDA
library (via the C-ABI binding) and through the CPU oracle."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2209_04634_gb300 import evsim
from paper_2209_04634_gb300 import synth


def oracle_run(seq: synth.Sequence, mode: int = evsim.SIM_DENSE, *, intensity=evsim.SIM_LOG,
               ref_mode=evsim.SIM_REF_ACCUM, c_act_q16: int = -1, substeps=None,
               c_pos_q16=None, c_neg_q16=None, use_maps=True,
               event_time=evsim.SIM_TIME_SUBSTEP) -> dict:
    if mode == evsim.SIM_DIFF:
        return oracle.run_diff(seq.frames, seq.flows, seq.t_us,
                               substeps=seq.substeps if substeps is None else substeps,
                               max_substeps=seq.max_substeps, intensity=intensity,
                               c_pos_q16=oracle.q16(seq.c_pos) if c_pos_q16 is None else c_pos_q16,
                               c_neg_q16=oracle.q16(seq.c_neg) if c_neg_q16 is None else c_neg_q16,
                               cpos_map=seq.cpos_map if use_maps else None,
                               cneg_map=seq.cneg_map if use_maps else None)
    return oracle.run(seq.frames, seq.flows, seq.t_us,
                      mode=oracle.SPARSE if mode == evsim.SIM_SPARSE else oracle.DENSE,
                      substeps=seq.substeps if substeps is None else substeps,
                      max_substeps=seq.max_substeps, intensity=intensity, ref_mode=ref_mode,
                      c_pos_q16=oracle.q16(seq.c_pos) if c_pos_q16 is None else c_pos_q16,
                      c_neg_q16=oracle.q16(seq.c_neg) if c_neg_q16 is None else c_neg_q16,
                      c_act_q16=c_act_q16,
                      cpos_map=seq.cpos_map if use_maps else None,
                      cneg_map=seq.cneg_map if use_maps else None,
                      event_time=oracle.T_CROSSING if event_time == evsim.SIM_TIME_CROSSING
                      else oracle.T_SUBSTEP)


def gpu_run(seq: synth.Sequence, mode: int = evsim.SIM_DENSE, *, device_inputs: bool = True,
            pop_every: int = 1, intensity=evsim.SIM_LOG, ref_mode=evsim.SIM_REF_ACCUM,
            c_act_q16: int = -1, substeps=None, c_pos_q16=None, c_neg_q16=None,
            use_maps=True, event_capacity: int = 0, stream=None, batch: int = 0,
            max_batch: int = 0, tile_height: int = 0,
            event_time: int = evsim.SIM_TIME_SUBSTEP) -> dict:
    """Push every frame of seq through the CUDA library; return the events,
    the committed reference and per-frame statistics."""
    import torch
    kw = dict(intensity=intensity, ref_mode=ref_mode, c_act_q16=c_act_q16,
              event_capacity=event_capacity)
    if substeps is not None:
        kw["substeps"] = substeps
    if c_pos_q16 is not None:
        kw["c_pos_q16"] = c_pos_q16
    if c_neg_q16 is not None:
        kw["c_neg_q16"] = c_neg_q16
    if not use_maps:
        kw["c_pos_map"] = None
        kw["c_neg_map"] = None
    if stream is not None:
        kw["stream"] = stream
    kw["max_batch"] = max_batch
    kw["tile_height"] = tile_height
    kw["event_time"] = event_time
    sim = evsim.simulator_for(seq, mode, **kw)
    if mode == evsim.SIM_DIFF:
        ref_mode = evsim.SIM_REF_RESET  # no reference state
    if batch:
        return _gpu_run_batched(sim, seq, batch, device_inputs, ref_mode)
    out, n_per_frame, ev_per_frame, active = [], [0], [0], [0]
    F = seq.frames.shape[0]
    if device_inputs:
        frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
        flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    for i in range(F):
        if device_inputs:
            sim.push(frames[i], flows[i] if i > 0 else None, int(seq.t_us[i]))
        else:
            sim.push(seq.frames[i], seq.flows[i] if i > 0 else None, int(seq.t_us[i]))
        if i > 0 and (i % pop_every == 0 or i == F - 1):
            st = sim.stats()
            if pop_every == 1:
                n_per_frame.append(st.last_substeps)
                ev_per_frame.append(st.last_batch_events)
                active.append(st.last_active)
            out.append(sim.pop())
    st = sim.stats()
    R = sim.reference() if ref_mode == evsim.SIM_REF_ACCUM else None
    sim.close()
    ev = np.concatenate(out) if out else np.zeros(0, dtype=evsim.EVENT_DTYPE)
    return {"events": ev, "R": R, "stats": st, "n_per_frame": np.array(n_per_frame),
            "ev_per_frame": np.array(ev_per_frame), "active_per_frame": np.array(active)}


def assert_same_events(got: np.ndarray, want: np.ndarray, what: str = "") -> None:
    """Bit-exact comparison of two event streams (same events, same order)."""
    g = got.view(np.uint64) if got.size else np.zeros(0, np.uint64)
    w = want.view(np.uint64) if want.size else np.zeros(0, np.uint64)
    if g.shape == w.shape and np.array_equal(g, w):
        return
    n = min(len(g), len(w))
    bad = np.nonzero(g[:n] != w[:n])[0]
    first = int(bad[0]) if bad.size else n
    gt, gx, gy, gp = oracle.unpack(got[first:first + 3]) if len(got) > first else ([], [], [], [])
    wt, wx, wy, wp = oracle.unpack(want[first:first + 3]) if len(want) > first else ([], [], [], [])
    raise AssertionError(
        f"{what}: event streams differ (gpu {len(got)}, oracle {len(want)} events); first "
        f"difference at {first}: gpu {list(zip(gt, gx, gy, gp))} vs oracle "
        f"{list(zip(wt, wx, wy, wp))}")


def _gpu_run_batched(sim, seq, batch, device_inputs, ref_mode):
    """Push the sequence in batches of `batch` frames (sim_push_frames)."""
    import torch
    F = seq.frames.shape[0]
    if device_inputs:
        frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
        flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    else:
        frames, flows = seq.frames, seq.flows
    out = []
    for i in range(0, F, batch):
        j = min(F, i + batch)
        sim.push_many(frames[i:j], flows[i:j], seq.t_us[i:j])
        out.append(sim.pop())
    st = sim.stats()
    R = sim.reference() if ref_mode == evsim.SIM_REF_ACCUM else None
    sim.close()
    ev = np.concatenate(out) if out else np.zeros(0, dtype=evsim.EVENT_DTYPE)
    return {"events": ev, "R": R, "stats": st}
