"""Multi-stream group (simb_*): every member's event stream equals that of a
single-stream handle fed the same frames (which the parity tests pin to the
oracle), whatever the mix of sizes, tile classes and frames per step, with
graphs on and off; admission by budget and by slots; eviction; failure
isolation between members."""
import ctypes

import numpy as np
import pytest

from paper_2209_04634_gb300 import evsim, synth
from .helpers import assert_same_events, oracle_run


def _mix():
    """(name, sequence, options): mixed sizes and every axis of the tile class."""
    blob = synth.blob_translation(frames=7)
    blob2 = synth.blob_translation(seed=77, frames=7, width=200, height=150, flow=(-2.5, 1.25))
    warp = synth.warped_texture(frames=7, width=320, height=240)
    rect = synth.moving_rectangles(frames=7, width=400, height=256, side=(40, 120))
    return [
        ("blob_dense", blob, dict(mode=evsim.SIM_DENSE)),
        ("blob_sparse_adaptive", blob2, dict(mode=evsim.SIM_SPARSE, substeps=0, max_substeps=6)),
        ("warp_dense_maps_adaptive", warp, dict(mode=evsim.SIM_DENSE)),
        ("warp_sparse_maps_adaptive", warp, dict(mode=evsim.SIM_SPARSE)),
        ("rect_dense_reset_rgb", rect, dict(mode=evsim.SIM_DENSE, ref_mode=evsim.SIM_REF_RESET)),
        ("blob_sparse_linear", blob, dict(mode=evsim.SIM_SPARSE, intensity=evsim.SIM_LINEAR,
                                          c_pos_q16=9 << 16, c_neg_q16=11 << 16)),
    ]


def _alone(seq, opts):
    """The same stream through a single-stream handle, one frame per push."""
    import torch
    sim = evsim.Simulator(seq.width, seq.height, **evsim.seq_options(seq, **opts))
    frames = torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda()
    flows = torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()
    out = []
    for i in range(seq.frames.shape[0]):
        sim.push(frames[i], flows[i] if i else None, int(seq.t_us[i]))
        out.append(sim.pop())
    sim.close()
    return np.concatenate(out)


def _run_group(mix, *, use_graphs, fmax, schedule, host=False):
    """Push the mixed streams through one group; member i queues schedule(i,
    step) frames before each step.  Returns the events of each member."""
    import torch
    g = evsim.Group(max_streams=16, frames_per_step=fmax, use_graphs=use_graphs)
    ids, inputs, nxt, out = [], [], [], []
    for name, seq, opts in mix:
        sid = g.admit(seq.width, seq.height, **evsim.seq_options(seq, **opts))
        assert sid is not None, name
        ids.append(sid)
        if host:
            inputs.append((seq.frames, seq.flows))
        else:
            inputs.append((torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda(),
                           torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()))
        g.push(sid, inputs[-1][0][0], None, int(seq.t_us[0]))
        nxt.append(1)
        out.append([])
    step = 0
    while any(nxt[i] < mix[i][1].frames.shape[0] for i in range(len(mix))):
        for i, (name, seq, _o) in enumerate(mix):
            F = seq.frames.shape[0]
            k = min(schedule(i, step), F - nxt[i], fmax)
            for _ in range(k):
                j = nxt[i]
                g.push(ids[i], inputs[i][0][j], inputs[i][1][j], int(seq.t_us[j]))
                nxt[i] += 1
        g.step()
        if step % 2 == 1:
            for i in range(len(mix)):
                out[i].append(g.pop(ids[i]))
        step += 1
    for i in range(len(mix)):
        out[i].append(g.pop(ids[i]))
    st = g.stats()
    g.close()
    return [np.concatenate(o) for o in out], st


@pytest.mark.gpu
@pytest.mark.parametrize("use_graphs", [True, False])
def test_group_members_match_single_stream_handles(use_graphs):
    mix = _mix()
    want = [_alone(seq, opts) for _n, seq, opts in mix]
    got, st = _run_group(mix, use_graphs=use_graphs, fmax=3,
                         schedule=lambda i, step: (i + step) % 4)
    for (name, _s, _o), gv, wv in zip(mix, got, want):
        assert len(wv) > 0, name
        assert_same_events(gv, wv, name)
    assert st.members == 0 or st.members == len(mix)
    assert st.tile_classes >= 5
    if use_graphs:
        assert st.graph_captures == 1 and st.graph_launches == st.steps
    else:
        assert st.graph_launches == 0


@pytest.mark.gpu
def test_group_member_matches_oracle_directly():
    seq = synth.blob_translation(seed=91, frames=5)
    want = oracle_run(seq)["events"]
    got, _ = _run_group([("blob", seq, dict(mode=evsim.SIM_DENSE))], use_graphs=True, fmax=2,
                        schedule=lambda i, step: 2)
    assert_same_events(got[0], want, "group vs oracle")


@pytest.mark.gpu
def test_group_host_frames_match_device_frames():
    mix = _mix()[:3]
    dev, _ = _run_group(mix, use_graphs=True, fmax=2, schedule=lambda i, s: 1 + (i + s) % 2)
    host, _ = _run_group(mix, use_graphs=True, fmax=2, schedule=lambda i, s: 1 + (i + s) % 2,
                         host=True)
    for (name, _s, _o), a, b in zip(mix, dev, host):
        assert_same_events(b, a, name)


@pytest.mark.gpu
def test_group_many_small_streams_one_frame_per_step():
    seqs = synth.mixed_streams(frames=4, sizes=((240, 180, 12), (320, 240, 4)))
    mix = [(s.name, s, dict(mode=evsim.SIM_DENSE if i % 2 else evsim.SIM_SPARSE))
           for i, s in enumerate(seqs)]
    want = [_alone(seq, opts) for _n, seq, opts in mix]
    got, st = _run_group(mix, use_graphs=True, fmax=1, schedule=lambda i, s: 1)
    for (name, _s, _o), gv, wv in zip(mix, got, want):
        assert_same_events(gv, wv, name)
    assert st.steps == 3 and st.frames_stepped == 3 * len(mix)


@pytest.mark.gpu
def test_group_admission_by_slots_and_budget_and_eviction():
    g = evsim.Group(max_streams=2, frames_per_step=2)
    a = g.admit(240, 180)
    b = g.admit(640, 480)
    assert a is not None and b is not None and a != b
    assert g.admit(240, 180) is None                  # no slot left
    g.evict(a)
    c = g.admit(240, 180)
    assert c == a                                     # ids are reused
    st = g.stats()
    assert st.members == 2 and st.admit_refused == 1
    assert st.bytes_used == g.state_bytes(240, 180) + g.state_bytes(640, 480)
    g.close()

    need = evsim.Group(max_streams=8).state_bytes(640, 480)
    g = evsim.Group(max_streams=8, hbm_budget_bytes=2 * need + need // 2, frames_per_step=4)
    assert g.admit(640, 480) is not None
    assert g.admit(640, 480) is not None
    assert g.admit(640, 480) is None                  # over the budget
    assert g.admit(240, 180) is not None              # a smaller stream still fits
    assert g.stats().bytes_used <= 2 * need + need // 2
    g.close()


@pytest.mark.gpu
def test_group_overflow_of_one_member_leaves_the_others_intact():
    import torch
    good = synth.blob_translation(frames=4)
    bad = synth.blob_translation(seed=5, frames=4)
    want = _alone(good, dict(mode=evsim.SIM_DENSE))
    g = evsim.Group(max_streams=4, frames_per_step=1)
    ig = g.admit(good.width, good.height, **evsim.seq_options(good))
    ib = g.admit(bad.width, bad.height, **evsim.seq_options(bad, event_capacity=16))
    tg = (torch.from_numpy(good.frames).cuda(), torch.from_numpy(good.flows).cuda())
    tb = (torch.from_numpy(bad.frames).cuda(), torch.from_numpy(bad.flows).cuda())
    g.push(ig, tg[0][0], None, int(good.t_us[0]))
    g.push(ib, tb[0][0], None, int(bad.t_us[0]))
    out = []
    for j in range(1, 4):
        g.push(ig, tg[0][j], tg[1][j], int(good.t_us[j]))
        g.push(ib, tb[0][j], tb[1][j], int(bad.t_us[j]))
        g.step()
        out.append(g.pop(ig))
        with pytest.raises(evsim.SimError) as e:
            g.pop(ib)
        assert e.value.code == evsim.SIM_ERR_EVENT_OVERFLOW
        assert g.stream_stats(ib).frames_committed == 1
    assert_same_events(np.concatenate(out), want, "good member")
    g.close()


def test_group_create_validates_and_needs_a_device():
    lib = evsim.load()
    cfg = evsim.simb_config()
    assert lib.simb_config_default(ctypes.byref(cfg)) == 0
    assert cfg.max_streams == 64 and cfg.frames_per_step == 4 and cfg.use_graphs == 1
    h = ctypes.c_void_p()
    bad = evsim.simb_config()
    lib.simb_config_default(ctypes.byref(bad))
    bad.max_streams = 0
    assert lib.simb_create(ctypes.byref(bad), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    bad.max_streams = evsim.SIM_MAX_GROUP + 1
    assert lib.simb_create(ctypes.byref(bad), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    lib.simb_config_default(ctypes.byref(bad))
    bad.frames_per_step = 0
    assert lib.simb_create(ctypes.byref(bad), ctypes.byref(h)) == evsim.SIM_ERR_ARG
    assert lib.simb_step(None, None) == evsim.SIM_ERR_ARG
    assert lib.simb_push(None, 0, None, 0, None, 0, 0) == evsim.SIM_ERR_ARG
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        assert lib.simb_create(ctypes.byref(cfg), ctypes.byref(h)) == evsim.SIM_ERR_NO_DEVICE


def _run_group_delivered(mix, *, fmax, schedule, delivery_events=0, depth=2):
    """As _run_group, with simb_step_deliver / simb_collect (up to `depth`
    deliveries in flight); returns each member's events."""
    import torch
    g = evsim.Group(max_streams=16, frames_per_step=fmax, delivery_events=delivery_events)
    ids, inputs, nxt = [], [], []
    for name, seq, opts in mix:
        sid = g.admit(seq.width, seq.height, **evsim.seq_options(seq, **opts))
        ids.append(sid)
        inputs.append((torch.from_numpy(np.ascontiguousarray(seq.frames)).cuda(),
                       torch.from_numpy(np.ascontiguousarray(seq.flows)).cuda()))
        g.push(sid, inputs[-1][0][0], None, int(seq.t_us[0]))
        nxt.append(1)
    got = {sid: [] for sid in ids}
    inflight = 0
    committed = {}

    def collect():
        tab, ev = g.collect()
        for r in tab:
            assert r["status"] == 0
            got[int(r["id"])].append(ev[r["first"]: r["first"] + r["count"]])
            committed[int(r["id"])] = int(r["frames_committed"])

    step = 0
    while any(nxt[i] < mix[i][1].frames.shape[0] for i in range(len(mix))):
        for i, (name, seq, _o) in enumerate(mix):
            k = min(schedule(i, step), seq.frames.shape[0] - nxt[i], fmax)
            for _ in range(k):
                j = nxt[i]
                g.push(ids[i], inputs[i][0][j], inputs[i][1][j], int(seq.t_us[j]))
                nxt[i] += 1
        if inflight == depth:
            collect()
            inflight -= 1
        g.step_deliver()
        inflight += 1
        step += 1
    while inflight:
        collect()
        inflight -= 1
    # deliveries without frames until nothing is left on the device
    for _ in range(10000):
        g.step_deliver()
        before = sum(len(x) for v in got.values() for x in v)
        collect()
        if sum(len(x) for v in got.values() for x in v) == before:
            break
    for i in range(len(mix)):
        assert committed[ids[i]] == mix[i][1].frames.shape[0]
    with pytest.raises(evsim.SimError) as e:
        g.pop(ids[0])
    assert e.value.code == evsim.SIM_ERR_STATE
    g.close()
    return [np.concatenate(got[sid]) if got[sid] else np.zeros(0, evsim.EVENT_DTYPE)
            for sid in ids]


@pytest.mark.gpu
@pytest.mark.parametrize("delivery_events,depth", [(0, 1), (0, 2), (3000, 2)])
def test_group_delivery_matches_single_stream_handles(delivery_events, depth):
    mix = _mix()
    want = [_alone(seq, opts) for _n, seq, opts in mix]
    got = _run_group_delivered(mix, fmax=2, schedule=lambda i, s: 1 + (i + s) % 2,
                               delivery_events=delivery_events, depth=depth)
    for (name, _s, _o), gv, wv in zip(mix, got, want):
        assert_same_events(gv, wv, name)


@pytest.mark.gpu
@pytest.mark.parametrize("th", [8, 16])
def test_group_members_in_either_tile_shape_match_the_oracle(th):
    """Members whose configuration asks for 64 x 8 (or 64 x 16) tiles run in
    the group's kernel of that shape; a mixed-size group of dense and sparse
    members, with threshold maps and adaptive N, equals the oracle."""
    mix = [(n, s, dict(o, tile_height=th)) for n, s, o in _mix()]
    got, st = _run_group(mix, use_graphs=True, fmax=2, schedule=lambda i, s: 1 + (i + s) % 2)
    for (name, seq, opts), ev in zip(mix, got):
        assert_same_events(ev, _oracle_events(seq, opts), f"{name} in 64x{th} tiles")


def _oracle_events(seq, opts):
    """The oracle's events for a member admitted with these options."""
    import oracle
    return oracle.run(
        seq.frames, seq.flows, seq.t_us,
        mode=oracle.SPARSE if opts.get("mode") == evsim.SIM_SPARSE else oracle.DENSE,
        substeps=opts.get("substeps", seq.substeps),
        max_substeps=opts.get("max_substeps", seq.max_substeps),
        intensity=oracle.LINEAR if opts.get("intensity") == evsim.SIM_LINEAR else oracle.LOG,
        ref_mode=oracle.RESET if opts.get("ref_mode") == evsim.SIM_REF_RESET else oracle.ACCUM,
        c_pos_q16=opts.get("c_pos_q16", oracle.q16(seq.c_pos)),
        c_neg_q16=opts.get("c_neg_q16", oracle.q16(seq.c_neg)),
        cpos_map=opts.get("c_pos_map", seq.cpos_map),
        cneg_map=opts.get("c_neg_map", seq.cneg_map))["events"]


@pytest.mark.gpu
def test_group_member_takes_the_autotuned_tile_shape(tmp_path):
    """A member admitted with the automatic tile shape takes the shape the
    autotuner table holds for its configuration (64 x 8 here), and its events
    equal the oracle's."""
    seq = synth.blob_translation(seed=93, frames=5, width=200, height=90)
    f = tmp_path / "table.txt"
    f.write_text(f"200 90 1 0 {seq.substeps} 0 0 0 0 8 0 1.0 2.0 0.0\\n")
    evsim.autotune_load(str(f))
    got, _ = _run_group([("blob", seq, dict(mode=evsim.SIM_DENSE, c_pos_map=None,
                                            c_neg_map=None))],
                        use_graphs=False, fmax=2, schedule=lambda i, s: 2)
    assert_same_events(got[0], _oracle_events(seq, dict(mode=evsim.SIM_DENSE, c_pos_map=None,
                                                         c_neg_map=None)), "tuned 64x8 member")
