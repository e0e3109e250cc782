#!/usr/bin/env python
"""Throughput benchmark of the GB300 event simulator.

Workload (one "step"): the 1280x720 moving-rectangles sequence (300 frames
of 8-bit RGB at 60 fps converted to BT.601 luma on the device, a static
textured background with six textured rectangles moving at 2-12 px/frame,
N = 10 substeps, C = 0.15 log units) run through the dense simulator
(Sec. III-A of arXiv 2209.04634) and through the sparse simulator
(Sec. III-B), each from frame 0, with the events popped into device memory.
It stands in for the paper's 1280x720 low events-per-frame recording (Sec.
IV-A, Fig. 4).  Inputs (3.0 GB) are resident in HBM when the timed region
starts; they exceed the 129 MB L2, so no flush is needed between steps.

Metric: Gpix-substeps/s = sum over frames and both passes of W H N, divided
by the device time of the timed steps (CUDA events on the simulators'
stream, max over ranks).  events/s is reported beside it.  The line also
carries the 640x480 warped-texture step (Sec. IV-A, Fig. 3 shape) and the
240x180 blob-translation step as objects, rooflines of every kernel, the
batched and serving patterns and the CPU oracle (one core and all cores).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain restatement of the method
used as the parity reference) on all of this host's cores on a bounded
sample of the same workload.  Under torchrun each rank runs its own
independently seeded stream (weak scaling, no collective on the data path);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("moving_rectangles 1280x720 RGB (BT.601 luma on device), 300 frames at 60 fps, "
            "static textured background + 6 textured rectangles at 2-12 px/frame "
            "(occlusions), N = 10, C = 0.15; dense + sparse passes")
C2_WORKLOAD = ("warped_texture 640x480 luma, 100 frames, smooth flow <= 8 px/frame, adaptive "
               "substeps <= 8, C = 0.2 with per-pixel noise sigma 0.03; dense + sparse passes")
C1_WORKLOAD = ("blob_translation 240x180 luma, 20 frames, 64 Gaussian blobs shifted by "
               "(3.2, -1.7) px/frame, N = 8, C = 0.2; dense + sparse passes")
METRIC = "Gpix-substeps/s"
C3_SEED, C2_SEED, C1_SEED = 5209, 4209, 3209


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=300,
                    help="frames of the headline workload (300; smaller for profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=50)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=12.0)
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving object (e.g. with --serve-seconds 120) and print it")
    ap.add_argument("--no-diff", action="store_true",
                    help="skip the paper-mode, accumulate, difference and crossing-time objects")
    ap.add_argument("--no-flow", action="store_true",
                    help="skip the device optical-flow object")
    ap.add_argument("--profile-flow", type=int, default=0,
                    help="profiling: only compute the device flow of this many frame pairs of "
                         "the 640x480 workload, then exit")
    ap.add_argument("--profile-adaptive", type=int, default=0,
                    help="profiling: only run this many dense + sparse steps of the 640x480 "
                         "warped-texture workload (adaptive N: flow-maximum and activity "
                         "pre-passes), 64x16 tiles in block order, then exit")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the 640x480 and 240x180 workload objects")
    ap.add_argument("--only", default="",
                    help="profiling: run only this headline pass (dense or sparse)")
    ap.add_argument("--tile-height", type=int, default=0, choices=[0, 8, 16],
                    help="batch kernel tile height; 0: the library's autotuner chooses")
    ap.add_argument("--substeps", type=int, default=0,
                    help="fixed substeps per frame for profiling runs; 0: the workload's N")
    return ap.parse_args()


def dist_setup(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(v: float, op) -> float:
    import torch
    import torch.distributed as dist
    # NCCL reduces device tensors; gloo (the CPU tests of this path) host ones
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch.distributed as dist
    return _reduce(v, dist.ReduceOp.MAX)


def sum_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch.distributed as dist
    return _reduce(v, dist.ReduceOp.SUM)


def weak_scaling_value(ws, units: float, ms: float) -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time (Gunits/s), and that time (ms)."""
    ms_max = max_over_ranks(ws, ms)
    return sum_over_ranks(ws, units) / (ms_max / 1e3) / 1e9, ms_max


def stream_seed(rank: int, base: int = C2_SEED) -> int:
    """Seed of rank's stream: every replica simulates its own sequence."""
    return base + 1000 * rank


def bind_host_to_gpu(gpu_index: int) -> dict:
    """Run this process on the host CPUs local to its GPU (sysfs
    local_cpulist of the GPU's PCI device), so that host memory it allocates
    from now on - pinned buffers included - is placed on the GPU's own
    memory node (first touch).  Returns what was done."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout.strip().splitlines()[0].strip()
        dom, rest = out.split(":", 1)
        dev = f"{int(dom, 16):04x}:{rest}".lower()
        base = f"/sys/bus/pci/devices/{dev}"
        node = open(base + "/numa_node").read().strip()
        cpus = set()
        for part in open(base + "/local_cpulist").read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        cpus &= os.sched_getaffinity(0)
        if cpus:
            os.sched_setaffinity(0, cpus)
        return {"pci": dev, "numa_node": node, "cpus": len(cpus)}
    except (OSError, ValueError, IndexError, subprocess.SubprocessError) as e:
        return {"unbound": str(e)[:120]}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                         if r[3].replace(".", "").isdigit())}


KERNEL_SOURCES = {  # kernel kind -> the sources that define it
    "dense": ("internal.h", "tile.cuh", "tile_dense.cu"),
    "sparse": ("internal.h", "tile.cuh", "tile_dense.cu", "tile_sparse.cu"),
    "order": ("internal.h", "tile.cuh", "kernels.cu"),
    "mask": ("internal.h", "tile.cuh", "kernels.cu"),
    "flowmax": ("internal.h", "tile.cuh", "kernels.cu"),
    "init": ("internal.h", "tile.cuh", "kernels.cu"),
}


def kernel_source_digest(kind: str = "dense") -> str:
    """Digest of one kernel's sources (its template, its translation unit and
    the structures they share)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2209_04634_gb300", "csrc")
    for name in KERNEL_SOURCES.get(kind, KERNEL_SOURCES["dense"]):
        with open(os.path.join(d, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(key: str, kind: str):
    """DRAM bytes per launch of kernel `kind` from the committed ncu capture
    recorded under `key` (profiles/traffic.json), if it was taken on the
    current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(key)
    if not e or e.get("source_digest") != kernel_source_digest(kind):
        return None
    return e.get("dram_bytes_per_launch")


PASS_NAMES = {0: "dense", 1: "sparse"}


class Passes:
    """The dense and sparse simulators of one workload, inputs resident on
    the device, events popped into one device buffer.  The two simulators
    are independent handles, each on a CUDA stream of its own, so their
    kernels run concurrently; `stream` orders the step around them (each
    step's work starts after what `stream` holds and `stream` waits for it).
    Each pass's tile shape comes from the library's autotuner, run on a
    sample of this stream (its first frames) before any timed region."""

    def __init__(self, seq, stream, cap, *, modes=(0, 1), tile_height=0, tune_frames=32,
                 substeps=0):
        import torch

        from paper_2209_04634_gb300 import evsim
        self.seq = seq
        self.stream = stream
        self.frames = torch.from_numpy(seq.frames).cuda()
        self.flows = torch.from_numpy(seq.flows).cuda()
        self.cap = cap
        self.out = torch.empty(cap * 8, dtype=torch.uint8, device="cuda")
        self.tune, self.sims, self.streams = {}, {}, {}
        W, H = seq.width, seq.height
        extra = {"substeps": substeps} if substeps else {}
        for m in modes:
            name = PASS_NAMES[m]
            if tile_height:
                th, tune = tile_height, {"tile_height": tile_height, "fixed": True}
            else:
                n = min(tune_frames, len(seq.t_us))
                th, us16, us8, usr = evsim.autotune_sample(
                    W, H, self.frames[:n], self.flows[:n], seq.t_us[:n],
                    **evsim.seq_options(seq, mode=m, **extra))
                tune = {"tile_height": th, "kernel": "rows" if th == evsim.SIM_TILE_ROWS
                        else f"tiles 64x{th}", "sample": f"first {n} frames",
                        "us_per_frame_64x16": us16, "us_per_frame_64x8": us8,
                        "us_per_frame_rows": usr}
            self.streams[name] = torch.cuda.Stream()
            sim = evsim.simulator_for(seq, m, event_capacity=cap, stream=self.streams[name],
                                      tile_height=th, **extra)
            st = sim.stats()
            assert st.tile_height == th
            tune["block_order"] = ["linear", "serpentine", "balanced"][st.block_order]
            self.tune[name], self.sims[name] = tune, sim

    def step(self, serial: bool = False) -> int:
        """One step: both passes enqueued (each on its own stream, after what
        `stream` holds) before either is popped, so they run concurrently;
        serial: each pass pushed and popped before the next starts (each
        kernel then runs alone, for per-kernel times)."""
        from paper_2209_04634_gb300 import evsim
        n_ev = 0
        order = [[n] for n in self.sims] if serial else [list(self.sims)]
        for names in order:
            for name in names:
                self.streams[name].wait_stream(self.stream)
                self.sims[name].reset()
                self.sims[name].push_many(self.frames, self.flows, self.seq.t_us)
            for name in names:
                n, rc = self.sims[name].pop_into(self.out, self.cap)
                assert rc == evsim.SIM_OK, rc
                n_ev += n
                self.stream.wait_stream(self.streams[name])
        return n_ev

    def profiled_kernel_times(self, steps: int) -> dict:
        """Per-kernel CUDA-event times of `steps` serial steps (each kernel
        alone on the GPU; in the concurrent timed steps a kernel's event pair
        would also span the other pass's kernels)."""
        self.profile(True)
        self.reset_kernel_times()
        for _ in range(steps):
            self.step(serial=True)
        kt = self.kernel_times()
        self.profile(False)
        return kt

    def stats(self) -> dict:
        """Per pass: the units of one step (read from the library's counters
        after a step)."""
        out = {}
        for name, sim in self.sims.items():
            st = sim.stats()
            out[name] = {"pixel_substeps": st.pixel_substeps,
                         "active_substeps": st.active_substeps,
                         "active_pixels": st.active_pixels, "events": st.events_popped,
                         "frames": st.frames_committed, "batch_frames": st.max_batch}
        return out

    def profile(self, on: bool):
        for sim in self.sims.values():
            sim.set_profiling(on)

    def reset_kernel_times(self):
        from paper_2209_04634_gb300 import evsim
        for sim in self.sims.values():
            for k in range(len(evsim.KERNEL_NAMES)):
                sim.kernel_time(k, reset=True)

    def kernel_times(self) -> dict:
        """{"pass.kernel": (total ms, launches)} since the last reset."""
        from paper_2209_04634_gb300 import evsim
        kt = {}
        for name, sim in self.sims.items():
            for k, kname in enumerate(evsim.KERNEL_NAMES):
                t, c = sim.kernel_time(k)
                if c:
                    kt[f"{name}.{kname}"] = (t, c)
        return kt

    def close(self):
        for sim in self.sims.values():
            sim.close()
        self.sims = {}


def timed_steps(passes, steps: int, warmup: int):
    """Device time of `steps` steps after `warmup` (CUDA events on the
    passes' stream, synchronised on both sides), with per-kernel device times
    from CUDA event pairs around every launch.  Returns (ms, events, kernel
    times, units per step)."""
    import torch
    passes.step()
    units = passes.stats()
    for _ in range(warmup):
        passes.step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(passes.stream)
    n_ev = 0
    for _ in range(steps):
        n_ev += passes.step()
    e1.record(passes.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = passes.profiled_kernel_times(steps)
    return ms, n_ev, kt, units


def workload_object(name, desc, seq, stream, args, cap, key):
    """A workload other than the headline one: value, kernel times and
    rooflines of its dense + sparse step."""
    ps = Passes(seq, stream, cap, tile_height=args.tile_height)
    steps = max(5, args.steps)
    ms, n_ev, kt, units = timed_steps(ps, steps, max(3, args.warmup))
    work = sum(u["pixel_substeps"] for u in units.values())
    out = {"workload": desc, "value": work * steps / (ms / 1e3) / 1e9, "unit": METRIC,
           "ms_per_step": ms / steps, "events_per_s": n_ev / (ms / 1e3),
           "pixel_substeps_per_step": work,
           "active_pixel_substeps_per_step_sparse": units["sparse"]["active_substeps"],
           "kernel_us_per_launch": {k: v[0] / v[1] * 1e3 for k, v in kt.items()},
           "rooflines": rooflines(seq, kt, units, key, steps), "autotune": ps.tune}
    ps.close()
    return out


def oracle_kwargs(s, mode):
    import oracle
    return dict(mode=oracle.DENSE if mode == 0 else oracle.SPARSE, substeps=s.substeps,
                max_substeps=s.max_substeps, c_pos_q16=oracle.q16(s.c_pos),
                c_neg_q16=oracle.q16(s.c_neg), cpos_map=s.cpos_map, cneg_map=s.cneg_map)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_step(s, threads: int):
    """One dense + sparse pass of the oracle over sequence s, on `threads`
    host threads (row bands, oracle.run_bands; 1: the plain single run).
    Returns (pixel-substeps, events, seconds, the event arrays)."""
    import oracle
    work = nev = 0
    evs = []
    t0 = time.perf_counter()
    for mode in (0, 1):
        kw = oracle_kwargs(s, mode)
        r = (oracle.run(s.frames, s.flows, s.t_us, **kw) if threads == 1 else
             oracle.run_bands(s.frames, s.flows, s.t_us, threads=threads, **kw))
        work += int((r["n_per_frame"][1:].astype("int64") * s.width * s.height).sum())
        nev += len(r["events"])
        evs.append(r["events"])
    return work, nev, time.perf_counter() - t0, evs


def cpu_baseline(seq, frames_sample: int, runs: int):
    """The oracle as it stands on a bounded head of the workload: (i) one
    core, once; (ii) all host cores (row bands over threads), `runs` times,
    its output checked identical to (i).  Gpix-substeps/s and events/s."""
    import numpy as np
    s = seq.head(frames_sample)
    cores = host_cores()
    w1, e1, dt1, ev1 = oracle_step(s, 1)
    vals, evps = [], []
    same = True
    for _ in range(runs):
        w, e, dt, ev = oracle_step(s, cores)
        same = same and all(a.shape == b.shape and np.array_equal(a.view(np.uint64),
                                                                  b.view(np.uint64))
                            for a, b in zip(ev, ev1))
        vals.append(w / dt / 1e9)
        evps.append(e / dt)
    mean = statistics.mean(vals)
    sd = statistics.stdev(vals) if len(vals) > 1 else 0.0
    sample = (f"first {frames_sample} frames of the workload, dense + sparse "
              f"({w1} pixel-substeps per run)")
    return {"value": mean, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
            "std": sd, "runs": runs, "events_per_s": statistics.mean(evps),
            "identical_to_single_core": bool(same),
            "single_core": {"value": w1 / dt1 / 1e9, "unit": METRIC, "cores": 1,
                            "seconds": dt1, "events_per_s": e1 / dt1}}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    from paper_2209_04634_gb300 import synth
    n = 6  # frames per sampled step: about 1-2 s of oracle work on all cores
    seq = synth.moving_rectangles(seed=C3_SEED, frames=n)  # the workload's first n frames
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_step(seq, cores)
    works, dts, evs = 0, 0.0, 0
    per = []
    for _ in range(args.steps):
        w, e, dt, _ = oracle_step(seq, cores)
        works += w
        dts += dt
        evs += e
        per.append(w / dt / 1e9)
    value = works / dts / 1e9
    sample = f"first {n} frames of the workload, dense + sparse, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dts / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": args.frames, "width": seq.width,
                   "height": seq.height, "substeps": seq.substeps,
                   "parallelism": f"the CPU oracle on rank 0, {cores} threads (row bands)",
                   "sample": sample},
        "events_per_s": evs / dts,
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                         "sample": sample,
                         "std": statistics.stdev(per) if len(per) > 1 else 0.0},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args, ws, rank, local):
    import torch

    from paper_2209_04634_gb300 import build, evsim, synth
    build.build()
    evsim.load()
    if args.serving_only:
        print(json.dumps({"serving": run_serving(args)}))
        return 0
    if args.profile_flow:
        s = synth.warped_texture(seed=C2_SEED, frames=args.profile_flow + 1)
        fr = torch.from_numpy(s.frames).cuda()
        out = torch.empty((s.height, s.width, 2), dtype=torch.float32, device="cuda")
        fl = evsim.Flow(s.width, s.height)
        for i in range(1, args.profile_flow + 1):
            fl.compute(fr[i - 1], fr[i], out)
        torch.cuda.synchronize()
        fl.close()
        print(json.dumps({"profile_flow": args.profile_flow, "width": s.width,
                          "height": s.height}))
        return 0

    if args.profile_adaptive:
        c2 = synth.warped_texture(seed=C2_SEED)
        pp = Passes(c2, torch.cuda.Stream(), 40_000_000, tile_height=16)
        n = sum(pp.step(serial=True) for _ in range(args.profile_adaptive))
        torch.cuda.synchronize()
        print(json.dumps({"profile_adaptive": args.profile_adaptive, "events": n}))
        return 0

    seq = synth.moving_rectangles(seed=stream_seed(rank, C3_SEED), frames=args.frames)
    F, H, W = seq.frames.shape[:3]
    stream = torch.cuda.Stream()
    cap = 80_000_000  # events of one pass (~65 M dense at C = 0.15)
    ps = Passes(seq, stream, cap, tile_height=args.tile_height, substeps=args.substeps,
                modes=(0,) if args.only == "dense" else (1,) if args.only == "sparse" else (0, 1))
    ps.step()
    units = ps.stats()
    work_step = sum(u["pixel_substeps"] for u in units.values())
    for _ in range(args.warmup):
        ps.step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    n_ev = 0
    for _ in range(args.steps):
        n_ev += ps.step()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(ws)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value, ms_max = weak_scaling_value(ws, work_step * args.steps, ms)
    # per-kernel times: the same steps again with the passes one after the
    # other (timed by the same event pairs, each kernel alone on the GPU)
    kt = ps.profiled_kernel_times(args.steps)
    # every order call of these passes is two kernels: k_units (the frames'
    # flagged row units) and k_order; a tile call in the balanced order is
    # preceded by two more (k_predict: the tiles' cost estimates, k_plan)
    def calls(k, c):
        pass_name, kind = k.split(".", 1)
        if kind == "order":
            return 2 * c
        if kind in ("dense", "sparse") and ps.tune.get(pass_name, {}).get("block_order") == "balanced":
            return 3 * c
        return c
    launches = sum(calls(k, c) for k, (_, c) in kt.items())
    total_ev = sum_over_ranks(ws, n_ev)
    roofs = rooflines(seq, kt, units, "moving_rectangles_1280x720", args.steps)
    dom = max(roofs, key=lambda k: roofs[k]["total_ms"]) if roofs else None

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32 (Q16 fixed point)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": F, "width": W, "height": H,
                   "pixel_format": "RGB8", "pixel_substeps_per_step": work_step,
                   "active_pixel_substeps_per_step_sparse":
                       units.get("sparse", {}).get("active_substeps"),
                   "l2": "inputs larger than L2 (3.0 GB resident), no flush",
                   "parallelism": f"{ws} independent stream(s), one per GPU",
                   "substeps": args.substeps if args.substeps else seq.substeps,
                   "passes": list(ps.sims),
                   "pass_streams": "each pass on a CUDA stream of its own; a step enqueues "
                                   "both before popping either, so they run concurrently"},
        "events_per_s": total_ev / (ms_max / 1e3),
        "wall_ms_per_step": wall / args.steps * 1e3,
        "kernel_us_per_launch": {k: v[0] / v[1] * 1e3 for k, v in kt.items()},
        "kernel_times_from": f"{args.steps} more steps with the passes one after the other "
                             "(CUDA event pairs around every launch, each kernel alone on the GPU)",
        "roofline": dict(roofs[dom], kernel=dom) if dom else None,
        "rooflines": roofs,
        "gpu_launches": launches,
        "clocks": clk,
        "autotune": ps.tune,
    }
    if rank == 0 and not args.no_e2e:
        # pinned buffers on the GPU's own memory node: run on its local CPUs
        # while they are allocated and used, then restore the affinity
        saved = os.sched_getaffinity(0)
        binding = bind_host_to_gpu(local)
        line["e2e"] = run_e2e(args, ps, work_step)
        line["e2e"]["host_binding"] = binding
        os.sched_setaffinity(0, saved)
    ps.close()
    del ps
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_small:
        c2 = synth.warped_texture(seed=stream_seed(rank, C2_SEED))
        line["warped_texture_640x480"] = workload_object(
            "warped_texture_640x480", C2_WORKLOAD, c2, stream, args, 24_000_000,
            "warped_texture_640x480")
        c1 = synth.blob_translation(seed=stream_seed(rank, C1_SEED))
        line["blob_translation_240x180"] = workload_object(
            "blob_translation_240x180", C1_WORKLOAD, c1, stream, args, 2_000_000,
            "blob_translation_240x180")
    if rank == 0 and not args.no_diff:
        c2 = synth.warped_texture(seed=stream_seed(rank, C2_SEED))
        frames = torch.from_numpy(c2.frames).cuda()
        flows = torch.from_numpy(c2.flows).cuda()
        ccap = 24_000_000
        cout = torch.empty(ccap * 8, dtype=torch.uint8, device="cuda")
        line["paper_mode"] = run_paper_mode(args, c2, frames, flows, stream)
        dsim = evsim.simulator_for(c2, evsim.SIM_DENSE, event_capacity=ccap, stream=stream)
        line["accumulate"] = run_accumulate(c2, dsim, frames, flows, stream, ccap, cout)
        dsim.close()
        line["difference"] = run_difference(args, c2, frames, flows, stream)
        line["crossing_time"] = run_crossing_time(args, c2, frames, flows, stream, ccap, cout)
        del frames, flows, cout
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_flow:
        line["lk_flow"] = run_flow(args, stream)
    if rank == 0 and not args.no_batched:
        line["batched"] = run_batched(args)
    if rank == 0 and not args.no_serve:
        line["serving"] = run_serving(args)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(seq, 12, 5)
    if rank == 0:
        print(json.dumps(line))
    return 0

def run_paper_mode(args, seq, frames, flows, stream):
    """The paper's own arithmetic as a configuration (Sec. III, III-A, Table I):
    linear intensity differences, consecutive interpolated frames differenced
    (no reference), the dense method's Table I threshold of 2 (8-bit units)
    and 10 interpolated frames, on the same device-resident sequence."""
    import torch

    from paper_2209_04634_gb300 import evsim
    cap = 60_000_000
    out = torch.empty(cap * 8, dtype=torch.uint8, device="cuda")
    sim = evsim.simulator_for(seq, evsim.SIM_DENSE, event_capacity=cap, stream=stream,
                              intensity=evsim.SIM_LINEAR, ref_mode=evsim.SIM_REF_RESET,
                              substeps=10, c_pos_q16=2 * 65536, c_neg_q16=2 * 65536,
                              c_pos_map=None, c_neg_map=None)

    def step():
        sim.reset()
        sim.push_many(frames, flows, seq.t_us)
        n, rc = sim.pop_into(out, cap)
        assert rc == evsim.SIM_OK, rc
        return n

    step()
    work = sim.stats().pixel_substeps
    for _ in range(3):
        step()
    sim.set_profiling(True)
    step()
    for k in range(len(evsim.KERNEL_NAMES)):
        sim.kernel_time(k, reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_ev = 0
    for _ in range(args.steps):
        n_ev += step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = {}
    for k, name in enumerate(evsim.KERNEL_NAMES):
        t, c = sim.kernel_time(k)
        if c:
            kt[name] = t / c * 1e3
    st = sim.stats()
    sim.close()
    return {"workload": "warped_texture 640x480, 100 frames, dense; linear intensity, "
                        "consecutive differences, C = 2 (Table I), N = 10",
            "value": work * args.steps / (ms / 1e3) / 1e9, "unit": METRIC,
            "ms_per_step": ms / args.steps, "ms_per_frame": ms / args.steps / (len(seq.t_us) - 1),
            "events_per_s": n_ev / (ms / 1e3), "kernel_us_per_launch": kt,
            "tile_height": st.tile_height}


def run_accumulate(seq, sim, frames, flows, stream, cap, out):
    """Accumulated event frames (the paper's second output form) of the dense
    pass: one sim_accumulate launch per frame window (99 per step), device
    time with CUDA events."""
    import torch

    from paper_2209_04634_gb300 import evsim
    sim.reset()
    sim.push_many(frames, flows, seq.t_us)
    n, rc = sim.pop_into(out, cap)
    assert rc == evsim.SIM_OK, rc
    H, W = seq.height, seq.width
    t = seq.t_us - seq.t_us[0]
    acc = torch.zeros((len(t), H, W), dtype=torch.int32, device="cuda")

    def step():
        for i in range(1, len(t)):
            evsim.accumulate(out, n, W, H, int(t[i - 1]) + 1, int(t[i]) + 1, acc[i], stream)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    launches = len(t) - 1
    return {"what": "sim_accumulate of the dense pass's events, one launch per frame window",
            "events": n, "launches_per_pass": launches, "ms_per_pass": ms,
            "us_per_launch": ms * 1e3 / launches,
            "events_scanned_per_s": n * launches / (ms / 1e3)}


def run_difference(args, seq, frames, flows, stream):
    """The difference-frame interpolation method (Sec. III-C) on the same
    device-resident sequence, the flows read as flows between difference
    frames: one 99-frame batch per step, device time with CUDA events."""
    import torch

    from paper_2209_04634_gb300 import evsim
    # every interpolated difference frame is thresholded on its own: far more
    # events than the reference-based methods, hence buffers of its own
    cap = 120_000_000
    out = torch.empty(cap * 8, dtype=torch.uint8, device="cuda")
    sim = evsim.simulator_for(seq, evsim.SIM_DIFF, event_capacity=cap, stream=stream,
                              c_pos_map=None, c_neg_map=None)

    def step():
        sim.reset()
        sim.push_many(frames, flows, seq.t_us)
        n, rc = sim.pop_into(out, cap)
        assert rc == evsim.SIM_OK, rc
        return n

    step()
    work = sim.stats().pixel_substeps
    for _ in range(3):
        step()
    sim.set_profiling(True)
    step()
    for k in range(len(evsim.KERNEL_NAMES)):
        sim.kernel_time(k, reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_ev = 0
    for _ in range(args.steps):
        n_ev += step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = {}
    for k, name in enumerate(evsim.KERNEL_NAMES):
        t, c = sim.kernel_time(k)
        if c:
            kt[name] = t / c * 1e3
    sim.close()
    return {"workload": "warped_texture 640x480, 100 frames, flows read as flows between "
                        "difference frames, adaptive N <= 8, C = 0.2 (uniform)",
            "value": work * args.steps / (ms / 1e3) / 1e9, "unit": METRIC,
            "ms_per_step": ms / args.steps, "events_per_s": n_ev / (ms / 1e3),
            "kernel_us_per_launch": kt}


def run_crossing_time(args, seq, frames, flows, stream, cap, out):
    """The headline step (dense + sparse passes of the same sequence and
    configuration) with per-crossing event times: every crossing at the time
    the line between consecutive substeps meets its level."""
    import torch

    from paper_2209_04634_gb300 import evsim
    sims = [evsim.simulator_for(seq, m, event_capacity=cap, stream=stream,
                                event_time=evsim.SIM_TIME_CROSSING)
            for m in (evsim.SIM_DENSE, evsim.SIM_SPARSE)]

    def step():
        n_ev = 0
        for sim in sims:
            sim.reset()
            sim.push_many(frames, flows, seq.t_us)
            n, rc = sim.pop_into(out, cap)
            assert rc == evsim.SIM_OK, rc
            n_ev += n
        return n_ev

    step()
    work = sum(sim.stats().pixel_substeps for sim in sims)
    for _ in range(3):
        step()
    for sim in sims:
        sim.set_profiling(True)
    step()
    for sim in sims:
        for k in range(len(evsim.KERNEL_NAMES)):
            sim.kernel_time(k, reset=True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_ev = 0
    for _ in range(args.steps):
        n_ev += step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = {}
    for sim, name in zip(sims, ("dense", "sparse")):
        for k, kname in enumerate(evsim.KERNEL_NAMES):
            t, c = sim.kernel_time(k)
            if c:
                kt[f"{name}.{kname}"] = t / c * 1e3
        sim.close()
    return {"workload": "the headline step (warped_texture 640x480, 100 frames, dense + "
                        "sparse) with per-crossing event times",
            "value": work * args.steps / (ms / 1e3) / 1e9, "unit": METRIC,
            "ms_per_step": ms / args.steps, "events_per_s": n_ev / (ms / 1e3),
            "kernel_us_per_launch": kt}


# Integer operations the method defines for one pixel-substep (Sec. III-A as
# restated in include/evsim.h): two offsets (mul, div each), four position
# adds, two bilinear samples (6 ops to split two Q16 positions, 2 neighbour
# indices, 3 blends of 5 ops), the temporal blend (5) and the threshold test
# (difference and two compares).
OPS_PER_PIXEL_SUBSTEP = 4 + 4 + 2 * (6 + 2 + 15) + 5 + 3
SEG_BYTES = 24  # one (frame, substep, tile row) segment of the order kernel's input


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def kernel_model(kind: str, seq, u: dict, launches: int):
    """Algorithmic work of one kernel over one pass of a step: (bytes, ops).
    u: the pass's units (pixel_substeps, active_substeps, active_pixels,
    events, frames).  Bytes are what the method must move through HBM in this
    design: per frame the new frame (ch B/px, the previous one is on chip) and
    its flow (8 B per simulated pixel), per launch (a batch of frames) the
    reference in and out (8 B/px) and the threshold maps (4 B/px); the order
    kernel reads one 24-byte segment per (frame, substep, 64-pixel row) and
    writes 8 B per event."""
    P = seq.width * seq.height
    ch = seq.channels
    Fp = max(0, u["frames"] - 1)  # frames simulated (the first only initialises)
    maps = seq.cpos_map is not None
    per_launch = 8 * P + (4 * P if maps else 0)
    if kind == "dense":
        return Fp * (ch + 8) * P + launches * per_launch, OPS_PER_PIXEL_SUBSTEP * u["pixel_substeps"]
    if kind == "sparse":
        return (Fp * ch * P + 8 * u["active_pixels"] + launches * per_launch,
                OPS_PER_PIXEL_SUBSTEP * u["active_substeps"])
    if kind == "order":
        nsum = u["pixel_substeps"] // max(1, P)
        segs = nsum * seq.height * ((seq.width + 63) // 64)
        return SEG_BYTES * segs + 8 * u["events"], 0
    if kind == "mask":
        return Fp * 2 * ch * P + 8 * u["active_pixels"], 0
    if kind == "flowmax":
        return Fp * 8 * P, 0
    if kind == "init":
        return (ch + 1 + 4) * P, 0
    return 0, 0


def rooflines(seq, kt: dict, units: dict, key: str, steps: int) -> dict:
    """Per kernel of a step: achieved integer issue rate and HBM bandwidth
    against the measured (HBM) and derived (issue) peaks, from the kernel's
    algorithmic work and its CUDA-event device time over `steps` steps (kt:
    total time and launches over those steps; units: one step's); the
    binding resource is the larger fraction."""
    import torch
    pk = measured_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    alu_peak = sms * 4 * 32 * sm_mhz * 1e6 / 1e12  # 4 schedulers x 32 lanes per SM per clock
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    out = {}
    for name, (t_ms, n) in kt.items():
        pass_name, kind = name.split(".", 1)
        u = units.get(pass_name)
        if u is None or kind == "copy":
            continue
        b1, o1 = kernel_model(kind, seq, u, n / steps)
        bytes_, ops = b1 * steps, o1 * steps
        s = t_ms / 1e3
        hbm = bytes_ / s / 1e9 if s > 0 else 0.0
        alu = ops / s / 1e12 if s > 0 else 0.0
        hf, af = hbm / hbm_peak, alu / alu_peak
        tile = kind in ("dense", "sparse")
        traffic = committed_traffic(f"{kind}@{key}", kind)
        r = {"total_ms": t_ms, "launches": n, "avg_launch_us": t_ms / n * 1e3,
             "hbm": {"achieved": hbm, "peak": hbm_peak, "unit": "GB/s", "frac": hf,
                     "algorithmic_bytes_per_launch": bytes_ / n,
                     "peak_source": "measured" if "hbm_gbs" in pk else "fallback"},
             "traffic": traffic}
        if tile:
            r["alu"] = {"achieved": alu, "peak": alu_peak, "unit": "Tops/s (32-bit integer lane ops)",
                        "frac": af, "ops_per_pixel_substep": OPS_PER_PIXEL_SUBSTEP,
                        "ops_per_launch": ops / n,
                        "peak_source": "derived: SMs x 128 lanes x max SM clock of measured peaks file"}
        if tile and af >= hf:
            r.update(bound="alu", achieved=alu, peak=alu_peak, unit=r["alu"]["unit"], frac=af)
        else:
            r.update(bound="hbm", achieved=hbm, peak=hbm_peak, unit="GB/s", frac=hf)
        out[name] = r
    return out

def run_flow(args, stream):
    """Pyramidal Lucas-Kanade flow on the device (the flow the paper's sparse
    and difference simulators use, Sec. III-B, Sec. IV-A), on the 640x480
    and 1280x720 workloads: time per frame pair (CUDA events), accuracy
    against the generators' flow, and the whole pipeline - frames to device
    flow to the dense and sparse simulators - in Gpix-substeps/s."""
    import numpy as np
    import torch

    from paper_2209_04634_gb300 import evsim, synth
    out = {"method": "pyramidal Lucas-Kanade, 3 levels, 7x7 window, 3 iterations, min_eig 64"}
    cases = (("warped_texture_640x480", synth.warped_texture(seed=C2_SEED)),
             ("moving_rectangles_1280x720", synth.moving_rectangles(seed=C3_SEED, frames=60)))
    for name, seq in cases:
        F, H, W = seq.frames.shape[:3]
        frames = torch.from_numpy(seq.frames).cuda()
        est = torch.zeros((F, H, W, 2), dtype=torch.float32, device="cuda")
        fl = evsim.Flow(W, H, pixel_format=seq.channels, stream=stream)

        def flow_pass():
            for i in range(1, F):
                fl.compute(frames[i - 1], frames[i], est[i])

        for _ in range(2):
            flow_pass()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            flow_pass()
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps / (F - 1)
        e = np.hypot(*(est[1:].cpu().numpy() - seq.flows[1:]).transpose(3, 0, 1, 2))
        # the pipeline: device flow into the simulators (dense + sparse)
        sims = [evsim.simulator_for(seq, m, stream=stream, event_capacity=40_000_000)
                for m in (evsim.SIM_DENSE, evsim.SIM_SPARSE)]
        ev_out = torch.empty(40_000_000 * 8, dtype=torch.uint8, device="cuda")

        def pipeline():
            flow_pass()
            n = 0
            for sim in sims:
                sim.reset()
                sim.push_many(frames, est, seq.t_us)
                k, rc = sim.pop_into(ev_out, 40_000_000)
                assert rc == evsim.SIM_OK, rc
                n += k
            return n

        pipeline()
        work = sum(sim.stats().pixel_substeps for sim in sims)
        torch.cuda.synchronize()
        e0.record(stream)
        n_ev = 0
        for _ in range(reps):
            n_ev += pipeline()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        for sim in sims:
            sim.close()
        fl.close()
        out[name] = {"us_per_frame_pair": us, "mpix_per_s": H * W / us,
                     "endpoint_error_px": {"median": float(np.median(e)),
                                           "p90": float(np.percentile(e, 90))},
                     "pipeline": {"value": work / (ms / 1e3) / 1e9, "unit": METRIC,
                                  "ms_per_step": ms, "ms_per_frame": ms / (F - 1),
                                  "events_per_s": n_ev / reps / (ms / 1e3),
                                  "frames": F}}
        del frames, est, ev_out
        torch.cuda.empty_cache()
    return out


BATCHED_WORKLOAD = ("64 concurrent streams (32 x 240x180, 24 x 640x480, 8 x 1280x720), warped "
                    "texture + smooth flow <= 8 px/frame, adaptive N <= 8, C = 0.2 with "
                    "per-pixel noise sigma 0.03, one frame of every stream per step")


def run_batched(args):
    """Batched multi-stream step: a group advances all 64 streams by one frame
    per step (one launch per kernel, replayed from a CUDA graph) against plain
    per-stream handles (one CUDA stream and a few launches per camera), same
    frames, dense and sparse.  Host wall time between device-wide syncs (it is
    the launch overhead that batching removes), events popped at the end; the
    event streams of the two are checked identical."""
    import numpy as np
    import torch

    from paper_2209_04634_gb300 import evsim, synth
    seqs = synth.shifted_streams()
    U = seqs[0].frames.shape[0]
    T = args.batched_steps
    dev = []
    for s in seqs:
        fr = torch.from_numpy(s.frames).cuda()
        fl = torch.from_numpy(s.flows).cuda()
        dev.append((fr, fl, -fl))
    plan = [synth.pingpong(t, U) for t in range(1, T + 1)]

    def inputs(i, t):
        b, a, sign = plan[t - 1]
        fr, fl, rfl = dev[i]
        return fr[b], (fl[b] if sign > 0 else rfl[a])

    def caps(s):
        return (32 if s.width * s.height <= 640 * 480 else 24) * s.width * s.height

    def group_run(mode, timed, th=0):
        g = evsim.Group(max_streams=len(seqs), frames_per_step=1, hbm_budget_bytes=64 << 30)
        ids = [g.admit(s.width, s.height, **evsim.seq_options(s, mode=mode, tile_height=th,
                                                               event_capacity=caps(s)))
               for s in seqs]
        assert all(i is not None for i in ids)
        for i, s in enumerate(seqs):
            g.push(ids[i], dev[i][0][0], None, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(1, T + 1):
            for i in range(len(seqs)):
                f, fl = inputs(i, t)
                g.push(ids[i], f, fl, t * 50_000)
            g.step()
        g.sync()
        wall = time.perf_counter() - t0
        st = g.stats()
        ev = [g.pop(ids[i]) for i in range(len(seqs))] if not timed else None
        work = sum(g.stream_stats(i).pixel_substeps for i in ids)
        g.close()
        return wall, work, st, ev

    def single_run(mode, timed):
        sims = [evsim.Simulator(s.width, s.height, max_batch=1,
                                **evsim.seq_options(s, mode=mode, event_capacity=caps(s)))
                for s in seqs]
        for i, sim in enumerate(sims):
            sim.push(dev[i][0][0], None, 0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(1, T + 1):
            for i, sim in enumerate(sims):
                f, fl = inputs(i, t)
                sim.push(f, fl, t * 50_000)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ev = [sim.pop() for sim in sims] if not timed else None
        work = sum(sim.stats().pixel_substeps for sim in sims)
        for sim in sims:
            sim.close()
        return wall, work, ev

    out = {"workload": BATCHED_WORKLOAD, "steps": T, "streams": len(seqs),
           "pixels_per_step": int(sum(s.width * s.height for s in seqs)), "autotune": {}}
    # the library's autotuner on a sample of each member configuration (its
    # first 6 frames); members admitted with the automatic shape take the
    # table's tile shape (the row kernel's choice maps to 64 x 16 tiles)
    sizes = {}
    for i, s in enumerate(seqs):
        sizes.setdefault((s.width, s.height), i)
    for mode, name in ((evsim.SIM_DENSE, "dense"), (evsim.SIM_SPARSE, "sparse")):
        for (w, h), i in sizes.items():
            fr, fl, _ = dev[i]
            th, u16, u8, ur = evsim.autotune_sample(
                w, h, fr[:U], fl[:U], (np.arange(U) * 50_000).astype(np.int64),
                **evsim.seq_options(seqs[i], mode=mode, event_capacity=caps(seqs[i])))
            out["autotune"][f"{name}.{w}x{h}"] = {
                "choice": "rows" if th == evsim.SIM_TILE_ROWS else f"64x{th}",
                "member_tiles": "64x16" if th == evsim.SIM_TILE_ROWS else f"64x{th}",
                "us_per_frame_64x16": u16, "us_per_frame_64x8": u8, "us_per_frame_rows": ur}
    for mode, name in ((evsim.SIM_DENSE, "dense"), (evsim.SIM_SPARSE, "sparse")):
        # parity of the two launch patterns on the same frames
        _w, _wk, _st, ev_g = group_run(mode, False)
        _w, _wk, ev_s = single_run(mode, False)
        same = all(a.shape == b.shape and np.array_equal(a.view(np.uint64), b.view(np.uint64))
                   for a, b in zip(ev_g, ev_s))
        n_events = int(sum(len(a) for a in ev_g))
        gw, work, st, _ = group_run(mode, True)
        g16, _w16, _st16, _ = group_run(mode, True, th=16)
        g8, _w8, _st8, _ = group_run(mode, True, th=8)
        sw, work_s, _ = single_run(mode, True)
        assert work == work_s
        out[name] = {
            "group": {"value": work / gw / 1e9, "unit": METRIC, "ms_per_step": gw / T * 1e3,
                      "kernel_launches_per_step": st.kernel_launches / max(1, st.steps),
                      "graph_launches": st.graph_launches, "tile_classes": st.tile_classes,
                      "tiles": "autotuned per member configuration"},
            "group_all_64x16": {"value": work / g16 / 1e9, "ms_per_step": g16 / T * 1e3},
            "group_all_64x8": {"value": work / g8 / 1e9, "ms_per_step": g8 / T * 1e3},
            "per_stream": {"value": work / sw / 1e9, "unit": METRIC,
                           "ms_per_step": sw / T * 1e3},
            "speedup": sw / gw,
            "identical_events": bool(same),
            "events_per_step": n_events / T,
        }
    return out


SERVING_WORKLOAD = ("Poisson stream arrivals (mean 4/s), sizes uniform over 240x180, 346x260, "
                    "640x480, 1280x720, 1920x1080 luma, 30/60/120 fps, 10-60 s each, warped "
                    "texture + smooth flow (adaptive N <= 8, C = 0.2, noise sigma 0.03), "
                    "steady-state population at t = 0, admission by an 8 GiB device budget; "
                    "frames device-resident, released on a wall-clock timeline")


def run_serving(args):
    """Serving loop on one arrival trace under both policies: continuous
    batching over a group, and one handle and CUDA stream per camera."""
    from paper_2209_04634_gb300 import evsim, serve
    pools = serve.Pools()
    out = {"workload": SERVING_WORKLOAD, "horizon_s": args.serve_seconds, "warmup_s": 2.0,
           "mode": "dense"}
    for policy in ("group", "per_stream"):
        res, _streams = serve.run(pools, policy, mode=evsim.SIM_DENSE,
                                  horizon_s=args.serve_seconds, warmup_s=2.0)
        keep = ("arrived", "admitted", "never_admitted", "peak_streams", "frames_released",
                "frames_completed", "frames_failed", "events", "pixel_substeps", "steps",
                "kernel_launches", "wall_s", "gpix_substeps_per_s", "events_per_s",
                "lat_p50_ms", "lat_p90_ms", "lat_p99_ms", "lat_max_ms", "lat_mean_ms",
                "admit_wait_p50_ms", "admit_wait_p99_ms", "latencies")
        out[policy] = {k: res[k] for k in keep}
    g, p = out["group"], out["per_stream"]
    out["p99_speedup"] = p["lat_p99_ms"] / g["lat_p99_ms"] if g["lat_p99_ms"] else None
    out["p50_speedup"] = p["lat_p50_ms"] / g["lat_p50_ms"] if g["lat_p50_ms"] else None
    return out


def run_e2e(args, ps, work_step):
    """Same metric through the C ABI with host buffers in pinned memory, every
    step: the step's frames and flows cross from the host (copied into device
    staging chunk by chunk, overlapping the kernels - the library's default;
    and, as `mapped`, read in place by the kernels through their device
    mapping) and the events are read back to pinned host memory."""
    import torch

    from paper_2209_04634_gb300 import evsim
    seq = ps.seq
    frames_h = torch.from_numpy(seq.frames).pin_memory()
    flows_h = torch.from_numpy(seq.flows).pin_memory()
    cap = ps.cap
    out_h = torch.empty(cap * 8, dtype=torch.uint8).pin_memory()
    fr_np, fl_np, out_np = frames_h.numpy(), flows_h.numpy(), out_h.numpy().view(evsim.EVENT_DTYPE)
    h2d = len(ps.sims) * (seq.frames.nbytes + seq.flows[1:].nbytes)

    def measure(sims):
        def step():
            d2h = 0
            for sim in sims:
                sim.reset()
                sim.push_many(fr_np, fl_np, seq.t_us)
                n, rc = sim.pop_into(out_np, cap)
                assert rc == evsim.SIM_OK, rc
                d2h += n * 8
            return d2h

        for _ in range(2):
            step()
        steps = max(3, args.steps // 4)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ps.stream)
        d2h = 0
        for _ in range(steps):
            d2h += step()
        e1.record(ps.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return {"value": work_step * steps / (ms / 1e3) / 1e9, "unit": METRIC,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h // steps),
                "steps": steps, "ms_per_step": ms / steps}

    line = measure(list(ps.sims.values()))
    line["host_inputs"] = "pinned, staged by device copies overlapping the kernels"
    mapped = [evsim.simulator_for(seq, m, event_capacity=cap, stream=ps.stream,
                                  tile_height=ps.tune[PASS_NAMES[m]]["tile_height"],
                                  host_inputs=evsim.SIM_HOST_MAPPED)
              for m in (0, 1) if PASS_NAMES[m] in ps.sims]
    line["mapped"] = measure(mapped)
    line["mapped"]["host_inputs"] = "pinned, read in place by the kernels"
    for sim in mapped:
        sim.close()
    return line


def main():
    args = parse()
    ws, rank, local = dist_setup(args) if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
