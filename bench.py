"""Benchmark: compact-fractal B3/S23 steps on the Sierpinski triangle, level 20.

One bench step = one run of the workload: 100 synchronous B3/S23 steps over
the 3,486,784,401-cell compact state (Bernoulli(0.5), seed 3), as launches of
the bit-sliced tile kernel that each advance several steps (for this fractal
24 launches of four steps and 2 of two; the intermediate steps stay in shared
memory), after one launch that writes the input's border records (the halo
of the first step).  The state (2 x 3.49 GB) is far larger than L2, so no
flush is needed between launches.  The roofline is that of the dominant
kernel (the four-step launches), timed alone as the difference of calls of
20 and of 10 such launches.

Printed (rank 0, one JSON line): value = fractal cell-updates/s over all
ranks; the roofline of the step kernel against the measured HBM copy
bandwidth; the end-to-end rate through the C ABI from and to pinned host
memory; the same-GPU bounding-box comparison at level 16; the integer-ALU
maps and per-cell step against their tensor-core (tcgen05) forms at level 20;
the block-level layouts at level 16; the von Neumann tiled step and fp32 heat
diffusion; the 256-instance batched mix (autotuned, 50 steps under a CUDA
graph) and the 10,000-request loop (Poisson arrivals at 80 % of the loop's
own saturated throughput, p50/p99 latency); the CPU oracle on a bounded
sample, on the level-10 workload and on the level-16 box; SM clocks sampled
during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl squeeze|reference]
                  [--requests N] [--no-serve] [--no-compare] [--no-cpu]
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
sys.path.insert(0, ROOT)

from paper_2201_00613_gb300 import inputs as I  # noqa: E402

WORKLOAD = I.TRIANGLE_R20
COMPARE = I.TRIANGLE_R16
METRIC = "cell-updates/s"
# the hot kernel's source: its device code and the host code that builds its program
STEP_KERNEL_SRC = [os.path.join(ROOT, "paper_2201_00613_gb300", "csrc", f)
                   for f in ("tile2d.cuh", "bitslice.cuh", "step_tiled.cu")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
CPU_SAMPLE_LEVEL = 14   # oracle sample: the level-14 top-left sub-replica of the r = 20 box
CPU_SAMPLE_STEPS = 800   # about 15 s of work on 16 cores


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="squeeze", choices=["squeeze", "reference"])
    p.add_argument("--no-compare", action="store_true", help="skip the level-16 BB comparison")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-serve", action="store_true",
                   help="skip the batched mix and the request loop")
    p.add_argument("--requests", type=int, default=10000, help="requests of the request loop")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def file_sha(paths):
    """sha256 (16 hex digits) of the concatenation of the files."""
    h = hashlib.sha256()
    for path in ([paths] if isinstance(paths, str) else paths):
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        if d.get("source_sha") != file_sha(STEP_KERNEL_SRC):
            return None
        return float(d["dram_bytes_per_launch_full"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _cpu_model():
    """CPU model from /proc/cpuinfo (model name on x86, implementer/part on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return None
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    parts = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1",
             "0xd8e": "Neoverse N3", "0xd84": "Neoverse V3"}
    if "CPU part" in fields:
        impl = {"0x41": "Arm"}.get(fields.get("CPU implementer", ""), fields.get("CPU implementer", ""))
        return ("%s %s (part %s)" % (impl, parts.get(fields["CPU part"], "core"), fields["CPU part"])).strip()
    return None


_R10_TIMER = """
import json, sys, time
sys.path.insert(0, %r)
import oracle
from paper_2201_00613_gb300 import inputs as I
w = I.TRIANGLE_R10
m = oracle.member_grid(w.fractal, w.r)
box = oracle.box_init(w.fractal, w.r, w.seed, I.p_q24(w.p))
t0 = time.perf_counter()
oracle.box_run(m, box, w.n_steps)
dt = time.perf_counter() - t0
print(json.dumps({"cells_per_s": w.fractal.cells(w.r) * w.n_steps / dt, "threads": oracle.threads()}))
"""


def oracle_r10_timing():
    """The oracle on the small triangle workload (r = 10, 100 steps), on one
    core and on all cores (separate processes: OpenMP fixes its thread count
    at start-up)."""
    out = {}
    for name, env in (("one_core", {"OMP_NUM_THREADS": "1"}), ("all_cores", {})):
        res = subprocess.run([sys.executable, "-c", _R10_TIMER % ROOT], capture_output=True,
                             text=True, env=dict(os.environ, **env), timeout=300)
        if res.returncode == 0 and res.stdout.strip():
            out[name] = json.loads(res.stdout.strip().splitlines()[-1])
    return out


_R16_TIMER = """
import json, sys, time
sys.path.insert(0, %r)
import oracle
from paper_2201_00613_gb300 import inputs as I
w = I.TRIANGLE_R16
steps = int(sys.argv[1])
m = oracle.member_grid(w.fractal, w.r)
box = oracle.box_init(w.fractal, w.r, w.seed, I.p_q24(w.p))
t0 = time.perf_counter()
oracle.box_run(m, box, steps)
dt = time.perf_counter() - t0
print(json.dumps({"cells_per_s": w.fractal.cells(w.r) * steps / dt, "steps": steps,
                  "seconds": dt, "threads": oracle.threads()}))
"""


def oracle_r16_timing():
    """The oracle on the level-16 workload's whole 65,536^2 box (13 GB of host
    memory): 10 steps on all cores, 2 steps on one core (separate processes)."""
    out = {}
    for name, env, steps in (("all_cores", {}, 10), ("one_core", {"OMP_NUM_THREADS": "1"}, 2)):
        res = subprocess.run([sys.executable, "-c", _R16_TIMER % ROOT, str(steps)],
                             capture_output=True, text=True, env=dict(os.environ, **env),
                             timeout=900)
        if res.returncode == 0 and res.stdout.strip():
            out[name] = json.loads(res.stdout.strip().splitlines()[-1])
        else:
            out[name] = {"error": (res.stderr or res.stdout)[-300:]}
    return out


def cpu_oracle_baseline(seconds_hint=True):
    """The oracle as it stands, on all host cores, on a bounded sample of the
    workload: the level-CPU_SAMPLE_LEVEL top-left sub-replica of the level-20
    box with the same seeded start, CPU_SAMPLE_STEPS box steps."""
    import oracle
    f, r = WORKLOAD.fractal, CPU_SAMPLE_LEVEL
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, WORKLOAD.seed, I.p_q24(WORKLOAD.p))
    t0 = time.perf_counter()
    oracle.box_run(m, box, CPU_SAMPLE_STEPS)
    dt = time.perf_counter() - t0
    cells = f.k ** r
    return {"value": cells * CPU_SAMPLE_STEPS / dt, "unit": METRIC, "cores": oracle.threads(),
            "kind": "oracle",
            "sample": "bounding-box oracle, top-left level-%d sub-replica of the level-20 triangle "
                      "(%d fractal cells, %d^2 box), same seed, %d steps, %.2f s"
                      % (r, cells, 2 ** r, CPU_SAMPLE_STEPS, dt)}


def run_reference(args, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_oracle_baseline()
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_oracle_baseline())
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    sample_s = float(cb["sample"].rsplit(", ", 1)[-1].rstrip(" s"))
    config = workload_config(None)
    config.update({"kernel": "cpu oracle (bounding box)", "sample": cb["sample"]})
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_s * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": config,
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(level, world=1):
    """The `config` object of both arms' JSON lines."""
    w = WORKLOAD
    return {"workload": w.name, "fractal": "sierpinski_triangle s=2 k=3 offsets (0,0),(1,0),(0,1)",
            "r": w.r, "cells": w.fractal.cells(w.r), "p_alive": w.p, "seed": w.seed,
            "ca_steps_per_step": w.n_steps, "kernel": "step_tiled", "tile_level": level,
            "l2": "inputs larger than L2 (2 x 3.49 GB)",
            "parallelism": "replicas" if world > 1 else "single"}


def replica_max(x, world, device):
    """Max of a per-rank number over all ranks (the slowest replica bounds the
    job); the ranks are independent replicas, this is the only collective."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells, ca_steps, bench_steps, ms_max, world):
    """Whole-job cell-updates/s: every replica steps `cells` cells `ca_steps`
    times per bench step; the job takes the slowest replica's time."""
    return world * cells * ca_steps * bench_steps / (ms_max / 1e3)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_2201_00613_gb300 as sq

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return replica_max(x, world, dev)

    w = WORKLOAD
    pq = I.p_q24(w.p)
    h = sq.Handle(w.fractal, w.r)
    cells = h.cells
    a = torch.empty(cells, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
    stream = torch.cuda.current_stream(dev)
    kind = sq.SQUEEZE_STEP_TILED
    level = sq.squeeze_tiled_level(h.h)

    # ---- device-resident timed region --------------------------------------
    for _ in range(args.warmup):
        sq.squeeze_step(h.h, a, b, w.n_steps, kind, stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            sq.squeeze_step(h.h, a, b, w.n_steps, kind, stream)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1))
    clocks = clk.summary()
    status = sq.squeeze_device_status(h.h)
    _, launches_per_step, by_steps = sq.squeeze_last_step_info(h.h)
    launches = args.steps * launches_per_step
    ms_per_step = ms / args.steps
    value = job_value(cells, w.n_steps, args.steps, ms, world)

    # ---- roofline of the dominant kernel (the launches of the most steps) ---
    # Its launches alone: calls of 20 and of 10 such launches, timed with CUDA
    # events on the stream they are launched on; every call also makes one
    # records-only launch, which the difference of the two removes.
    top = max(i for i in range(4) if by_steps[i])
    steps_per_launch = 1 << top

    def timed_calls(n_launches, reps=3):
        run = n_launches * steps_per_launch
        sq.squeeze_step(h.h, a, b, run, kind, stream)
        assert sq.squeeze_last_step_info(h.h)[2][top] == n_launches
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(reps):
            sq.squeeze_step(h.h, a, b, run, kind, stream)
        k1.record(stream)
        torch.cuda.synchronize()
        return k0.elapsed_time(k1) / 1e3 / reps

    launch_s = (timed_calls(20) - timed_calls(10)) / 10
    # Algorithmic bytes: 2 per cell-update (own state read once, new state
    # written once) times the cell-updates of one launch.
    algo_bytes = 2 * cells * steps_per_launch
    peak, peak_kind = peaks()
    achieved = algo_bytes / launch_s / 1e9
    traffic = traffic_per_launch()

    # ---- end to end through the C ABI from pinned host memory ---------------
    hin = torch.empty(cells, dtype=torch.uint8, pin_memory=True)
    hout = torch.empty(cells, dtype=torch.uint8, pin_memory=True)
    hin.copy_(a.cpu())
    e2e_steps = max(1, min(args.steps, 3))
    sq.squeeze_step_host(h.h, hin, hout, a, b, w.n_steps, kind, stream)  # warm
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sq.squeeze_step_host(h.h, hin, hout, a, b, w.n_steps, kind, stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * cells * w.n_steps * e2e_steps / e2e_s
    del hin, hout
    h.close()
    del a, b
    torch.cuda.empty_cache()

    # ---- same-GPU bounding box at level 16 ----------------------------------
    compare = maps = blocks = workloads = nbb3d = None
    if not args.no_compare:
        compare = bb_compare(sq, torch, dev, stream)
        maps = map_compare(sq, torch, dev, stream)
        blocks = block_compare(sq, torch, dev, stream)
        workloads = workload_compare(sq, torch, dev, stream)
        try:
            nbb3d = nbb3d_compare(sq, torch, dev, stream)
        except Exception as e:   # reported in the line, never fatal to it
            nbb3d = {"error": str(e)[:300]}

    mix = loop = None
    if not args.no_serve:
        mix = batch_mix_leg(sq, torch, dev, peaks()[0])
        if args.requests > 0 and world == 1:
            loop = request_loop_leg(args.requests, mix["shape"]["levels"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_baseline()
        cpu["cpu_model"] = _cpu_model()
        cpu["sierpinski_triangle_r10_100_steps"] = oracle_r10_timing()
        cpu["sierpinski_triangle_r16_box"] = oracle_r16_timing()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic",
            "config": workload_config(level, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": traffic, "algorithmic_bytes_per_launch": algo_bytes,
                         "steps_per_launch": steps_per_launch,
                         "state_bytes_per_launch": 2 * cells,
                         "state_gbs": 2 * cells / launch_s / 1e9,
                         "state_frac": 2 * cells / launch_s / 1e9 / peak,
                         "dram_gbs": traffic / launch_s / 1e9 if traffic else None,
                         "note": "algorithmic bytes: 2 per cell-update (the state read and "
                                 "written once per step); a launch advances steps_per_launch "
                                 "steps per pass of the state over HBM (state_gbs)",
                         "kernel": "step_tiled_kernel, B3/S23, 27-wide rows, %d steps per launch"
                                   % steps_per_launch,
                         "launches_by_steps_per_bench_step": {str(1 << i): by_steps[i]
                                                              for i in range(4) if by_steps[i]},
                         "avg_launch_ms": launch_s * 1e3},
            "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": cells,
                    "d2h_bytes_per_step": cells, "api": "squeeze_step_host",
                    "ca_steps_per_step": w.n_steps},
            "gpu_launches": launches,
            "clocks": clocks,
            "device_status": status,
            "bb_compare": compare,
            "map_compare": maps,
            "block_compare": blocks,
            "workload_compare": workloads,
            "nbb3d_compare": nbb3d,
            "batch_mix": mix,
            "request_loop": loop,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_mix_leg(sq, torch, dev, peak_gbs, steps=50):
    """The 256-instance mixed batch (triangle r 8-14, carpet r 4-8, Vicsek r
    5-9, Bernoulli(0.5), seed 5): autotuned tile levels and launch shape, then
    `steps` steps in one captured CUDA graph (one launch per tile-row
    instantiation and step), timed with CUDA events after a warm replay.  Two
    bytes per cell-update against the copy bandwidth (the 0.9 GB of states
    exceed L2)."""
    from paper_2201_00613_gb300.batch import MixedBatch, autotune
    mix = I.batch_mix(5, 256)
    t0 = time.perf_counter()
    shape = autotune(mix)
    tune_s = time.perf_counter() - t0
    with MixedBatch(mix, levels=shape["levels"], threads=shape["threads"],
                    ctas_per_sm=shape["ctas_per_sm"]) as mb:
        mb.run(steps)   # capture + warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mb.run(steps)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        rate = mb.cells * steps / sec
        status = max((abs(sq.squeeze_device_status(h.h)) for h in mb.handles), default=0)
        launches = sq.squeeze_batch_info(mb.batch)
        return {"workload": "batched mix, 256 instances, seed 5", "instances": len(mix),
                "cells": mb.cells, "steps": steps, "seconds": sec, "cell_updates_per_s": rate,
                "hbm_frac": 2 * rate / 1e9 / peak_gbs, "state_bytes": 2 * mb.cells,
                "shape": {k: shape[k] for k in ("levels", "threads", "ctas_per_sm")},
                "ctas_per_step": launches[0], "tuning_seconds": tune_s, "status": -status}


def request_loop_leg(n, levels, calibration=1500):
    """`n` requests (seed 6): type uniform over the mix, level uniform up to
    triangle 18 / carpet 9 / Vicsek 12, steps uniform 10-500, Poisson arrivals
    at a rate that offers 80 % of the loop's own saturated throughput
    (measured first on `calibration` requests of seed 7 that all arrive at
    once); continuous batching with admission by free HBM (64 slots, rounds of
    at most 25 steps)."""
    from paper_2201_00613_gb300.serve import RequestLoop
    proto = I.request_stream(seed=6, count=2000, rate_per_s=1.0)
    mean_work = statistics.mean(r.instance.fractal.cells(r.instance.r) * r.n_steps for r in proto)
    loop = RequestLoop(max_slots=64, chunk=25, levels=levels)
    sat = loop.run(I.request_stream(seed=7, count=calibration, rate_per_s=1e9))
    loop.close()
    capacity = sat["cell_updates_per_s"]
    rate = 0.8 * capacity / mean_work
    reqs = I.request_stream(seed=6, count=n, rate_per_s=rate)
    loop = RequestLoop(max_slots=64, chunk=25, levels=levels)
    out = loop.run(reqs)
    loop.close()
    out.update({"offered_rate_per_s": rate,
                "offered_load": "80 % of the loop's saturated throughput",
                "saturated_cell_updates_per_s": capacity,
                "saturated_requests": calibration, "mean_work_cell_updates": mean_work})
    return out


def bb_compare(sq, torch, dev, stream, steps=20):
    """Compact tiled step vs the bounding-box kernel and the lambda(omega)
    approach (compact threads over the expanded box) at level 16, same GPU.
    Compact state (86 MB) fits in L2, so L2 is flushed before every timed
    compact step; the box (2 x 4.29 GB) does not."""
    w = COMPARE
    pq = I.p_q24(w.p)
    h = sq.Handle(w.fractal, w.r)
    a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    for _ in range(3):
        sq.squeeze_step(h.h, a, b, 2, sq.SQUEEZE_STEP_TILED, stream)
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED, stream)
        s1.record(stream)
        torch.cuda.synchronize()
        tot += s0.elapsed_time(s1)
        a, b = b, a
    compact = h.cells * steps / (tot / 1e3)
    # resident (no flush) for context
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    sq.squeeze_step(h.h, a, b, 200, sq.SQUEEZE_STEP_TILED, stream)
    r1.record(stream)
    torch.cuda.synchronize()
    resident = h.cells * 200 / (r0.elapsed_time(r1) / 1e3)
    del flush
    g0 = torch.empty(h.side * h.side, dtype=torch.uint8, device=dev)
    g1 = torch.empty_like(g0)
    sq.squeeze_bb_init(h.h, g0, w.seed, pq)
    sq.squeeze_bb_step(h.h, g0, g1, 2, stream)
    torch.cuda.synchronize()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    sq.squeeze_bb_step(h.h, g0, g1, steps, stream)
    q1.record(stream)
    torch.cuda.synchronize()
    bb_ms = q0.elapsed_time(q1)
    bb = h.cells * steps / (bb_ms / 1e3)
    bb_gbs = 2 * h.side * h.side * steps / (bb_ms / 1e3) / 1e9
    # the lambda(omega) approach on the same boxes (compact threads, expanded memory)
    g1.copy_(g0)
    sq.squeeze_lambda_step(h.h, g0, g1, 2, stream)
    torch.cuda.synchronize()
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    sq.squeeze_lambda_step(h.h, g0, g1, steps, stream)
    l1.record(stream)
    torch.cuda.synchronize()
    lam = h.cells * steps / (l0.elapsed_time(l1) / 1e3)
    peak = peaks()[0]
    compact_frac = 2 * compact / 1e9 / peak     # one step per launch: 2 bytes per cell-update
    bb_frac = bb_gbs / peak
    out = {"workload": w.name, "r": w.r, "steps": steps,
           "compact_cell_updates_per_s": compact,
           "compact_l2": "one step per launch, L2 flushed before every launch",
           "compact_hbm_frac": compact_frac,
           "compact_resident_cell_updates_per_s": resident,
           "compact_resident": "200 steps in one call (the default steps per launch, state in L2)",
           "bb_cell_updates_per_s": bb, "bb_box_gbs": bb_gbs, "bb_hbm_frac": bb_frac,
           "lambda_approach_cell_updates_per_s": lam,
           "speedup_compact_over_bb": compact / bb,
           "speedup_compact_resident_over_bb": resident / bb,
           "speedup_compact_over_bb_at_equal_hbm_frac": compact / bb * bb_frac / compact_frac,
           "speedup_compact_over_lambda_approach": compact / lam,
           "memory_bytes": {"compact": 2 * h.cells, "bb": 2 * h.side * h.side}}
    h.close()
    del g0, g1, a, b
    torch.cuda.empty_cache()
    return out


def workload_compare(sq, torch, dev, stream):
    """Other neighbourhood workloads: the tiled step over the von Neumann
    neighbourhood at level 20; fp32 heat diffusion and Ising Metropolis sweeps
    (per-cell lambda / nu) at level 16."""
    def timed(fn, steps):
        fn(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3
    out = {"unit": "cell-updates/s"}
    w = WORKLOAD
    with sq.Handle(w.fractal, w.r) as h:
        sq.squeeze_set_neighbourhood(h.h, sq.SQUEEZE_VON_NEUMANN)
        a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, w.seed, I.p_q24(w.p))
        t = timed(lambda n: sq.squeeze_step(h.h, a, b, n, sq.SQUEEZE_STEP_TILED, stream), 10)
        out["von_neumann_tiled_" + w.name] = h.cells * 10 / t
        del a, b
    c = COMPARE
    with sq.Handle(c.fractal, c.r) as h:
        sq.squeeze_set_neighbourhood(h.h, sq.SQUEEZE_VON_NEUMANN)
        gen = torch.Generator(device=dev)
        gen.manual_seed(c.seed)
        u = torch.rand(h.cells, generator=gen, device=dev)
        v = torch.empty_like(u)
        t = timed(lambda n: sq.squeeze_heat_step(h.h, u, v, n, 0.25, stream), 10)
        out["heat_fp32_von_neumann_" + c.name] = h.cells * 10 / t
        del u, v
        spins = torch.empty(h.cells, dtype=torch.uint8, device=dev)
        sq.squeeze_init_bernoulli(h.h, spins, c.seed, I.p_q24(0.5))
        t = timed(lambda n: sq.squeeze_ising_sweep(h.h, spins, n, n, 2.269, stream), 10)
        out["ising_sweep_von_neumann_" + c.name] = h.cells * 10 / t
        out["status"] = sq.squeeze_device_status(h.h)
    torch.cuda.empty_cache()
    return out


def nbb3d_compare(sq, torch, dev, stream, steps=4):
    """Three-dimensional fractals (26 neighbours, B5/S45): the Sierpinski
    tetrahedron at level 15 (1.07e9 cells) with the bit-sliced tile kernel and
    with the per-cell kernel, the Menger sponge at level 7 (1.28e9 cells, rows
    of 20 cells: per-cell kernel only); hbm_frac counts two bytes per
    cell-update against the copy bandwidth."""
    out = {"unit": "cell-updates/s", "steps": steps, "rule": "B5/S45, 26 neighbours"}
    for f, r, kernel in ((I.TETRA, 15, "tiled"), (I.TETRA, 15, "per_cell"), (I.MENGER, 7, "auto")):
        with sq.Handle3(f, r) as h:
            if kernel == "per_cell":
                sq.squeeze_3d_set_tiled_level(h.h, 0)
            a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
            b = torch.empty_like(a)
            sq.squeeze_3d_init_bernoulli(h.h, a, 3, I.p_q24(0.3), stream)
            sq.squeeze_3d_step(h.h, a, b, 2, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sq.squeeze_3d_step(h.h, a, b, steps, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            rate = h.cells * steps / t
            level = sq.squeeze_3d_tiled_level(h.h)
            out["%s_r%d_%s" % (f.name, r, "tiled" if level else "per_cell")] = {
                "cells": h.cells, "ms_per_step": 1e3 * t / steps, "cell_updates_per_s": rate,
                "hbm_frac": 2 * rate / 1e9 / peaks()[0], "tile_level": level,
                "status": sq.squeeze_3d_device_status(h.h)}
            del a, b
    torch.cuda.empty_cache()
    return out


def block_compare(sq, torch, dev, stream, steps=20):
    """Block-level layouts (rho x rho micro-boxes, rho = 2^b) at level 16: bytes
    per state and cell-updates/s of the block step, next to the compact layout."""
    w = COMPARE
    out = {"workload": w.name, "r": w.r, "steps": steps, "unit": "cell-updates/s", "levels": []}
    with sq.Handle(w.fractal, w.r) as h:
        for b in range(0, 6):
            nbytes = sq.squeeze_block_bytes(h.h, b)
            x = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            y = torch.empty_like(x)
            sq.squeeze_block_init(h.h, b, x, w.seed, I.p_q24(w.p), stream)
            sq.squeeze_block_step(h.h, b, x, y, 2, stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sq.squeeze_block_step(h.h, b, x, y, steps, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            out["levels"].append({"rho": 2 ** b, "bytes_per_state": nbytes,
                                  "cell_updates_per_s": h.cells * steps / (e0.elapsed_time(e1) / 1e3)})
            del x, y
        out["status"] = sq.squeeze_device_status(h.h)
    torch.cuda.empty_cache()
    return out


def map_compare(sq, torch, dev, stream, points=1 << 25):
    """Integer-ALU maps against the tensor-core (tcgen05 kind::f16) maps at the
    benchmark level: lambda and nu over `points` seeded compact indices, and
    one per-cell step of each kind over the whole state, checked bit for bit."""
    w = WORKLOAD
    h = sq.Handle(w.fractal, w.r)
    gen = torch.Generator(device=dev)
    gen.manual_seed(I.R20_SAMPLE_SEED)
    om = torch.randint(0, h.cells, (points,), generator=gen, dtype=torch.int64, device=dev)
    xy = {k: torch.empty((points, 2), dtype=torch.int32, device=dev) for k in ("alu", "tc")}
    back = {k: torch.empty(points, dtype=torch.int64, device=dev) for k in ("alu", "tc")}
    TC = sq.SQUEEZE_MAP_TC_BF16

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    rate = {"lambda": {}, "nu": {}, "step": {}}
    rate["lambda"]["alu"] = points / timed(lambda: sq.squeeze_lambda(h.h, om, xy["alu"], points, stream))
    rate["lambda"]["tc"] = points / timed(lambda: sq.squeeze_map_tc(h.h, 0, om, xy["tc"], points, TC, stream))
    rate["nu"]["alu"] = points / timed(lambda: sq.squeeze_nu(h.h, xy["alu"], back["alu"], points, stream))
    rate["nu"]["tc"] = points / timed(lambda: sq.squeeze_map_tc(h.h, 1, xy["alu"], back["tc"], points, TC, stream))
    maps_exact = (torch.equal(xy["alu"], xy["tc"]) and torch.equal(back["alu"], back["tc"])
                  and torch.equal(back["alu"], om))
    del om, xy, back
    a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
    sq.squeeze_init_bernoulli(h.h, a, w.seed, I.p_q24(w.p))
    outs = {}
    for name, kind in (("alu", sq.SQUEEZE_MAP_ALU), ("tc", TC), ("tiled", sq.SQUEEZE_STEP_TILED)):
        outs[name] = torch.empty_like(a)
        t = timed(lambda: sq.squeeze_step(h.h, a, outs[name], 1, kind, stream), reps=1)
        rate["step"][name] = h.cells / t
    step_exact = torch.equal(outs["alu"], outs["tc"]) and torch.equal(outs["alu"], outs["tiled"])
    status = sq.squeeze_device_status(h.h)
    h.close()
    del a, outs
    torch.cuda.empty_cache()
    return {"workload": w.name, "points": points, "unit": "points/s (steps: cell-updates/s)",
            "lambda": rate["lambda"], "nu": rate["nu"], "step": rate["step"],
            "bit_exact": bool(maps_exact and step_exact and status == 0),
            "tc": "tcgen05.mma kind::f16, bf16 digits x radix-256 weight limbs, fp32 accumulate; "
                  "column sums < 2^21"}


if __name__ == "__main__":
    main()
