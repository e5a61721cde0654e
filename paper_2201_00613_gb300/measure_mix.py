"""Measure the batched mix and the request loop; prints one JSON line each.

  python -m paper_2201_00613_gb300.measure_mix [--requests N] [--no-tune]

Batched mix: 256 instances (triangle r 8-14, carpet r 4-8, Vicsek r 5-9,
Bernoulli(0.5), seed 5), autotuned tile levels and launch shape, 50 steps in
one captured graph; aggregate fractal cell-updates/s over CUDA events.
Request loop: Poisson arrivals (seed 6), type uniform, level uniform up to
triangle 18 / carpet 9 / Vicsek 12, steps uniform 10-500, at a rate set from
the measured mean work per request so that the offered load is about 80 % of
the batched throughput; p50/p99 latency and aggregate cell-updates/s.
"""
import argparse
import json
import statistics
import sys

import torch

from . import inputs as I
from .batch import MixedBatch, autotune
from .serve import RequestLoop


def batch_mix(tune=True):
    mix = I.batch_mix(5, 256)
    shape = autotune(mix) if tune else {"levels": None, "threads": 288, "ctas_per_sm": 0}
    with MixedBatch(mix, levels=shape["levels"], threads=shape["threads"],
                    ctas_per_sm=shape["ctas_per_sm"]) as mb:
        mb.run(50)  # capture + warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mb.run(50)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        return {"what": "batched_mix", "instances": len(mix), "cells": mb.cells, "steps": 50,
                "seconds": s, "cell_updates_per_s": mb.cells * 50 / s,
                "shape": {k: shape[k] for k in ("levels", "threads", "ctas_per_sm")}}


def request_loop(n, capacity, levels=None):
    proto = I.request_stream(seed=6, count=2000, rate_per_s=1.0)
    mean_work = statistics.mean(r.instance.fractal.cells(r.instance.r) * r.n_steps for r in proto)
    rate = 0.8 * capacity / mean_work
    reqs = I.request_stream(seed=6, count=n, rate_per_s=rate)
    loop = RequestLoop(max_slots=64, chunk=25, levels=levels)
    out = loop.run(reqs)
    loop.close()
    out.update({"what": "request_loop", "offered_rate_per_s": rate,
                "mean_work_cell_updates": mean_work})
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--requests", type=int, default=10000)
    p.add_argument("--no-tune", action="store_true")
    a = p.parse_args(argv)
    b = batch_mix(not a.no_tune)
    print(json.dumps(b), flush=True)
    print(json.dumps(request_loop(a.requests, b["cell_updates_per_s"], b["shape"]["levels"])),
          flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
