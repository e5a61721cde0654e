"""Batched mixed-fractal runs over the C ABI (squeeze_batch_*), plus the tuner.

A `MixedBatch` owns one handle and one pair of device state buffers per
instance (allocated with torch), seeds every instance's Bernoulli start on
the device, and steps all of them together through one batch object: one
persistent launch per CA step, the steps captured in a CUDA graph.

`autotune` picks the tile level per fractal type, the CTA size (0: each tile
instantiation's own) and the CTAs per SM for a given mix by timing candidate
batches, and caches the choice in
``_build/autotune.json`` keyed by the mix, the device name and its SM count.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from . import _lib as sq
from . import inputs as I

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


class MixedBatch:
    """Instances (fractal, r, seed, p) stepped together on one device."""

    def __init__(self, instances, device="cuda", levels=None, threads=0, ctas_per_sm=0,
                 use_graph=True, init=True):
        self.instances = list(instances)
        self.device = torch.device(device)
        self.handles, self.buf0, self.buf1 = [], [], []
        for inst in self.instances:
            h = sq.Handle(inst.fractal, inst.r)
            if levels and inst.fractal.name in levels:
                lvl = min(levels[inst.fractal.name], inst.r)
                if lvl >= 1:
                    try:
                        sq.squeeze_set_tiled_level(h.h, lvl)
                    except sq.SqueezeError:
                        pass  # keep the default level for this instance
            a = torch.empty(h.cells, dtype=torch.uint8, device=self.device)
            b = torch.empty_like(a)
            if init:
                sq.squeeze_init_bernoulli(h.h, a, inst.seed, I.p_q24(inst.p))
            self.handles.append(h)
            self.buf0.append(a)
            self.buf1.append(b)
        self.batch = None
        try:
            self.batch = sq.squeeze_batch_create(
                [(h.h, a, b) for h, a, b in zip(self.handles, self.buf0, self.buf1)])
            if threads or ctas_per_sm or not use_graph:
                sq.squeeze_batch_configure(self.batch, threads, ctas_per_sm, use_graph)
        except Exception:
            self.close()
            raise
        self.steps_done = 0

    @property
    def cells(self) -> int:
        return sum(h.cells for h in self.handles)

    def run(self, n_steps: int, stream=None):
        sq.squeeze_batch_run(self.batch, n_steps, stream)
        self.steps_done += n_steps

    def state(self, i: int):
        """Current state of instance i (the buffer the last step wrote)."""
        return self.buf1[i] if self.steps_done % 2 else self.buf0[i]

    def close(self):
        if self.batch:
            sq.squeeze_batch_destroy(self.batch)
            self.batch = None
        for h in self.handles:
            h.close()
        self.handles = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _signature(instances) -> str:
    key = ",".join("%s:%d" % (i.fractal.name, i.r) for i in instances)
    return hashlib.sha256(key.encode()).hexdigest()[:16]


def _device_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def time_config(instances, levels, threads, ctas_per_sm, steps=6) -> float:
    """Seconds per batched step of one configuration (after a warm-up); inf when
    the library cannot run that configuration (UNSUPPORTED)."""
    try:
        mb = MixedBatch(instances, levels=levels, threads=threads, ctas_per_sm=ctas_per_sm)
    except sq.SqueezeError as e:
        if e.code != sq.SQUEEZE_ERR_UNSUPPORTED:
            raise
        return float("inf")
    with mb:
        mb.run(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        mb.run(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps


def _level_candidates(f, max_r):
    """The three largest tile levels the library accepts for fractal f."""
    out = []
    for L in range(1, max_r + 1):
        width = f.k ** ((L + 1) // 2)   # tile-row width: one slot word, or exactly two
        if width > 64 or (32 < width < 64):
            break
        with sq.Handle(f, L) as h:      # the program's size depends on f and L only
            try:
                sq.squeeze_set_tiled_level(h.h, L)
            except sq.SqueezeError:
                break
        out.append(L)
    return out[-3:]


def autotune(instances, use_cache=True, log=None) -> dict:
    """Coordinate search over tile level per type, CTA size and CTAs per SM."""
    sig, dev = _signature(instances), _device_key()
    cache = {}
    if use_cache and os.path.exists(_CACHE):
        try:
            with open(_CACHE) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    key = sig + "@" + dev
    if use_cache and key in cache:
        return cache[key]
    types = {}
    for inst in instances:
        types.setdefault(inst.fractal.name, (inst.fractal, 0))
        f, r = types[inst.fractal.name]
        types[inst.fractal.name] = (f, max(r, inst.r))
    best = {"levels": {}, "threads": 0, "ctas_per_sm": 0}
    t0 = time.time()
    best_t = time_config(instances, None, 0, 0)
    trials = [(dict(best), best_t)]
    for name, (f, max_r) in types.items():
        for L in _level_candidates(f, max_r):
            levels = dict(best["levels"])
            levels[name] = L
            t = time_config(instances, levels, best["threads"], best["ctas_per_sm"])
            trials.append(({"levels": levels, "threads": best["threads"],
                            "ctas_per_sm": best["ctas_per_sm"]}, t))
            if t < best_t:
                best_t, best = t, {"levels": levels, "threads": best["threads"],
                                   "ctas_per_sm": best["ctas_per_sm"]}
    for threads in (0, 192, 256, 288):    # 0: each instantiation's own CTA size
        for ctas in (0, 2, 3):
            if (threads, ctas) == (0, 0):   # the shape the level search already timed
                continue
            t = time_config(instances, best["levels"], threads, ctas)
            trials.append(({"levels": best["levels"], "threads": threads, "ctas_per_sm": ctas}, t))
            if t < best_t:
                best_t, best = t, {"levels": best["levels"], "threads": threads, "ctas_per_sm": ctas}
    result = dict(best)
    result["seconds_per_step"] = best_t
    result["trials"] = len(trials)
    result["tuning_seconds"] = time.time() - t0
    if log:
        log(result)
    if use_cache:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        cache[key] = result
        tmp = "%s.tmp%d" % (_CACHE, os.getpid())
        with open(tmp, "w") as f:        # replaced whole: readers never see a partial file
            json.dump(cache, f, indent=1)
        os.replace(tmp, _CACHE)
    return result
