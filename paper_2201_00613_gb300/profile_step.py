"""Run the compact step on one level for profiler captures.

  python -m paper_2201_00613_gb300.profile_step --level 18 --steps 3 [--kind tiled|alu|tc]
      [--fractal triangle|carpet|vicsek|menger|tetrahedron] [--maps N]
  python -m paper_2201_00613_gb300.profile_step --batch-mix --steps 12
  python -m paper_2201_00613_gb300.profile_step --bb --level 15 --steps 3

Initialises the seeded Bernoulli(0.5) state of the fractal at the given level
and runs `steps` steps, one kernel launch per step (the three-dimensional
fractals take the per-cell 3-D step; --kind and --maps apply to the planar
ones).  --batch-mix steps the 256-instance mixed batch (default launch
shape, no tuning) `steps` times through its CUDA graph instead; --bb runs
the same-GPU bounding-box step on the level's expanded box.  Used with
ncu on a case that is larger than L2 but small enough for a multi-pass
capture.
"""
import argparse
import sys

import torch

from . import _lib as sq
from . import inputs as I

KINDS = {"tiled": sq.SQUEEZE_STEP_TILED, "alu": sq.SQUEEZE_MAP_ALU, "tc": sq.SQUEEZE_MAP_TC_BF16}
FRACTALS = {"triangle": I.TRIANGLE, "carpet": I.CARPET, "vicsek": I.VICSEK}
FRACTALS_3D = {"menger": I.MENGER, "tetrahedron": I.TETRA}


def run_3d(f, level, steps):
    with sq.Handle3(f, level) as h:
        s0 = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        s1 = torch.empty_like(s0)
        sq.squeeze_3d_init_bernoulli(h.h, s0, 3, I.p_q24(0.5))
        sq.squeeze_3d_step(h.h, s0, s1, steps)
        torch.cuda.synchronize()
        st = sq.squeeze_3d_device_status(h.h)
        print("3-D %s level %d cells %d steps %d status %d" % (f.name, level, h.cells, steps, st))
        return 0 if st == 0 else 1


def run_batch_mix(steps):
    from .batch import MixedBatch
    with MixedBatch(I.batch_mix(5, 256)) as mb:
        mb.run(steps)
        torch.cuda.synchronize()
        st = [sq.squeeze_device_status(h.h) for h in mb.handles]
        grid, threads, smem = sq.squeeze_batch_info(mb.batch)
        print("batched mix: %d instances, %d cells, %d steps, %d CTAs per step, status %d"
              % (len(mb.handles), mb.cells, steps, grid, min(st)))
        return 0 if not any(st) else 1


def run_bb(f, level, steps):
    with sq.Handle(f, level) as h:
        g0 = torch.empty(h.side * h.side, dtype=torch.uint8, device="cuda")
        g1 = torch.empty_like(g0)
        sq.squeeze_bb_init(h.h, g0, 3, I.p_q24(0.5))
        sq.squeeze_bb_step(h.h, g0, g1, steps)
        torch.cuda.synchronize()
        st = sq.squeeze_device_status(h.h)
        print("bounding box level %d side %d steps %d status %d" % (level, h.side, steps, st))
        return 0 if st == 0 else 1


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--level", type=int, default=18)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--kind", default="tiled", choices=sorted(KINDS))
    p.add_argument("--fractal", default="triangle", choices=sorted(FRACTALS) + sorted(FRACTALS_3D))
    p.add_argument("--maps", type=int, default=0,
                   help="first run lambda then nu over this many seeded points (with --kind tc "
                        "on the tensor cores, else on the ALU)")
    p.add_argument("--batch-mix", action="store_true",
                   help="step the 256-instance mixed batch instead of one fractal")
    p.add_argument("--bb", action="store_true", help="the bounding-box step instead")
    a = p.parse_args(argv)
    if a.batch_mix:
        return run_batch_mix(a.steps)
    if a.bb:
        return run_bb(FRACTALS[a.fractal], a.level, a.steps)
    if a.fractal in FRACTALS_3D:
        return run_3d(FRACTALS_3D[a.fractal], a.level, a.steps)
    f = FRACTALS[a.fractal]
    with sq.Handle(f, a.level) as h:
        if a.maps:
            gen = torch.Generator(device="cuda")
            gen.manual_seed(I.R20_SAMPLE_SEED)
            om = torch.randint(0, h.cells, (a.maps,), generator=gen, dtype=torch.int64, device="cuda")
            xy = torch.empty((a.maps, 2), dtype=torch.int32, device="cuda")
            back = torch.empty_like(om)
            if a.kind == "tc":
                sq.squeeze_map_tc(h.h, 0, om, xy, a.maps, sq.SQUEEZE_MAP_TC_BF16)
                sq.squeeze_map_tc(h.h, 1, xy, back, a.maps, sq.SQUEEZE_MAP_TC_BF16)
            else:
                sq.squeeze_lambda(h.h, om, xy, a.maps)
                sq.squeeze_nu(h.h, xy, back, a.maps)
            torch.cuda.synchronize()
            if not torch.equal(back, om):
                print("nu(lambda(omega)) != omega")
                return 1
        s0 = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        s1 = torch.empty_like(s0)
        sq.squeeze_init_bernoulli(h.h, s0, 3, I.p_q24(0.5))
        sq.squeeze_step(h.h, s0, s1, a.steps, KINDS[a.kind])
        torch.cuda.synchronize()
        st = sq.squeeze_device_status(h.h)
        print("level %d cells %d steps %d kind %s status %d" % (a.level, h.cells, a.steps, a.kind, st))
        return 0 if st == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
