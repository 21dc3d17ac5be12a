"""Run one configuration's operator applies, for profiling a kernel in
isolation (``ncu`` captures a named kernel of this process).

    python -m paper_1809_00845_gb300.workloads ellipsoid --n 128 --layer single --reps 5
    python -m paper_1809_00845_gb300.workloads star --n 4096 --layer system --reps 20 [--three-pass]

Workloads (seeded synthetic inputs, the bench's geometry recipes):
  star       2D Laplace, r = 0.3 (1 + 0.3 cos 5 theta), mixed boundary conditions
  panels     the same star as flat panels (accuracy mode, order 3, near radius 5), mixed conditions
  circle     2D Laplace, radius 0.35
  ellipsoid  3D Laplace, semi-axes (0.4, 0.3, 0.2)
  cube       3D Kelvin (nu = 0.3, mu = 1), side 0.5 on node planes
Densities are N(0, 1); every apply runs on the current stream and the script
synchronises once at the end and prints the mean time per apply.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_plan(workload: str, n: int, precision: str, flags: int = 0):
    from paper_1809_00845_gb300 import inputs as I
    from paper_1809_00845_gb300.bem import Plan
    if workload == "star":
        b = I.star_boundary(n)
        p = Plan.from_boundary(b, "laplace2d", precision, flags=flags)
        p.set_bc(I.mixed_bc_theta(b), 0.5)
    elif workload == "circle":
        b = I.circle_boundary(n, 0.35)
        p = Plan.from_boundary(b, "laplace2d", precision, flags=flags)
        p.set_bc(I.mixed_bc_theta(b), 0.5)
    elif workload == "panels":
        b = I.curve_panels(n, I.star_curve(0.3, 0.3, 5))
        p = Plan.from_panel_boundary(b, precision, 3, 5)
        p.set_bc((np.asarray(b.param) >= np.pi).astype(np.uint8), 0.5)
    elif workload == "ellipsoid":
        b = I.ellipsoid_boundary(n)
        p = Plan.from_boundary(b, "laplace3d", precision, flags=flags)
        p.set_bc(np.zeros(b.nb, np.uint8), 0.5)
    elif workload == "cube":
        b = I.cube_boundary(n)
        p = Plan.from_boundary(b, "kelvin3d", precision, flags=flags)
        p.set_bc(np.zeros(3 * b.nb, np.uint8), 0.5)
    else:
        raise ValueError(f"unknown workload {workload}")
    return b, p


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("workload", choices=["star", "panels", "circle", "ellipsoid", "cube"])
    ap.add_argument("--n", type=int, default=None, help="grid cells per axis (default: the bench's size)")
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--layer", default="single", choices=["single", "double", "system"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--three-pass", action="store_true", help="2D FP32: BEM_PLAN_THREE_PASS")
    args = ap.parse_args(argv)
    import torch
    from paper_1809_00845_gb300 import build
    build.build()
    n = args.n or {"star": 4096, "panels": 4096, "circle": 128, "ellipsoid": 256, "cube": 128}[args.workload]
    from paper_1809_00845_gb300.bem import BEM_PLAN_THREE_PASS
    b, p = make_plan(args.workload, n, args.precision, BEM_PLAN_THREE_PASS if args.three_pass else 0)
    dt = torch.float32 if args.precision in ("f32", "tc_bf16x3", "tc_f16x3") else torch.float64
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x = torch.randn(p.nb * p.ncomp, generator=g, device="cuda", dtype=torch.float64).to(dt)
    y = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        p.apply(args.layer, x, y)
    e1.record()
    torch.cuda.synchronize()
    print(f"{args.workload} n={n} nb={p.nb} {args.precision} {args.layer}: "
          f"{e0.elapsed_time(e1) / max(1, args.reps):.3f} ms per apply over {args.reps}")
    p.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
