"""A fixed workload for external profilers (ncu): set-up on a cube box, then
repeated stiffness actions K.u (Alg. 2).

    python -m paper_2403_19854_gb300.profile_target --box 256 --dtype f32 --degree 1 --reps 4

Box sides a x b x c (``--box 256x256x128``) embed the cube domain of the smallest
side in a larger box, which keeps the kernels of the long axes while holding less
device memory.  Prints the device memory held and a checksum of the result.
"""
from __future__ import annotations

import argparse


def main(argv=None):
    import torch

    from . import rk
    from . import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("--box", default="128")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--degree", type=int, default=1, choices=[1, 2])
    ap.add_argument("--reps", type=int, default=4)
    a = ap.parse_args(argv)
    box = tuple(int(v) for v in a.box.split("x"))
    if len(box) == 1:
        box = box * 3
    at = 2.5 if a.degree == 1 else 3.0
    p = W.cube_problem(min(box), at, a.degree, "zero")
    if box != p.n:
        p = W.embed(p, box)
    dev = torch.device("cuda:0")
    H = rk.Handle.from_problem(p, device=dev)
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    g = torch.Generator(device=dev)
    g.manual_seed(20240328)
    x = torch.rand(p.nbox, dtype=dt, device=dev, generator=g)
    y = torch.empty_like(x)
    for _ in range(a.reps):
        H.apply_K(x, y)
    torch.cuda.synchronize()
    print(f"box {box} degree {a.degree} {a.dtype}: {a.reps} K.u, checksum {float(y.abs().sum()):.6e}, "
          f"device memory {torch.cuda.mem_get_info()[1] - torch.cuda.mem_get_info()[0]:.3e} B in use")
    H.close()


if __name__ == "__main__":
    main()
