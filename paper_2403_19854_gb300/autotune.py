"""Padded box sides for uneven domains, chosen by measurement.

A domain of side S can be solved in any built FFT box side S' >= S (the extra
nodes lie outside the domain, chi = 0).  For each candidate S' this module times
the FP32 stiffness action on an S'^3 box once (per basis degree), caches the
result in a JSON file beside the built library, and picks the side with the
smallest measured time.  The radix schedule of a side is fixed by the build, so
choosing S' chooses the FFT tile shapes.
"""
from __future__ import annotations

import json
import os

from . import rk
from . import workloads as W

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def built_sides(lo=8, hi=512):
    return [n for n in range(lo, hi + 1) if n % 2 == 0 and rk.supported_length(n)]


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def measure(side, degree, reps=10, device="cuda:0"):
    """Mean ms of one FP32 K.u on a side^3 box (cube domain), timed with CUDA events."""
    import torch
    a = 2.5 if degree == 1 else 3.0
    p = W.cube_problem(side, a, degree, "zero")
    H = rk.Handle.from_problem(p, device=torch.device(device))
    x = torch.rand(p.nbox, dtype=torch.float32, device=device)
    y = torch.empty_like(x)
    for _ in range(3):
        H.apply_K(x, y)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        H.apply_K(x, y)
    e.record()
    torch.cuda.synchronize()
    H.close()
    return s.elapsed_time(e) / reps


def best_side(S, degree, max_candidates=3):
    """The built side S' >= S with the smallest measured K.u time (cached)."""
    cache = _load()
    cands = [n for n in built_sides() if n >= S][:max_candidates]
    if not cands:
        raise ValueError(f"no built box side >= {S}")
    best, best_t = None, None
    changed = False
    for n in cands:
        key = f"{n}x{n}x{n}/f32/s{4 if degree == 1 else 10}"
        if key not in cache:
            cache[key] = measure(n, degree)
            changed = True
        if best_t is None or cache[key] < best_t:
            best, best_t = n, cache[key]
    if changed:
        _save(cache)
    return best
