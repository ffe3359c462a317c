"""Padded box sides for uneven domains, and the replacement settings of the mixed
solve for a given problem, chosen by measurement.

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


# Residual-replacement settings of the mixed solve (inner_tol, check_every): the
# FP32 recurrence is replaced by the true FP64 residual each time it has dropped
# by inner_tol, checked every check_every iterations.  Which setting needs the
# fewest iterations depends on the problem, irregularly (a replacement resets the
# rounding the FP32 recurrence has gathered), so it is measured.
MIXED_CANDIDATES = ((0.1, 25), (0.5, 10), (0.3, 10))


def best_mixed_opts(handle, r, g, tol=1e-10, candidates=MIXED_CANDIDATES, precond="none"):
    """Time one mixed solve of (r, g) on handle per candidate (inner_tol,
    check_every) and return (inner_tol, check_every, {candidate: (seconds,
    iterations, status)}).  A candidate may use at most twice the iterations of
    the first one; one that does not reach tol is not chosen."""
    import time

    import torch
    timings = {}
    best, best_t, cap = None, None, None
    for itol, ce in candidates:
        kw = dict(precision="mixed", tol=tol, inner_tol=itol, check_every=ce, precond=precond)
        if cap is not None:
            kw["max_iter"] = cap
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, info = handle.solve(r, g, raise_on_error=False, **kw)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        timings[f"{itol}/{ce}"] = (t, info["iterations"], info["status"])
        if cap is None:
            cap = 2 * max(info["iterations"], 1)
        if info["status"] == 0 and (best_t is None or t < best_t):
            best, best_t = (itol, ce), t
    if best is None:
        best = candidates[0]
    return best[0], best[1], timings
