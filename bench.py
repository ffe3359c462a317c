#!/usr/bin/env python
"""FC-RKPM benchmark: K.u throughput and time-to-solve of the 3D Poisson unit-cube
problem (linear basis, a = 2.5h, manufactured solution sin(pi x) sin(pi y) sin(pi z))
on a 256^3 periodic box (254^3 domain nodes).

One step = the whole solve path on inputs resident in HBM: rk_setup (kernel tables,
FP64 moment convolutions, per-node M^{-1} -> b; Alg. 1) + f^r (Alg. 4) + CG with FP32
K.u inside FP64 iterative refinement (Alg. 2, 5) to the requested FP64 residual +
u^h (Alg. 3).  value = domain DOF x K.u applications / second over the timed steps.

Also reported: the same path through the C ABI with pinned host buffers (e2e), the
plain FP64 GPU solve of the same problem (time-to-solve, iterations, agreement),
isolated K.u rates, the dominant kernel's HBM roofline from live CUDA-event timing,
and the FP64 oracle timed on the host (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own replica (independent problems, weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "K·u DOF/s and time-to-solve at 256³, FP32-mixed vs FP64 GPU at 1e-9 rel L2"
UNIT = "DOF/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_over_ranks(ms, units, world, device):
    """Whole-job figures of independent replicas: the slowest rank's time and the
    units (DOF x K.u applications) of all ranks.  Returns (max ms, total units)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------- oracle
def oracle_kd_rate(n_box=64, a_tilde=2.5, reps=3):
    """FP64 oracle matrix-free K.d (neighbour loops on all host threads) on a bounded
    cube sample; returns (DOF/s, sample description, seconds, threads)."""
    from oracle.oracle import Oracle, threads
    from paper_2403_19854_gb300 import workloads as W
    p = W.cube_problem(n_box, a_tilde, 1, "sin")
    t0 = time.perf_counter()
    o = Oracle(p.n, p.h, a_tilde, 1, p.chi)
    tb = time.perf_counter() - t0
    d = W.random_field(p.nbox, 1) * p.chi
    o.apply_K(p.V, d)
    t0 = time.perf_counter()
    for _ in range(reps):
        o.apply_K(p.V, d)
    dt = (time.perf_counter() - t0) / reps
    nt = threads()
    desc = (f"oracle matrix-free K.d (FP64 neighbour loops, {nt} host threads) on the {n_box}^3-box unit cube "
            f"({p.n_omega} DOF, a=2.5h, linear), mean of {reps} after 1 warm-up; shape-function build "
            f"{tb:.2f} s excluded")
    return p.n_omega / dt, desc, dt, nt


def oracle_timings():
    """The traditional method's other costs on the host (all threads), each on the
    largest cube the host handles in seconds: moment matrices, M^{-1} and shape
    functions (64^3 box), CSR assembly of K (Eq. 26) and one CSR product (48^3),
    and the full Dirichlet solve (assembly, f^r, CG on the CSR to 1e-10; 32^3)."""
    from oracle.oracle import Oracle, threads
    from paper_2403_19854_gb300 import workloads as W
    out = {"threads": threads()}
    p = W.cube_problem(64, 2.5, 1, "sin")
    t0 = time.perf_counter()
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    out["moments_Minv_shape_functions_64"] = {"s": time.perf_counter() - t0, "dof": p.n_omega}
    del o
    p = W.cube_problem(48, 2.5, 1, "sin")
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    t0 = time.perf_counter()
    nnz = o.assemble_K(p.V)
    ta = time.perf_counter() - t0
    x = W.random_field(p.nbox, 2) * p.chi
    o.spmv(x)
    t0 = time.perf_counter()
    for _ in range(3):
        o.spmv(x)
    out["assembly_48"] = {"s": ta, "dof": p.n_omega, "nnz": nnz}
    out["csr_spmv_48"] = {"s": (time.perf_counter() - t0) / 3, "dof": p.n_omega, "nnz": nnz}
    del o
    p = W.cube_problem(32, 2.5, 1, "sin")
    o = Oracle(p.n, p.h, 2.5, 1, p.chi)
    t0 = time.perf_counter()
    _, info = o.solve(p.V, p.chi_gamma, p.r, p.g, tol=1e-10)
    out["dirichlet_solve_32"] = {"s": time.perf_counter() - t0, "dof": p.n_omega, "cg_iterations": info["iterations"],
                                 "rel_residual": info["rel_residual"]}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    vals = []
    desc = ""
    nt = 1
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        v, desc, dt, nt = oracle_kd_rate(reps=1)
        if i >= args.warmup:
            vals.append(v)
    elapsed = time.perf_counter() - t_all
    value = statistics.mean(vals)
    timings = oracle_timings()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / (args.warmup + args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cube256-linear-a2.5-sin (oracle on a bounded 64^3-box sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": desc},
            "oracle_timings": timings,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ku(args):
    """K.u alone, for external profilers: set-up on a cube box, then --reps stiffness
    actions (Alg. 2).  Box sides a x b x c (--box 256x256x128) embed the cube domain
    of the smallest side in a larger box, which keeps the kernels of the long axes
    while holding less device memory.  Prints the device memory held and a checksum."""
    import torch
    from paper_2403_19854_gb300 import rk
    from paper_2403_19854_gb300 import workloads as W
    box = tuple(int(v) for v in args.box.split("x"))
    if len(box) == 1:
        box = box * 3
    at = 2.5 if args.degree == 1 else 3.0
    p = W.cube_problem(min(box), at, args.degree, "zero")
    if box != p.n:
        p = W.embed(p, box)
    dev = torch.device("cuda:0")
    H = rk.Handle.from_problem(p, device=dev)
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    g = torch.Generator(device=dev)
    g.manual_seed(20240328)
    x = torch.rand(p.nbox, dtype=dt, device=dev, generator=g)
    y = torch.empty_like(x)
    for _ in range(args.reps):
        H.apply_K(x, y)
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    print(f"box {box} degree {args.degree} {args.dtype}: {args.reps} K.u, checksum {float(y.abs().sum()):.6e}, "
          f"device memory {total - free:.3e} B in use")
    H.close()
    return 0


def run_cg(args):
    """A short mixed CG solve alone, for external profilers: set-up as run_ku (the
    cube domain of the smallest side in the --box), then --reps iterations of the
    FP32 CG with its fused x passes (Alg. 5; the iteration cap ends it).  Prints the
    iterations and the device memory held."""
    import torch
    from paper_2403_19854_gb300 import rk
    from paper_2403_19854_gb300 import workloads as W
    box = tuple(int(v) for v in args.box.split("x"))
    if len(box) == 1:
        box = box * 3
    at = 2.5 if args.degree == 1 else 3.0
    p = W.cube_problem(min(box), at, args.degree, "sin")
    if box != p.n:
        p = W.embed(p, box)
    dev = torch.device("cuda:0")
    H = rk.Handle.from_problem(p, device=dev)
    r = torch.as_tensor(p.r, device=dev)
    g = torch.as_tensor(p.g, device=dev)
    _, _, info = H.solve(r, g, opts=rk.default_opts(precision="mixed", tol=1e-10, max_iter=args.reps),
                         raise_on_error=False)
    torch.cuda.synchronize()
    free, total = torch.cuda.mem_get_info()
    print(f"box {box} degree {args.degree}: mixed CG, {info['iterations']} iterations (status {info['status']}), "
          f"device memory {total - free:.3e} B in use")
    H.close()
    return 0


# ------------------------------------------------------------- our arm
# Algorithmic bytes per box node of one launch of each kernel class inside the CG
# iteration (linear basis s = 4, w = bytes per real, u8 masks, int32 node index):
#   x_split       p_old, r in; p, 2 fields out  (direction update fused, no input mask)
#   y_split       2 in, 3 out
#   z_merge       the z axis of Alg. 2 as its regular part: the 3 y outputs in, the 3
#                 z outputs out (one spectral multiplier per group)
#   stiff_pointwise  the local corrections of the non-regular nodes along z (reads and
#                 updates the fields on the boundary layers only: no per-box-node figure)
#   y_merge       3 in, 2 out
#   x_merge       2 in + output mask, Ap out, p in (p.Ap fused)
#   cg_vector     x, r, p, Ap in; x, r out
def pass_bytes(cls, w, s=4):
    return {"x_split": 5 * w, "y_split": 5 * w, "z_merge": 6 * w, "y_merge": 5 * w, "x_merge": 4 * w + 1,
            "cg_vector": 6 * w}.get(cls)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# kernel that dominates a step, from one ncu capture of the 256^3-box cube K.u
# (profiles/dram_zpass_f32_cube256.md; one-pass metrics on the full-size box).
# A value holds only while the kernel is unchanged: the sha256 of each listed
# source region (the kernel and its block shape) is checked at run time, and the
# traffic is null otherwise.
_PASSES = "paper_2403_19854_gb300/csrc/rk_passes.cuh"
_STRIDED = (_PASSES, "template <typename T, int N, int L>\nstruct Strided {", "// PW > 0 (z SPLIT",
            "650985d9545296426b74b48de165243a553705407e8d1c7b69a28f53a204202a")
_SPLIT_START = ("template <typename T, int N, int L, int PW>\n__global__ void __launch_bounds__(Strided<T, N, L>::THREADS, "
                "Strided<T, N, L>::MIN_BLOCKS_SPLIT)")
_MERGE_START = "template <typename T, int N, int L>\n__global__ void __launch_bounds__(Strided<T, N, L>::THREADS, "
_API = "paper_2403_19854_gb300/csrc/rk_api.cu"
MEASURED_TRAFFIC = {
    # the z pass (regular part of the z axis, 3 fields in, 3 out) on the split kernel
    ("z_merge", "f32", 256): (201385472 + 144517120, [
        _STRIDED,
        (_PASSES, _SPLIT_START, _MERGE_START, "c68852f1a89adb44417aa6fbff51d6c92e9eccbfd5e40db56c6d0249da4d1bd0"),
        (_API, "    // Every group has one multiplier at most, so the pass is split-shaped",
         "    {\n      ProfScope ps(h, prof_cls<T>(RK_PROF_Z_STIFF), s);", "94d721f4d25a9cdae6710882bb5af1f3683c567f0edb2804743e02eb3ee4396e"),
    ]),
}


def measured_traffic(cls, prec, size):
    import hashlib
    ent = MEASURED_TRAFFIC.get((cls, prec, size))
    if ent is None:
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    for rel, start, end, digest in ent[1]:
        try:
            with open(os.path.join(root, rel)) as f:
                text = f.read()
            i = text.index(start)
            region = text[i:text.index(end, i)]
        except (OSError, ValueError):
            return None
        if hashlib.sha256(region.encode()).hexdigest() != digest:
            return None
    return ent[0]


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2403_19854_gb300 import rk
    from paper_2403_19854_gb300 import workloads as W

    rk.lib()
    p = W.cube_problem(args.size, 2.5, 1, "sin")
    n_dof = p.n_omega
    chi = torch.as_tensor(p.chi, device=dev)
    cg = torch.as_tensor(p.chi_gamma, device=dev)
    V = torch.as_tensor(p.V, device=dev)
    r = torch.as_tensor(p.r, device=dev)
    g = torch.as_tensor(p.g, device=dev)
    d = torch.empty(p.nbox, dtype=torch.float64, device=dev)
    u = torch.empty_like(d)
    # the replacement settings of the mixed solve, measured on this problem
    # (autotune.best_mixed_opts: one solve per candidate before the warm-up)
    from paper_2403_19854_gb300 import autotune
    Ht = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
    itol, ce, tune_t = autotune.best_mixed_opts(Ht, r, g, tol=args.tol)
    Ht.close()
    # the timed steps use the library's default settings (value = K.u throughput at
    # those); the tuned settings' time-to-solve is one extra step, reported beside it
    opts = rk.default_opts(precision="mixed", tol=args.tol)
    opts_tuned = rk.default_opts(precision="mixed", tol=args.tol, inner_tol=itol, check_every=ce)
    solver_opts = {"timed_steps": {"inner_tol": opts.inner_tol, "check_every": opts.check_every},
                   "autotuned": {"inner_tol": itol, "check_every": ce, "chosen_by": "autotune.best_mixed_opts",
                                 "candidates_s_iterations_status": tune_t}}
    stream = torch.cuda.current_stream()

    def step(prof=False, o=None):
        H = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
        if prof:
            H.profile(True)
        _, _, info = H.solve(r, g, d, u, opts=o if o is not None else opts)
        pr = H.profile_read() if prof else None
        H.close()
        return info, pr

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    clk = Clocks(local)
    barrier()
    clk.start()
    L0 = rk.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        info, _ = step()
        infos.append(info)
    e1.record(stream)
    barrier()
    L1 = rk.kernel_launches()
    clocks = clk.stop()
    ms_local = e0.elapsed_time(e1)
    # one more step, not timed, with CUDA events around every kernel class on the
    # launching stream (this disables the graph replay of CG chunks): per-kernel
    # durations for the roofline
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    _, pr = step(prof=True)
    p1.record(stream)
    torch.cuda.synchronize()
    profiled_ms = p0.elapsed_time(p1)
    profs = [pr]
    # one more step, not in the timed region: the mixed solve with the tuned settings
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    info_tuned, _ = step(o=opts_tuned)
    q1.record(stream)
    torch.cuda.synchronize()
    solver_opts["autotuned"].update({"time_to_solve_s": q0.elapsed_time(q1) / 1e3,
                                     "iterations": info_tuned["iterations"], "status": info_tuned["status"]})
    matvecs = sum(i["matvec_f32"] + i["matvec_f64"] for i in infos)
    ms, units = aggregate_over_ranks(ms_local, float(n_dof * matvecs), world, dev)
    value = units / (ms / 1e3)
    u_mixed = u.cpu().numpy().copy()

    # kernel profile of the profiled step: dominant class and its roofline
    agg = {}
    for pr in profs:
        for k, (t_ms, n) in pr.items():
            a = agg.setdefault(k, [0.0, 0])
            a[0] += t_ms
            a[1] += n
    tot = sum(v[0] for v in agg.values())
    dom = max(agg.items(), key=lambda kv: kv[1][0])
    (dname, dprec), (dms, dn) = dom
    w = 8 if dprec == "f64" else 4
    peak, peak_kind = _peaks()
    bpn = pass_bytes(dname, w)
    roofline = None
    if bpn is not None:
        traffic = args.traffic_bytes if args.traffic_bytes > 0 else measured_traffic(dname, dprec, args.size)
        per_launch = bpn * p.nbox
        achieved = per_launch / (dms / dn / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": f"{dname}_{dprec}", "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                    "algorithmic_bytes_per_launch": per_launch, "peak_source": peak_kind,
                    "share_of_step_kernel_time": dms / tot}
    profile_summary = {f"{k[0]}_{k[1]}": {"ms_total": v[0], "launches": v[1], "share": v[0] / tot}
                       for k, v in sorted(agg.items(), key=lambda kv: -kv[1][0])}

    # comparison point: the FFT work alone of a cuFFT-based Alg. 2 (plain 3D real
    # transforms, no fusion possible): s+1 forward and s+1 inverse per K.u
    cufft = {}
    for dt_name, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        f = torch.rand(p.n[2], p.n[1], p.n[0], dtype=tdt, device=dev)
        for _ in range(2):
            torch.fft.irfftn(torch.fft.rfftn(f), s=f.shape)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        c0.record(stream)
        for _ in range(reps):
            for _ in range(5):  # s + 1 = 5 pairs for the linear basis
                torch.fft.irfftn(torch.fft.rfftn(f), s=f.shape)
        c1.record(stream)
        torch.cuda.synchronize()
        cufft[dt_name] = {"ms_fft_only_per_Ku": c0.elapsed_time(c1) / reps, "real_3d_ffts_per_Ku": 10}
        del f

    # the operators of Appendices A and C at the same size (one launch sequence each)
    appendix = {}
    Ha = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
    qa = torch.rand(p.nbox, dtype=torch.float64, device=dev) * cg
    Aw = cg.double() * (p.h[0] ** 2)
    v64 = torch.rand(p.nbox, dtype=torch.float64, device=dev) * chi
    f_out = torch.empty_like(v64)
    v32 = v64.float()
    f32 = torch.empty_like(v32)
    dd = v64.clone()

    def timed(fn, reps):
        fn()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / reps

    appendix["boundary_rhs_f64_ms"] = timed(lambda: Ha.boundary_rhs(qa, Aw, out=f_out), 3)
    appendix["apply_M_f64_ms"] = timed(lambda: Ha.apply_M(v64, out=f_out), 3)
    appendix["apply_M_f32_ms"] = timed(lambda: Ha.apply_M(v32, out=f32), 10)
    appendix["lumped_mass_f64_ms"] = timed(lambda: Ha.lumped_mass(out=f_out), 3)
    appendix["explicit_step_f64_ms"] = timed(lambda: Ha.transient_explicit(f_out, g, 1e-9, 1, dd), 3)
    Ha.close()
    del qa, Aw, v64, f_out, v32, f32, dd

    # the embedded-domain workload at full size: 12 spheres in a 256^3 box,
    # quadratic basis, a = 3h (set-up and K.u; with direct nodal integration the
    # quadratic-basis stiffness matrix has near-null oscillatory modes, kappa above
    # 1e8 already at 24^3, so its solves do not reach 1e-10)
    sph = W.spheres_problem(n_box=args.size, n_spheres=12, a_tilde=3.0, degree=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Hs = rk.Handle.from_problem(sph, device=dev)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    spheres = {"n_omega": sph.n_omega, "setup_s": setup_s}
    for dt_name, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        x = torch.rand(sph.nbox, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        for _ in range(2):
            Hs.apply_K(x, y)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10 if tdt == torch.float32 else 3
        a0.record(stream)
        for _ in range(reps):
            Hs.apply_K(x, y)
        a1.record(stream)
        torch.cuda.synchronize()
        spheres[f"kU_{dt_name}_ms"] = a0.elapsed_time(a1) / reps
        del x, y
    # time to a common reachable residual: direct nodal integration with the
    # quadratic basis keeps near-zero-energy modes, so neither precision gets far
    # below 1e-2 in a few thousand iterations; both solves use the spectral
    # preconditioner (plain FP64 CG does not reach 1e-2 in 3000 iterations)
    if args.spheres_solve:
        rs, gs = torch.as_tensor(sph.r, device=dev), torch.as_tensor(sph.g, device=dev)
        sol = {"tol": 1e-2, "precond": "spectral"}
        for prec in ("mixed", "fp64"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, si = Hs.solve(rs, gs, precision=prec, tol=1e-2, precond="spectral", max_iter=4000, fp64_finish=0,
                                raise_on_error=False)
            torch.cuda.synchronize()
            sol[prec] = {"time_to_solve_s": time.perf_counter() - t0, "iterations": si["iterations"],
                         "rel_residual": si["rel_residual"], "status": si["status"]}
        spheres["solve_to_1e-2"] = sol
    Hs.close()
    del sph

    # isolated K.u rates (resident d, f)
    H = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
    kd = {}
    for dt_name, tdt in (("f32", torch.float32), ("f64", torch.float64)):
        x = torch.rand(p.nbox, dtype=tdt, device=dev)
        y = torch.empty_like(x)
        reps = 20 if tdt == torch.float32 else 5
        for _ in range(3):
            H.apply_K(x, y)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            H.apply_K(x, y)
        a1.record(stream)
        torch.cuda.synchronize()
        t_ku = a0.elapsed_time(a1) / reps
        kd[dt_name] = {"ms": t_ku, "dof_per_s": n_dof / (t_ku / 1e3)}
    H.close()

    # plain FP64 GPU solve of the same problem, and agreement with the mixed solution
    fp64 = None
    if args.fp64_ref:
        H = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
        d64 = torch.empty_like(d)
        u64 = torch.empty_like(d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, i64 = H.solve(r, g, d64, u64, opts=rk.default_opts(precision="fp64", tol=args.tol),
                             raise_on_error=False)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        H.close()
        u64n = u64.cpu().numpy()
        m = p.chi > 0
        diff = float(np.linalg.norm((u_mixed - u64n)[m]) / np.linalg.norm(u64n[m]))
        err_exact = float(np.linalg.norm((u64n - p.u_exact)[m]) / np.linalg.norm(p.u_exact[m]))
        fp64 = {"time_to_solve_s": t64, "iterations": i64["iterations"], "matvec_f64": i64["matvec_f64"],
                "rel_residual": i64["rel_residual"], "status": i64["status"],
                "rel_l2_u_mixed_vs_fp64": diff, "rel_l2_u_fp64_vs_exact": err_exact}

    # the same solves with the spectral preconditioner (an addition to the paper's
    # plain CG): time-to-solve of set-up + PCG + u^h, mixed and FP64
    pcg = {}
    for prec in ("mixed", "fp64"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Hp = rk.Handle(p.n, p.h, chi, cg, V, 1, 2.5)
        dp = torch.empty_like(d)
        up = torch.empty_like(d)
        _, _, ip = Hp.solve(r, g, dp, up, opts=rk.default_opts(precision=prec, tol=args.tol, precond="spectral"),
                            raise_on_error=False)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        Hp.close()
        m = p.chi > 0
        upn = up.cpu().numpy()
        pcg[prec] = {"time_to_solve_s": tp, "iterations": ip["iterations"], "matvec_f32": ip["matvec_f32"],
                     "matvec_f64": ip["matvec_f64"], "rel_residual": ip["rel_residual"], "status": ip["status"],
                     "rel_l2_u_vs_mixed_cg": float(np.linalg.norm((upn - u_mixed)[m]) / np.linalg.norm(u_mixed[m]))}
        del dp, up

    # end to end through the C ABI with pinned host buffers (copies inside the timing)
    hp = {k: torch.as_tensor(getattr(p, k)).pin_memory() for k in ("chi", "chi_gamma", "V", "r", "g")}
    hd = torch.empty(p.nbox, dtype=torch.float64).pin_memory()
    hu = torch.empty(p.nbox, dtype=torch.float64).pin_memory()
    e2e_ms = []
    e2e_mv = 0
    for i in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = rk.Handle(p.n, p.h, hp["chi"], hp["chi_gamma"], hp["V"], 1, 2.5, stream=rk.ctypes.c_void_p(stream.cuda_stream))
        _, _, ie = H.solve(hp["r"], hp["g"], hd, hu, opts=opts, stream=rk.ctypes.c_void_p(stream.cuda_stream))
        H.close()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_mv += ie["matvec_f32"] + ie["matvec_f64"]
    e2e_total_ms, e2e_units = aggregate_over_ranks(sum(e2e_ms), float(n_dof * e2e_mv), world, dev)
    e2e_value = e2e_units / (e2e_total_ms / 1e3)
    h2d = p.nbox * (1 + 1 + 8 + 8 + 8)
    d2h = p.nbox * (8 + 8)

    # the batched workload (uneven embedded domains, several right-hand sides), small
    # enough for the default run: one rk_solve_batched, spectral PCG
    batched = None
    if args.batched_domains > 0 and world == 1:
        b = batched_core(args.batched_domains, 1e-10, 2000, "spectral", 1, 20240328 + 5000, dev, local, world)
        batched = {"value": b["units_local"] / (b["ms_local"] / 1e3), "unit": "DOF/s", "ms_per_step": b["ms_local"],
                   "config": b["config"], "per_degree": b["per_degree"], "launch_groups": b["launch_stats"],
                   "gpu_launches": b["launches"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, _, nt = oracle_kd_rate()
        cpu = {"value": v, "unit": UNIT, "cores": nt, "kind": "oracle", "sample": desc}

    if rank == 0:
        m = p.chi > 0
        err = float(np.linalg.norm((u_mixed - p.u_exact)[m]) / np.linalg.norm(p.u_exact[m]))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"cube{args.size}-linear-a2.5-sin", "box": list(p.n), "n_omega": n_dof,
                       "degree": 1, "a_tilde": 2.5, "precision": "mixed (FP32 K.u, FP64 dots/refinement)",
                       "tol": args.tol, "l2": "inputs and working set larger than L2 (no flush needed)",
                       "parallelism": f"replicas x{world}", "mixed_solver": solver_opts},
            "time_to_solve_s": {"mixed": ms / args.steps / 1e3,
                                "mixed_autotuned": solver_opts["autotuned"]["time_to_solve_s"],
                                "fp64": fp64["time_to_solve_s"] if fp64 else None,
                                "mixed_pcg": pcg["mixed"]["time_to_solve_s"], "fp64_pcg": pcg["fp64"]["time_to_solve_s"],
                                # the timed mixed steps split into the rk_solve call (right-hand
                                # side, CG, u^h) and the rest (set-up and release of the handle)
                                "mixed_solve_call": statistics.mean(i["solve_ms"] for i in infos) / 1e3,
                                "mixed_setup_and_release": ms / args.steps / 1e3
                                - statistics.mean(i["solve_ms"] for i in infos) / 1e3},
            "pcg_solve": pcg,
            "solve": {"iterations": infos[-1]["iterations"], "outer": infos[-1]["outer"],
                      "matvec_f32": infos[-1]["matvec_f32"], "matvec_f64": infos[-1]["matvec_f64"],
                      "rel_residual": infos[-1]["rel_residual"], "rel_l2_u_vs_exact": err},
            "fp64_solve": fp64,
            "kU_isolated": kd,
            "cufft_comparison": cufft,
            "appendix_ops": appendix,
            "spheres256_quadratic": spheres,
            "batched": batched,
            "profiled_step_ms": profiled_ms,
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms)},
            "gpu_launches": int(L1 - L0),
            "roofline": roofline,
            "kernel_profile": profile_summary,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batched_core(domains, tol, max_iter, precond, steps, seed, dev, local, world):
    """Batched solves of uneven embedded domains: seeded domains of box side
    U{32..160} (1-12 spheres, linear a = 2.5h or quadratic a = 3.0h), 4 right-hand
    sides each, every domain padded to the built FFT side the autotuner measures
    fastest; one step = one rk_solve_batched of all (domain, right-hand side) items
    (mixed precision, a fixed iteration budget per item).  Returns the measured
    quantities (rank-local ms; units aggregated by the caller)."""
    import numpy as np
    import torch
    from paper_2403_19854_gb300 import autotune, rk
    from paper_2403_19854_gb300 import workloads as W

    rk.lib()
    doms = W.batched_domains(n_domains=domains, n_rhs=4, seed=seed)
    items, handles, skipped = [], [], 0
    for p0, rhs in doms:
        free, _ = torch.cuda.mem_get_info()
        if free < 16e9:
            skipped += 1
            continue
        side = autotune.best_side(p0.n[0], p0.degree)
        p = W.embed(p0, (side,) * 3)
        H = rk.Handle.from_problem(p, device=dev)
        hs = [H] + [H.clone() for _ in rhs[1:]]
        handles.append(hs)
        for h, r in zip(hs, rhs):
            rp = W.embed(W.Problem(n=p0.n, h=p0.h, a_tilde=p0.a_tilde, degree=p0.degree, chi=p0.chi,
                                   chi_gamma=p0.chi_gamma, V=p0.V, r=r, g=p0.g), p.n).r
            items.append({"p": p, "S": p0.n[0], "h": h, "r": torch.as_tensor(rp, device=dev),
                          "g": torch.as_tensor(p.g, device=dev),
                          "d": torch.empty(p.nbox, dtype=torch.float64, device=dev)})
    opts = rk.default_opts(precision="mixed", tol=tol, check_every=16, max_iter=max_iter, fp64_finish=0,
                           precond=precond)
    batch = [(it["h"], it["r"], it["g"], it["d"], None) for it in items]
    rk.solve_batched(batch, opts=opts, raise_on_error=False)  # warm-up: graphs, tables
    stream = torch.cuda.current_stream()
    clk = Clocks(local)
    torch.cuda.synchronize()
    clk.start()
    L0 = rk.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = None
    for _ in range(steps):
        infos = rk.solve_batched(batch, opts=opts, raise_on_error=False)
    e1.record(stream)
    torch.cuda.synchronize()
    L1 = rk.kernel_launches()
    clocks = clk.stop()
    ms_local = e0.elapsed_time(e1)
    units_local = float(sum(it["p"].n_omega * (i["matvec_f32"] + i["matvec_f64"]) for it, i in zip(items, infos)))
    per_deg = {}
    for it, i in zip(items, infos):
        dd = per_deg.setdefault(f"degree{it['p'].degree}", {"items": 0, "converged": 0, "iterations": [], "rel": []})
        dd["items"] += 1
        dd["converged"] += int(i["status"] == 0)
        dd["iterations"].append(i["iterations"])
        dd["rel"].append(i["rel_residual"])
    for dd in per_deg.values():
        dd["mean_iterations"] = float(np.mean(dd.pop("iterations")))
        rel = dd.pop("rel")
        dd["median_rel_residual"] = float(np.median(rel))
        dd["worst_rel_residual"] = float(np.max(rel))
    max_it = max(i["iterations"] for i in infos)
    out = {"ms_local": ms_local, "units_local": units_local * steps, "clocks": clocks,
           "launches": int(L1 - L0), "per_degree": per_deg,
           "launch_stats": {"gpu_launches_per_step": int((L1 - L0) / steps),
                            "launches_per_cg_iteration_of_the_batch": (L1 - L0) / steps / max(max_it, 1),
                            "max_iterations": int(max_it)},
           "config": {"domains": len(handles), "skipped_for_memory": skipped, "items": len(items), "tol": tol,
                      "max_iter": max_iter, "precond": precond,
                      "box_nodes": int(sum(it["p"].nbox for it in items)),
                      "dof": int(sum(it["p"].n_omega for it in items)),
                      "padded_sides": [list(v) for v in sorted({(it["S"], it["p"].n[0]) for it in items})]}}
    for hs in handles:
        for h in hs[1:]:
            h.close()
        hs[0].close()
    return out


def run_batched(args):
    """The batched workload on its own line (batched_core)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = batched_core(args.domains, args.tol, args.max_iter, args.precond, args.steps,
                     20240328 + 5000 + 97 * rank, dev, local, world)
    ms, units = aggregate_over_ranks(b["ms_local"], b["units_local"], world, dev)
    if rank == 0:
        cfg = dict(b["config"])
        cfg["workload"] = f"batched {cfg['domains']} domains x 4 rhs"
        line = {"metric": "batched DOF x K.u applications per second (uneven domains, mixed precision)",
                "value": units / (ms / 1e3), "unit": "DOF/s", "n_gpus": world, "steps": args.steps, "warmup": 1,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic", "config": cfg, "per_degree": b["per_degree"],
                "launch_groups": b["launch_stats"], "clocks": b["clocks"], "gpu_launches": b["launches"]}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--fp64-ref", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traffic-bytes", type=float, default=0.0,
                    help="ncu dram bytes per launch of the dominant kernel (from profiles/), if measured")
    ap.add_argument("--workload", default="cube", choices=["cube", "batched", "ku", "cg"],
                    help="cube: the 256^3 cube solve (default); batched: uneven embedded domains; "
                         "ku: set-up and --reps K.u on --box (for external profilers); "
                         "cg: set-up and --reps mixed CG iterations on --box (for external profilers)")
    ap.add_argument("--box", default="128", help="ku, cg: box sides, n or a x b x c")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"], help="ku: precision of K.u")
    ap.add_argument("--degree", type=int, default=1, choices=[1, 2], help="ku: basis degree")
    ap.add_argument("--reps", type=int, default=4, help="ku: number of K.u; cg: iteration cap")
    ap.add_argument("--domains", type=int, default=64, help="batched: number of domains")
    ap.add_argument("--spheres-solve", type=int, default=1,
                    help="time the 12-spheres quadratic solves (mixed and FP64 PCG to 1e-2; about 45 s)")
    ap.add_argument("--batched-domains", type=int, default=16,
                    help="domains of the batched key of the default line (0: none)")
    ap.add_argument("--max-iter", type=int, default=2000, help="batched: CG iterations per item")
    ap.add_argument("--precond", default="none", choices=["none", "spectral"], help="batched: preconditioner")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "cg":
        return run_cg(args)
    if args.workload == "ku":
        return run_ku(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
