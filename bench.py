"""Benchmark of the time-multigrid solve on GB300.

Workload (one step = one full solve from u = 0 to relative residual 1e-10):
one long horizon u' + lambda u = f, lambda = 1, tau = 1e-6, N = 2^24 intervals,
p_t = 1 (Legendre), u0 = 1, f a seeded sum of 4 sinusoids; mixed precision
(FP32 cycles inside FP64-accurate refinement), V(2,2) with the optimal damping
per level (the paper's convergence plots use nu1 = nu2 = nu in {1, 2, 5}; its
numerical section does not state nu).  The metric is time-DoFs/s = N (p_t+1) /
solve time.  Inputs (268 MB load vector, 268 MB solution) are resident in HBM
and larger than L2.

Also reported: the exact scan solve, the plain FP64 form, p_t = 0, 2, 3 on the
same horizon, other sweep counts (V(1,1), V(1,3), V(2,3), V(3,3)), the batched
workloads, per-kernel times and the HBM roofline of the dominant kernel, an
end-to-end number through the host-array entry point, and the CPU oracle.

--impl reference times the FP64 CPU oracle (the textbook multigrid) on a
bounded sample of the same workload.  Multi-GPU: the single long-horizon
problem does not shard; N > 1 ranks run independent replicas.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_FULL = 1 << 24          # overridden by --n-log2 (profiling cases)
TAU = 1e-6
LAM = 1.0
U0 = 1.0
P_MAIN = 1
NU = (2, 2)               # pre-/post-smoothing sweeps of the timed cycles (the paper's plots use nu1 = nu2 in {1, 2, 5})
N_MIN = 1 << 17           # coarsen while N_l > N_MIN: at N = 2^24 the coarsest level has 2^17 intervals,
                          # solved exactly by the parallel affine scan (11 cycles, as with 64 intervals)


def n_min_p(p: int) -> int:
    """Coarsest level of the long-horizon lines: 2^17 intervals (scan) for
    p_t <= 1; from p_t = 2 on the FP32 scan of so long a level costs more than
    the levels it replaces, and the default 64 intervals (one warp) is faster."""
    return N_MIN if p <= 1 else 64


def n_min_for(n: int) -> int:
    """The same hierarchy depth for a sample of n intervals (oracle runs)."""
    return max(64, N_MIN * n // N_FULL)
TOL = 1e-10
METRIC = "time-DoFs/s solved to 1e-10 rel residual (mixed vs FP64 form), % HBM peak"
WORKLOAD = ("long horizon u'+lambda u=f, lambda=1, tau=1e-6, N=2^24, p_t=1, mixed FP32 cycles + FP64-accurate "
            "refinement, V(2,2), omega*, coarsest level 2^17 intervals solved by the parallel affine scan")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_updown0
# launch on the default workload, from one ncu capture; valid only for the
# kernel source it was taken with (first 16 hex digits of the SHA-256 of
# tmg_kernels.cuh), else null.
BATCH_STRIDE = 1          # every s-th heat mode (profiling of smaller cases only)
UPDOWN0_TRAFFIC = {"bytes_per_launch": 1.0180e9, "kernels_sha256": "042edcbfa8d15bc3"}


def measured_traffic():
    import hashlib
    path = os.path.join(ROOT, "paper_1409_5254_gb300", "csrc", "tmg_kernels.cuh")
    try:
        with open(path, "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None
    return UPDOWN0_TRAFFIC["bytes_per_launch"] if h == UPDOWN0_TRAFFIC["kernels_sha256"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cycle_bytes(N: int, d: int, lt: int):
    """Algorithmic HBM bytes of the mixed-precision solve's kernels (FP32 cycle).

    The level-0 residual is a float pair stored in 6 bytes per value (float
    high part, 16-bit low part).
    Start of a solve from u = 0 (k_down0, once): read F, write the residual
    pair and the level-1 right-hand side (N/2 intervals, FP32): 16 B/DoF.
    Confirmation (k_down0, once): read u, F; write the pair and f_1: 24 B/DoF.
    Every cycle, level 0 (k_updown0): read the residual pair, the level-1
    correction and u; write u, the new residual pair and the next level-1
    right-hand side: 6 + 2 + 8 + 8 + 6 + 2 = 32 B/DoF.
    Streaming levels l >= 1 run two per kernel: down reads f_l and writes
    f_{l+2}; up reads f_l and u_{l+2} and writes u_l (FP32); a last single
    level moves 1.5 + 2.5 level vectors.  The on-chip solver reads f_lt and
    writes u_lt once.
    """
    nd = N * d
    half = (N // 2) * d * 4
    start0 = nd * (8 + 6) + half
    confirm0 = nd * (8 + 8 + 6) + half
    updown0 = nd * (6 + 8 + 8 + 6) + 2 * half
    coarse = 0
    l = 1
    while l < lt:
        nl = (N >> l) * d * 4
        if l + 1 < lt:
            coarse += nl + nl // 4 + nl + nl // 4 + nl
            l += 2
        else:
            coarse += nl + nl // 2 + nl + nl // 2 + nl
            l += 1
    tail_io = 2 * (N >> lt) * d * 4 if lt > 0 else 0
    return {"start0": start0, "confirm0": confirm0, "updown0": updown0, "cycle": updown0 + coarse + tail_io}


# Nominal FP64 rate: 2 FP64 FMA per clock per SM, 152 SMs, 2.07 GHz maximum SM
# clock; an FMA, an add or a multiply counts as one operation.
FP64_PEAK_OPS = 152 * 2 * 2.07e9


def fp64_ops_per_interval(d: int, nu1: int, nu2: int):
    """FP64 operations of the useful work per interval and level visit of the
    FP64 cycle's streaming kernels (the halo lanes' recompute excluded):
    zero-start pre-smoothing d^2 + 2d (A^{-1} f, u and A u), each further
    pre-sweep 7d (4d for u, 3d for A u), the residual 3d, the restriction d^2
    per fine interval; the way up repeats the pre-smoothing of u alone
    (d^2 + d, then 4d per further sweep) and adds the prolongation (d^2) and
    nu2 post-sweeps of 4d.  Level 0 adds the residual of the original system
    from u (6d, Legendre running sums) on the way down and u += c (d) on the
    way up.  Returns (down, up, down0, up0)."""
    extra = max(nu1 - 1, 0)
    down = d * d + 2 * d + 7 * d * extra + 3 * d + d * d
    up = d * d + d + 4 * d * extra + d * d + 4 * d * nu2
    return down, up, down + 6 * d, up + d


def fp64_cycle_model(N: int, d: int, nu, lt: int, scanned: bool):
    """Algorithmic bytes and FP64 operations of one cycle of the plain FP64
    form (one level per kernel): level 0 reads u, F and writes r, f_1 on the
    way down (8 + 8 + 8 + 4 B/DoF) and reads r, c_1, u and writes u on the way
    up (8 + 4 + 8 + 8); level l moves 1.5 + 2.5 level vectors; the coarsest
    level (scan: F read twice, u written; on chip: f read, u written)."""
    down, up, down0, up0 = fp64_ops_per_interval(d, *nu)
    nb = N * d * 8
    b = {"down0": 28 * N * d, "up0": 28 * N * d}
    ops = {"down0": down0 * N, "up0": up0 * N}
    coarse_b = coarse_ops = 0
    for l in range(1, lt):
        coarse_b += 4 * (nb >> l)
        coarse_ops += (down + up) * (N >> l)
    coarse_b += (3 if scanned else 2) * (nb >> lt)
    coarse_ops += (d * d + 3 * d + 3) * (N >> lt) * (2 if scanned else 1)
    b["cycle"] = b["down0"] + b["up0"] + coarse_b
    ops["cycle"] = ops["down0"] + ops["up0"] + coarse_ops
    return b, ops


def level0_mixed_recomputed_bytes(N: int, d: int):
    """The mixed form that recomputes the level-0 residual from u every cycle
    (p_t = 10): k_down0 reads u, F and writes the FP32 residual and f_1
    (8 + 8 + 4 + 2 B/DoF); k_up0 reads r, c_1, u and writes u (4 + 2 + 8 + 8)."""
    return {"down0": 22 * N * d, "up0": 22 * N * d}


def kernel_roofline(name, t_ms, nbytes, ops, hbm_peak, peak_kind):
    """Roofline of one kernel launch: the larger of its HBM time (algorithmic
    bytes at the measured copy bandwidth) and its FP64 time (operations at the
    nominal FP64 rate) bounds it; frac = that bound over the measured time."""
    t = t_ms * 1e-3
    t_hbm = nbytes / (hbm_peak * 1e9)
    t_alu = ops / FP64_PEAK_OPS if ops else 0.0
    out = {"kernel": name, "launch_ms": round(t_ms, 5), "bytes_per_launch": int(nbytes),
           "fp64_ops_per_launch": int(ops) if ops else 0,
           "achieved_gbs": round(nbytes / t / 1e9, 1),
           "achieved_fp64_gops": round(ops / t / 1e9, 1) if ops else 0.0}
    if t_alu > t_hbm:
        out.update({"bound": "alu", "achieved": round(ops / t / 1e9, 1), "peak": round(FP64_PEAK_OPS / 1e9, 1),
                    "unit": "G FP64 ops/s", "peak_kind": "nominal (152 SMs x 2 FP64 FMA/clock x 2.07 GHz)",
                    "frac": round(t_alu / t, 4), "hbm_frac": round(t_hbm / t, 4)})
    else:
        out.update({"bound": "hbm", "achieved": round(nbytes / t / 1e9, 1), "peak": hbm_peak, "unit": "GB/s",
                    "peak_kind": peak_kind, "frac": round(t_hbm / t, 4),
                    "fp64_frac": round(t_alu / t, 4) if ops else 0.0})
    return out


def whole_solve_roofline(t_ms, nbytes, ops, hbm_peak, peak_kind, model):
    """Roofline of a whole solve (batched workloads, whose kernels are timed
    together): algorithmic bytes (and FP64 operations) of every kernel of the
    solve over the solve's time."""
    r = kernel_roofline("whole solve", t_ms, nbytes, ops, hbm_peak, peak_kind)
    r["scope"] = "whole solve"
    r["model"] = model
    return r


def time_each(fn, steps: int, stream, torch):
    """Device time of each of `steps` calls of fn (CUDA events on `stream`
    around every call), in ms."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def time_solves(plan, F, u, steps: int, stream, torch):
    """Median device time of `steps` solves (each timed by its own events)."""
    return statistics.median(time_each(lambda: plan.solve(F, U0, u), steps, stream, torch))


def single_line(tmg, torch, stream, F, u, p: int, tau: float, prec: str, n_min: int, steps: int, eager: bool,
                hbm_peak: float, peak_kind: str, nu=None):
    """One single-problem side line: median of `steps` solves, cycles, FP64
    residual, error against the exact FP64 solve, and the roofline of its
    dominant level-0 kernel from per-kernel event times of 10 eager cycles."""
    nu = NU if nu is None else nu
    N, d = F.shape[0], p + 1
    with tmg.Plan(p, tau, LAM, N, precision=prec, tol=TOL, stream=stream, max_cycles=300, nu1=nu[0], nu2=nu[1],
                  n_min=n_min, use_graph=not eager) as pl:
        pl.solve(F, U0, u)
        times = time_each(lambda: pl.solve(F, U0, u), steps, stream, torch)
        st = pl.stats()
        info = pl.info()
        err = pl.error_vs_fp64(F, U0, u)
        prof = pl.profile_cycle(F, U0, u.clone(), reps=10)
    ms = statistics.median(times)
    roof = level0_roofline(prec, p, N, nu, prof, info, hbm_peak, peak_kind)
    return {"value": N * d / (ms * 1e-3), "unit": "DoF/s", "ms_per_step": round(ms, 4),
            "ms_mean": round(statistics.fmean(times), 4), "solves_timed": steps, "precision": prec,
            "cycles": st.cycles, "rel_res": st.rel_res, "err_vs_fp64": err, "cycle": f"V{tuple(nu)}",
            "levels": info["levels"], "coarsest_intervals": info["tail_intervals"], "roofline": roof}


def level0_roofline(prec: str, p: int, N: int, nu, prof: dict, info: dict, hbm_peak: float, peak_kind: str):
    """Roofline of the dominant level-0 kernel of a single-problem solve from
    the per-kernel event times of tmg_profile_cycle (`prof`) and the byte and
    FP64-operation models above."""
    d = p + 1
    lt = info["tail_level"]
    scanned = p + 1 > 6 or info["tail_intervals"] > 8192
    if prec == "fp64":
        b, ops = fp64_cycle_model(N, d, nu, lt, scanned)
        k = [kernel_roofline("k_down0 (FP64 residual from u, pre-smoothing, restriction)", prof["down0"], b["down0"],
                             ops["down0"], hbm_peak, peak_kind),
             kernel_roofline("k_up0 (recomputed pre-smoothing, prolongation, post-smoothing, u += c)", prof["up0"],
                             b["up0"], ops["up0"], hbm_peak, peak_kind)]
        cyc = {"cycle_bytes": b["cycle"], "cycle_fp64_ops": ops["cycle"], "cycle_ms": round(prof["cycle"], 5),
               "cycle_frac": round(max(b["cycle"] / (hbm_peak * 1e9), ops["cycle"] / FP64_PEAK_OPS)
                                   / (prof["cycle"] * 1e-3), 4)}
    elif d > 6:
        b = level0_mixed_recomputed_bytes(N, d)
        k = [kernel_roofline("k_down0 (mixed, residual recomputed from u)", prof["down0"], b["down0"], 0, hbm_peak,
                             peak_kind),
             kernel_roofline("k_up0 (mixed)", prof["up0"], b["up0"], 0, hbm_peak, peak_kind)]
        cyc = {"cycle_ms": round(prof["cycle"], 5)}
    else:
        cb = cycle_bytes(N, d, lt)
        k = [kernel_roofline("k_updown0", prof["up0"], cb["updown0"], 0, hbm_peak, peak_kind)]
        steady = prof["cycle"] - prof["down0"]
        cyc = {"cycle_bytes": cb["cycle"], "cycle_ms": round(steady, 5),
               "cycle_frac": round(cb["cycle"] / (steady * 1e-3) / 1e9 / hbm_peak, 4)}
    dom = max(k, key=lambda r: r["launch_ms"])
    roof = dict(dom)
    roof.update(cyc)
    if len(k) > 1:
        roof["other_level0_kernel"] = min(k, key=lambda r: r["launch_ms"])
    return roof


def run_ours(args):
    import numpy as np
    import torch

    import __graft_entry__
    from paper_1409_5254_gb300 import inputs, replicas, tmg

    rank, local, world = replicas.rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    hbm_peak, peak_kind = peaks()

    d = P_MAIN + 1
    prob = inputs.scalar_problem(1, N_FULL, P_MAIN, lam=LAM, tau=TAU, u0=U0)
    F = torch.from_numpy(prob["F"]).to(dev)
    u = torch.empty_like(F)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    plan = tmg.Plan(P_MAIN, TAU, LAM, N_FULL, precision="mixed", tol=TOL, stream=stream, use_graph=not args.eager,
                    nu1=NU[0], nu2=NU[1], n_min=n_min_p(P_MAIN))
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    for _ in range(args.warmup):
        plan.solve(F, U0, u)
    st = plan.stats()
    info = plan.info()

    # the timed region: exactly `steps` solves, a barrier and a device
    # synchronisation on both sides, each solve timed by its own events
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    times = time_each(lambda: plan.solve(F, U0, u), args.steps, stream, torch)
    clk.stop()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ms = replicas.max_over_ranks(statistics.median(times), dev)
    ms_mean = replicas.max_over_ranks(statistics.fmean(times), dev)
    st = plan.stats()
    value = replicas.aggregate_throughput([N_FULL * d] * world, ms)    # one replica per rank

    # accuracy of the timed result, in FP64 on the GPU (residual entry point)
    r = plan.residual(F, U0, u)
    Fh = torch.from_numpy(prob["F"].copy()).to(dev)
    Fh[0, 0] += U0
    Fh[0, 1] -= U0
    rel_fp64 = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(Fh))
    del r, Fh
    # error of the timed result against the exact FP64 solve (tmg_error_vs_fp64)
    err_vs_fp64 = plan.error_vs_fp64(F, U0, u)

    # the exact FP64 solve by the parallel affine scan as a throughput ceiling
    # (one pass to reduce each tile of F, one to replay it: reads F twice,
    # writes u once)
    u_ex = torch.empty_like(F)
    plan.solve_direct(F, U0, u_ex)
    n_dir = max(10, args.steps // 2)
    ms_dir = statistics.median(time_each(lambda: plan.solve_direct(F, U0, u_ex), n_dir, stream, torch))
    dir_bytes = 3 * N_FULL * d * 8
    # FP64 operations (an FMA or an add counts one) per interval: pass 1 c^T f and
    # the map composition (d + 2), pass 3 c^T f, A^{-1} f + g e and the carry
    # (d^2 + 2d + 1)
    fp64_ops = N_FULL * (d * d + 3 * d + 3)
    direct = {"value": N_FULL * d / (ms_dir * 1e-3), "unit": "DoF/s", "ms_per_step": round(ms_dir, 4),
              "solves_timed": n_dir, "precision": "fp64", "bytes_per_dof": 24, "lower_bound_bytes_per_dof": 16,
              "roofline": kernel_roofline("k_scan_tiles + k_scan_prefix + k_scan_apply", ms_dir, dir_bytes,
                                          fp64_ops, hbm_peak, peak_kind),
              "note": "exact parallel-scan solve (not multigrid), same problem and stream"}
    del u_ex

    # per-kernel times of one cycle (events on the plan's stream) and the
    # roofline of the dominant kernel, k_updown0 (the level-0 kernel of every
    # cycle; k_down0 runs once per solve, plus once to confirm convergence)
    prof = plan.profile_cycle(F, U0, u.clone(), reps=20)
    cb = cycle_bytes(N_FULL, d, info["tail_level"])
    t_dom = prof["up0"]
    achieved = cb["updown0"] / (t_dom * 1e-3) / 1e9
    steady_ms = prof["cycle"] - prof["down0"]
    roofline = {"bound": "hbm", "kernel": "k_updown0", "achieved": round(achieved, 1),
                "peak": hbm_peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
                "traffic": args.traffic if args.traffic else
                (measured_traffic() if N_FULL == 1 << 24 and NU == (2, 2) else None),
                "bytes_per_launch": cb["updown0"], "bytes_per_dof": 32,
                "byte_model": "k_updown0 per DoF: read the level-0 residual pair 6 (FP32 high part + 16-bit low "
                              "code), u 8, the level-1 correction 2; write u 8, the updated residual pair 6, the "
                              "next level-1 right-hand side 2 = 32 B",
                "survey_bytes_per_dof": 60,
                "survey_byte_model_note": "the survey's 26 + 34 B/DoF counts a level-0 down and up kernel per cycle "
                                          "that store the correction c and an FP32 residual and re-read F; here "
                                          "one kernel does the way up of a cycle and the way down of the next, "
                                          "the residual is updated by r -= L c from the float pair (F is read only "
                                          "at the start and to confirm), and c is recomputed instead of stored",
                "launch_ms": round(t_dom, 5), "launches_per_solve": st.cycles,
                "cycle_bytes": cb["cycle"], "cycle_ms": round(steady_ms, 5),
                "cycle_frac": round(cb["cycle"] / (steady_ms * 1e-3) / 1e9 / hbm_peak, 4),
                "solve_ms_per_cycle": round(ms / max(st.cycles, 1), 5),
                "kernel_ms": {"down0_confirm_once_per_solve": round(prof["down0"], 5),
                              "down_levels": round(prof["down_levels"], 5),
                              "coarsest_solve": round(prof["coarse_on_chip"], 5),
                              "up_levels": round(prof["up_levels"], 5), "updown0": round(prof["up0"], 5),
                              "cycle_events": round(prof["cycle"], 5)}}

    if d > 6:   # --p-t 10 / 20 (profiling runs): no fused level-0 kernel at these widths
        roofline = level0_roofline("mixed", P_MAIN, N_FULL, NU, prof, info, hbm_peak, peak_kind)
    # every kernel of the graph body launches in each of the cycles + 1 loop iterations
    launches = args.steps * (st.cycles + 1) * plan.launches_per_cycle()

    extra = {}
    if rank == 0 and not args.quick:
        nside = max(10, args.steps // 4)
        # plain FP64 form on the same problem
        extra["fp64_form"] = single_line(tmg, torch, stream, F, u, P_MAIN, TAU, "fp64", N_MIN, nside, args.eager,
                                         hbm_peak, peak_kind)
        # the other degrees of the same long horizon, mixed precision
        per_p = {}
        for p in (0, 2, 3, 4, 5):
            pr = inputs.scalar_problem(1, N_FULL, p, lam=LAM, tau=TAU, u0=U0)
            Fp = torch.from_numpy(pr["F"]).to(dev)
            up = torch.empty_like(Fp)
            try:
                per_p[str(p)] = single_line(tmg, torch, stream, Fp, up, p, TAU, "mixed", n_min_p(p), nside,
                                            args.eager, hbm_peak, peak_kind)
            except tmg.TmgError as e:
                per_p[str(p)] = {"error": str(e)}
            del Fp, up
        extra["per_p_mixed"] = per_p
        # the same long horizon at the larger step tau = 1/1024 (z ~ 1e-3; T = 16384)
        tau2 = 1.0 / 1024
        pr = inputs.scalar_problem(1, N_FULL, P_MAIN, lam=LAM, tau=tau2, u0=U0)
        Fp = torch.from_numpy(pr["F"]).to(dev)
        up = torch.empty_like(Fp)
        del pr
        try:
            extra["tau_1_1024"] = single_line(tmg, torch, stream, Fp, up, P_MAIN, tau2, "mixed", N_MIN, nside,
                                              args.eager, hbm_peak, peak_kind)
            extra["tau_1_1024"]["z"] = LAM * tau2
        except tmg.TmgError as e:
            extra["tau_1_1024"] = {"error": str(e)}
        del Fp, up
        # p_t = 10 on the same long horizon, in both forms (the coarsest level is
        # solved by the scan; the mixed form recomputes the level-0 residual from u)
        pr = inputs.scalar_problem(1, N_FULL, 10, lam=LAM, tau=TAU, u0=U0)
        Fp = torch.from_numpy(pr["F"]).to(dev)
        up = torch.empty_like(Fp)
        del pr
        for prec in ("mixed", "fp64"):
            try:
                extra[f"p10_{prec}"] = single_line(tmg, torch, stream, Fp, up, 10, TAU, prec, 64,
                                                   10 if prec == "mixed" else 3, args.eager, hbm_peak, peak_kind)
            except tmg.TmgError as e:
                extra[f"p10_{prec}"] = {"error": str(e)}
        del Fp, up
        # p_t = 20 (21 x 21 blocks, the paper's largest degree) on the first
        # 2^22 intervals of the same step (3.7e8 values per vector at 2^24)
        n20 = N_FULL >> 2
        pr = inputs.scalar_problem(1, n20, 20, lam=LAM, tau=TAU, u0=U0)
        Fp = torch.from_numpy(pr["F"]).to(dev)
        up = torch.empty_like(Fp)
        del pr
        for prec in ("mixed", "fp64"):
            try:
                extra[f"p20_{prec}"] = single_line(tmg, torch, stream, Fp, up, 20, TAU, prec, 64,
                                                   10 if prec == "mixed" else 3, args.eager, hbm_peak, peak_kind)
                extra[f"p20_{prec}"]["N"] = n20
            except tmg.TmgError as e:
                extra[f"p20_{prec}"] = {"error": str(e)}
        del Fp, up
        # other sweep counts on the headline problem (same solver, same tolerance)
        nus = {}
        for nu in ((1, 1), (1, 3), (2, 3), (3, 3)):
            nus[f"V({nu[0]},{nu[1]})"] = single_line(tmg, torch, stream, F, u, P_MAIN, TAU, "mixed", N_MIN, nside,
                                                     args.eager, hbm_peak, peak_kind, nu=nu)
        extra["nu_variants"] = nus
        # the space-time heat equation with a spatial operator (Section 7 outlook)
        extra["space_time_heat"] = _space_time_heat(dev, stream, nside, torch, hbm_peak, peak_kind, args.eager)

    if not args.quick:
        # every rank solves its shard of the batched workloads
        extra_b = run_batched_configs(dev, stream, args.steps, torch, rank, world, hbm_peak=hbm_peak,
                                      peak_kind=peak_kind)
        if rank == 0:
            extra["batched"] = extra_b

    # end to end through the host-array entry point (pinned buffers, copies inside the call)
    F_h = torch.from_numpy(prob["F"]).pin_memory()
    u_h = torch.empty_like(F_h).pin_memory()
    plan.solve_host(F_h, U0, u_h)
    if dist is not None:
        dist.barrier()
    n_e2e = max(10, args.steps // 2)
    t_list = []
    for _ in range(n_e2e):
        t0 = time.perf_counter()
        plan.solve_host(F_h, U0, u_h)
        t_list.append(time.perf_counter() - t0)
    t_e2e = replicas.max_over_ranks(statistics.median(t_list), dev)
    nbytes = N_FULL * d * 8
    e2e = {"value": replicas.aggregate_throughput([N_FULL * d] * world, t_e2e * 1e3), "unit": "DoF/s",
           "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": round(t_e2e * 1e3, 3), "steps_timed": n_e2e,
           "timing": "host wall clock per call, median"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(batched=not args.quick)
        if not args.quick:
            cpu["space_time_heat"] = heat_cpu_baseline()

    plan.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms, 4), "ms_mean": round(ms_mean, 4),
                "timing": "median of per-solve CUDA-event times on the plan's stream",
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": N_FULL, "p_t": P_MAIN, "tau": TAU, "lambda": LAM, "u0": U0,
                           "tol": TOL, "cycles": st.cycles, "levels": info["levels"],
                           "tail_level": info["tail_level"], "coarsest_intervals": info["tail_intervals"],
                           "precision": "mixed",
                           "l2": "inputs larger than L2 (268 MB load vector + 268 MB solution)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "rel_res_fp64": rel_fp64, "err_vs_fp64": err_vs_fp64, "time_steps_per_s": value / d,
                "setup_ms": round(setup_ms, 2), "direct_scan": direct, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary()}
        line.update(extra)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


HEAT_N, HEAT_NX, HEAT_P = 4096, 127, 1   # space-time heat: intervals, interior grid points a side, degree
HEAT_NU, HEAT_NUC = (2, 2), 1             # V(2,2) in time (as the long horizon), one V-cycle on the last interval


def _space_time_heat(dev, stream, nsteps, torch, hbm_peak, peak_kind, eager):
    """The space-time heat equation of the paper's outlook (Section 7): the
    5-point Laplacian on a 127 x 127 interior grid (h = 1/128), N = 4096 DG
    intervals of degree 1 on (0, 1), 1.32e8 space-time unknowns (the size of
    the paper's own heat run), to TOL.  One step = one solve from zero,
    median of `nsteps` (mixed form) or 3 (FP64 form) CUDA-event timed solves
    on the plan's stream.  The roofline is the level-0 post kernel's
    (prolongation + post-smoothing accumulating into the correction: reads
    r and the coarse correction, reads and writes the output, 4-byte
    values)."""
    from paper_1409_5254_gb300 import inputs, tmg
    tau, F, u0 = inputs.heat_problem(1, HEAT_N, HEAT_P, HEAT_NX)
    Fd = torch.from_numpy(F).to(dev)
    u0d = torch.from_numpy(u0).to(dev)
    del F
    u = torch.empty_like(Fd)
    d, n, N = HEAT_P + 1, HEAT_NX, HEAT_N
    nc = (n - 1) // 2
    dofs = Fd.numel()
    out = {"unit": "DoF/s", "grid": f"{n}x{n}", "N": N, "p_t": HEAT_P, "tau": tau, "dofs": dofs, "tol": TOL,
           "cycle": f"V{HEAT_NU} in time, one spatial V(1,1)-cycle per block solve, nu_c = {HEAT_NUC}",
           "data": "synthetic: f(t,x) = sum of 3 space fields U(-1,1) x sin(2 pi m t), u0 ~ U(-1,1)"}
    u_mixed = None
    for prec, steps in (("mixed", nsteps), ("fp64", 3)):
        with tmg.HeatPlan(HEAT_P, tau, n, N, tol=TOL, max_cycles=100, precision=prec, use_graph=not eager,
                          nu1=HEAT_NU[0], nu2=HEAT_NU[1], nu_c=HEAT_NUC, stream=stream) as hp:
            hp.solve(Fd, u0d, u)
            times = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hp.solve(Fd, u0d, u)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            ms = statistics.median(times)
            st = hp.stats()
            info = hp.info()
            res = {"value": dofs / (ms * 1e-3), "ms_per_step": round(ms, 3), "solves_timed": steps,
                   "cycles": st.cycles, "rel_res_fp64": st.rel_res,
                   "launches_per_cycle": info["launches_per_cycle"], "time_levels": info["time_levels"],
                   "space_levels": info["space_levels"], "workspace_bytes": info["workspace_bytes"]}
            if prec == "mixed":
                u_mixed = u.clone()
            else:
                res["mixed_vs_fp64_max_rel"] = float((u_mixed - u).abs().max() / u.abs().max())
            prof = hp.profile(Fd, u0d, u, reps=10)
            es = 4 if prec == "mixed" else 8
            post_bytes = es * d * N * (3 * n * n + nc * nc)
            res["kernels_ms"] = {k: round(v, 4) for k, v in prof.items()}
            if prec == "mixed":
                res["roofline"] = {"kernel": "kh_post_w (spatial level 0, accumulating)", "bound": "hbm",
                                   "achieved": post_bytes / (prof["post"] * 1e-3) / 1e9, "peak": hbm_peak,
                                   "unit": "GB/s",
                                   "frac": post_bytes / (prof["post"] * 1e-3) / 1e9 / hbm_peak,
                                   "traffic": None, "peak_kind": peak_kind,
                                   "bytes_model": "4 B x (p_t+1) x N x (3 n^2 + nc^2): r, out read+write, "
                                                  "coarse correction"}
                pre_bytes = 4 * d * N * (n * n + nc * nc)
                res_bytes = 4 * d * N * n * n * 3
                upd_bytes = d * N * n * n * (4 + 16 + 16)
                res["kernel_fracs"] = {
                    "pre": round(pre_bytes / (prof["pre"] * 1e-3) / 1e9 / hbm_peak, 3),
                    "post": round(post_bytes / (prof["post"] * 1e-3) / 1e9 / hbm_peak, 3),
                    "time_residual": round(res_bytes / (prof["resid"] * 1e-3) / 1e9 / hbm_peak, 3),
                    "pair_update": round(upd_bytes / (prof["update"] * 1e-3) / 1e9 / hbm_peak, 3),
                    "note": "algorithmic bytes / event time / measured HBM copy bandwidth"}
            out[prec] = res
    # other sweep counts in time, mixed form
    variants = {}
    for nu in ((1, 1), (3, 3)):
        with tmg.HeatPlan(HEAT_P, tau, n, N, tol=TOL, max_cycles=100, precision="mixed", use_graph=not eager,
                          nu1=nu[0], nu2=nu[1], nu_c=HEAT_NUC, stream=stream) as hp:
            hp.solve(Fd, u0d, u)
            times = []
            for _ in range(max(3, nsteps // 2)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hp.solve(Fd, u0d, u)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            st = hp.stats()
            variants[f"V({nu[0]},{nu[1]})"] = {"ms_per_step": round(statistics.median(times), 3), "cycles": st.cycles,
                                               "rel_res_fp64": st.rel_res}
    out["mixed_variants"] = variants
    out["value"] = out["mixed"]["value"]
    del Fd, u0d, u, u_mixed
    torch.cuda.empty_cache()
    return out


def heat_cpu_baseline(sample_N: int = 16):
    """The heat oracle (oracle/heat.py) on one host core, on the first
    sample_N of the 4096 intervals of the same problem (same grid, step and
    forcing)."""
    import oracle.heat as oheat
    from paper_1409_5254_gb300 import inputs
    tau, F, u0 = inputs.heat_problem(1, HEAT_N, HEAT_P, HEAT_NX)
    F = F[:sample_N].copy()
    t0 = time.perf_counter()
    _, hist = oheat.solve(HEAT_P, tau, HEAT_NX, F, u0, tol=TOL, max_cycles=100, nu1=HEAT_NU[0], nu2=HEAT_NU[1],
                          nu_c=HEAT_NUC)
    t = time.perf_counter() - t0
    return {"value": F.size / t, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"first {sample_N} of the 4096 intervals, {HEAT_NX}x{HEAT_NX} grid, textbook space-time "
                      f"V{HEAT_NU} cycle to {TOL} ({len(hist) - 1} cycles), {t:.2f} s"}


def _time_batch(batch, f, u0, u, steps, stream, torch):
    """Median device time of `steps` batched solves."""
    return statistics.median(time_each(lambda: batch.solve(f, u0, u), steps, stream, torch))


def oracle_levels(N: int, n_min: int = 64) -> int:
    """Levels of an instance's own hierarchy: coarsen while even and longer
    than n_min intervals (the paper's nested meshes)."""
    L, n = 1, N
    while n % 2 == 0 and n > n_min:
        n //= 2
        L += 1
    return L


def batched_solve_model(Nv, pv, cyc, prec: str):
    """Algorithmic bytes (and FP64 operations for the FP64 form) of one
    batched solve on the instances' real lengths (the padding of a group is
    not algorithmic work).  Mixed form per instance: the start (read F, write
    the residual pair and f_1: 16 B/DoF), c cycles of the level-0 kernel and
    the coarse levels (cycle_bytes: 32 B/DoF at level 0, two streaming levels
    per kernel), and the norm-only confirmation (read u, F: 16 B/DoF).  FP64
    form: c cycles of fp64_cycle_model plus the final residual from u."""
    nbytes = ops = 0
    for N, p, c in zip(Nv, pv, cyc):
        N, d, c = int(N), int(p) + 1, int(c)
        lt = oracle_levels(N) - 1
        if prec == "mixed":
            per = cycle_bytes(N, d, lt)["cycle"] if lt > 0 else 32 * N * d
            nbytes += 16 * N * d + c * per + 16 * N * d
        else:
            b, o = fp64_cycle_model(N, d, NU, lt, False)
            nbytes += c * b["cycle"] + b["down0"]
            ops += c * o["cycle"] + o["down0"]
    return nbytes, ops


def run_batched_configs(dev, stream, steps, torch, rank: int = 0, world: int = 1,
                        only=("heat", "uneven", "gradients"), precisions=("mixed", "fp64"), eager=False,
                        hbm_peak=None, peak_kind="measured"):
    """The batched workloads: decoupled 2-D heat modes, an uneven batch, and
    gradients through the adjoint.  One step = one batched solve (plus the
    adjoint for the gradient workload); inputs resident in HBM; the median of
    at least 10 steps.  With several ranks each solves its shard of the
    instances (balanced by N (p_t+1)); the value is all instances' DoFs over
    the slowest rank's time.  `only` and `precisions` select workloads and
    forms (for profiling one of them)."""
    import numpy as np
    from paper_1409_5254_gb300 import inputs, replicas, tmg

    if hbm_peak is None:
        hbm_peak, peak_kind = peaks()

    def shard(weights):
        return replicas.partition_instances(weights, world)[rank]

    nsteps = max(10, steps // 4)
    out = {}
    if "heat" in only:
        out.update(_heat_modes(dev, stream, nsteps, torch, shard, precisions, eager, hbm_peak, peak_kind))
    if "uneven" in only:
        out.update(_uneven(dev, stream, nsteps, torch, shard, precisions, eager, hbm_peak, peak_kind))
    if "gradients" in only:
        out.update(_gradients(dev, stream, nsteps, torch, shard, eager, hbm_peak, peak_kind))
    if world > 1:
        out["sharding"] = f"instances split over {world} ranks (no data exchange), weak in per-rank time"
    return out


def _batched_form(tmg, torch, stream, dev, replicas, prec, pv, tau, lamv, Nv, f, u0, u, nsteps, eager, hbm_peak,
                  peak_kind, n_dofs_all, **kw):
    """One batched form: setup time, median solve time, per-instance cycles,
    residuals and errors against the exact FP64 solves, whole-solve roofline."""
    import numpy as np
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    with tmg.Batch(pv, tau, lamv, Nv, precision=prec, tol=TOL, max_cycles=300, stream=stream,
                   nu1=NU[0], nu2=NU[1], use_graph=not eager, **kw) as B:
        torch.cuda.synchronize()
        setup_ms = (time.perf_counter() - t_setup) * 1e3
        B.solve(f, u0, u)
        ms = _time_batch(B, f, u0, u, nsteps, stream, torch)
        cyc, rel, mx = B.stats()
        err = B.error_vs_fp64(f, u0, u)
        info = B.info()
    nbytes, ops = batched_solve_model(Nv, pv, cyc, prec)
    ms = replicas.max_over_ranks(ms, dev)
    kinds = [g["schedule"] for g in info["group_info"]]
    model = ("mixed: 16 B/DoF start + cycles x (32 B/DoF level 0 + coarse levels) + 16 B/DoF confirmation, per "
             "instance on its real length and its own cycle count" if prec == "mixed" else
             "FP64: cycles x (28 + 28 B/DoF level 0 + 4 level vectors per coarse level) and the FP64 operations "
             "of fp64_ops_per_interval, per instance on its real length and its own cycle count")
    return {"value": n_dofs_all / (ms * 1e-3), "ms_per_step": round(ms, 3), "solves_timed": nsteps,
            "precision": prec,
            "max_cycles": int(replicas.max_over_ranks(mx, dev)),
            "mean_cycles": round(float(np.mean(cyc)), 2),
            "max_cycles_by_degree": {str(int(q)): int(np.max(cyc[np.asarray(pv) == q]))
                                     for q in sorted(set(int(x) for x in np.asarray(pv)))},
            "max_rel_res": replicas.max_over_ranks(float(rel.max()), dev),
            "err_vs_fp64": {"max": replicas.max_over_ranks(float(np.max(err)), dev),
                            "median": float(np.median(err))},
            "setup_ms": round(setup_ms, 1),
            "groups": info["groups"], "computed_dofs": info["padded_values"],
            "groups_cta": kinds.count("cta"), "groups_grid": kinds.count("grid"),
            "autotune_whole_batch_ms": {k: (round(v, 3) if v == v else None)
                                        for k, v in info["whole_batch_ms"].items()},
            "roofline": whole_solve_roofline(ms, nbytes, ops, hbm_peak, peak_kind, model)}


def _heat_modes(dev, stream, nsteps, torch, shard, precisions, eager, hbm_peak, peak_kind):
    import numpy as np
    from paper_1409_5254_gb300 import inputs, replicas, tmg
    out = {}
    # 65,536 heat modes, N = 4096, p_t = 1, T = 1
    lam_all, amps_all, freqs_all = inputs.heat_modes_batch(2, 256, 4096, 1)
    lam_all, amps_all, freqs_all = lam_all[::BATCH_STRIDE], amps_all[::BATCH_STRIDE], freqs_all[::BATCH_STRIDE]
    n_all, N, p = lam_all.shape[0], 4096, 1
    idx = shard(np.full(n_all, N * (p + 1)))
    lam, amps, freqs = lam_all[idx], amps_all[idx], freqs_all[idx]
    n = len(idx)
    f = inputs.sine_load_vectors(amps, freqs, 1.0, N, p, device=dev).reshape(-1)
    u0 = torch.zeros(n, dtype=torch.float64, device=dev)
    u = torch.empty_like(f)
    res = {}
    for prec in precisions:
        res[prec] = _batched_form(tmg, torch, stream, dev, replicas, prec, [p] * n, 1.0 / N, lam, [N] * n, f, u0,
                                  u, nsteps, eager, hbm_peak, peak_kind, n_all * N * (p + 1))
    out["heat_modes_65536x4096_p1" if BATCH_STRIDE == 1 else f"heat_modes_{n_all}x4096_p1"] = {
        "unit": "DoF/s", "instances": n_all, "N": N, "p_t": p,
        "lambda_range": [float(lam_all.min()), float(lam_all.max())], **res}
    del f, u, u0
    torch.cuda.empty_cache()
    return out


def _uneven(dev, stream, nsteps, torch, shard, precisions, eager, hbm_peak, peak_kind):
    from paper_1409_5254_gb300 import inputs, replicas, tmg
    out = {}
    # uneven batch: 10,000 instances, N log-uniform in [2^6, 2^16], p_t in {0..3}, lambda tau in [1e-3, 1e3]
    Nv_all, pv_all, z_all = inputs.uneven_batch(3, 10000)
    A_all, K_all = inputs.sinusoid_batch_params(3, len(Nv_all))
    dofs = int((Nv_all * (pv_all + 1)).sum())
    idx = shard(Nv_all * (pv_all + 1))
    Nv, pv, z, A, K = Nv_all[idx], pv_all[idx], z_all[idx], A_all[idx], K_all[idx]
    tau = 1.0 / Nv
    lamv = z / tau
    parts = [inputs.sine_load_vectors(A[i:i + 1], K[i:i + 1], 1.0, int(Nv[i]), int(pv[i]), device=dev).reshape(-1)
             for i in range(len(Nv))]
    f = torch.cat(parts)
    del parts
    u0 = torch.ones(len(Nv), dtype=torch.float64, device=dev)
    u = torch.empty_like(f)
    res = {}
    for prec in precisions:
        res[prec] = _batched_form(tmg, torch, stream, dev, replicas, prec, pv, tau, lamv, Nv, f, u0, u, nsteps,
                                  eager, hbm_peak, peak_kind, dofs)
    if "mixed" in precisions:
        # W(2,2) cycles for the whole batch (the p_t = 0 instances need fewer cycles)
        res["mixed_W"] = _batched_form(tmg, torch, stream, dev, replicas, "mixed", pv, tau, lamv, Nv, f, u0, u,
                                       nsteps, eager, hbm_peak, peak_kind, dofs, gamma=2)
        res["mixed_W"]["cycle"] = f"W{NU}"
    out["uneven_10000"] = {"unit": "DoF/s", "instances": len(Nv_all), "dofs": dofs, **res}
    del f, u, u0
    torch.cuda.empty_cache()
    return out


def _gradients(dev, stream, nsteps, torch, shard, eager, hbm_peak, peak_kind):
    import numpy as np
    from paper_1409_5254_gb300 import inputs, replicas, tmg
    out = {}
    # gradients: 4096 instances, N = 16384, p_t = 2, lambda log-uniform in [1, 1e4], T = 1
    n_all, N, p = 4096, 16384, 2
    lam_all, u0_all, target_all = inputs.adjoint_problem(4, n_all, N, p)
    A_all, K_all = inputs.sinusoid_batch_params(4, n_all)
    idx = shard(np.full(n_all, N * (p + 1)))
    n = len(idx)
    f = inputs.sine_load_vectors(A_all[idx], K_all[idx], 1.0, N, p, device=dev).reshape(-1)
    u0 = torch.from_numpy(u0_all[idx]).to(dev)
    y = torch.from_numpy(target_all[idx]).to(dev)
    u = torch.empty_like(f)
    with tmg.Batch([p] * n, 1.0 / N, lam_all[idx], N, precision="mixed", tol=TOL, max_cycles=300, stream=stream,
                   nu1=NU[0], nu2=NU[1], use_graph=not eager) as B:
        def step():
            B.solve(f, u0, u)
            e = u.view(n, N, p + 1).sum(dim=2)
            g = ((e - y)[:, :, None].expand(n, N, p + 1)).contiguous().reshape(-1)
            return B.adjoint(g, u)
        B.solve(f, u0, u)
        cyc_f, _, _ = B.stats()
        err_f = B.error_vs_fp64(f, u0, u)
        step()
        cyc_a, rel_a, mx = B.stats()
        ms = replicas.max_over_ranks(statistics.median(time_each(step, nsteps, stream, torch)), dev)
    Nv, pv = [N] * n, [p] * n
    b_f, _ = batched_solve_model(Nv, pv, cyc_f, "mixed")
    b_a, _ = batched_solve_model(Nv, pv, cyc_a, "mixed")
    nbytes = b_f + b_a + 16 * n * N * (p + 1)      # + the gradient reductions (read mu, u)
    out["adjoint_4096x16384_p2"] = {
        "unit": "DoF/s (forward + adjoint)", "instances": n_all, "N": N, "p_t": p,
        "value": n_all * N * (p + 1) / (ms * 1e-3), "gradients_per_s": 1e3 / ms,
        "ms_per_step": round(ms, 3), "solves_timed": nsteps,
        "forward_max_cycles": int(np.max(cyc_f)),
        "adjoint_max_cycles": int(replicas.max_over_ranks(mx, dev)),
        "forward_err_vs_fp64": {"max": float(np.max(err_f)), "median": float(np.median(err_f))},
        "precision": "mixed", "cycle": f"V{NU}",
        "roofline": whole_solve_roofline(ms, nbytes, 0, hbm_peak, peak_kind,
                                         "forward + adjoint solves as the mixed batched model, plus the gradient "
                                         "reductions (read mu, u: 16 B/DoF); the reversals of g and mu and the "
                                         "loss gradient in torch are not counted")}
    del f, u, u0, y
    torch.cuda.empty_cache()
    return out


def _oracle_worker(task):
    """One host process of the instance-parallel oracle baseline: assemble the
    load vectors of its instances, then time the oracle's textbook multigrid
    (the same V-cycle, tolerance and coarsening) and its forward substitution
    on them, one instance after the other."""
    import numpy as np

    import oracle
    from paper_1409_5254_gb300 import inputs
    items, nu, tol = task
    Fs = [inputs.load_vector(p, N, T, inputs.Forcing(A, K, T)) for (p, N, T, z, u0, A, K) in items]
    dofs = sum(N * (p + 1) for (p, N, T, z, u0, A, K) in items)
    t0 = time.perf_counter()
    for (p, N, T, z, u0, A, K), F in zip(items, Fs):
        oracle.mg_solve(p, z, F, u0, tol=tol, max_cycles=300, nu1=nu[0], nu2=nu[1], n_min=64)
    t_mg = time.perf_counter() - t0
    t0 = time.perf_counter()
    for (p, N, T, z, u0, A, K), F in zip(items, Fs):
        oracle.fsub(p, z, F, u0)
    t_fs = time.perf_counter() - t0
    return dofs, t_mg, t_fs


def _oracle_batch(items, cores: int, note: str):
    """The oracle over `items` = (p, N, T, z, u0, amps, freqs) instances,
    instance-parallel over `cores` host processes (spawned: the parent holds a
    CUDA context), largest instances dealt first round-robin.  The parallel
    rate is all DoFs over the slowest process's time."""
    import multiprocessing as mp
    order = sorted(range(len(items)), key=lambda i: -items[i][1] * (items[i][0] + 1))
    tasks = [([items[i] for i in order[w::cores]], NU, TOL) for w in range(cores)]
    tasks = [t for t in tasks if t[0]]
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        res = pool.map(_oracle_worker, tasks)
    dofs = sum(r[0] for r in res)
    t_mg = max(r[1] for r in res)
    t_fs = max(r[2] for r in res)
    return {"value": dofs / t_mg, "unit": "DoF/s", "cores": len(tasks), "kind": "oracle",
            "sample": f"{note}; {len(items)} instances, {dofs} DoFs, textbook V{NU} multigrid to {TOL} on every "
                      f"host core ({t_mg:.2f} s on the slowest)",
            "single_core_value": dofs / sum(r[1] for r in res),
            "fsub_value": dofs / t_fs, "fsub_note": "exact forward substitution, same instances and cores"}


def cpu_baseline(sample_N: int = 1 << 21, batched: bool = True):
    """The FP64 oracle as it stands on the GPU machine's host cores.  The long
    horizon: textbook multigrid, one host thread, on the first sample_N
    intervals of the same workload (same tau, lambda, p_t, forcing).  The
    batched workloads: instance-parallel over all host cores on a stated
    fraction of their instances."""
    import numpy as np

    import oracle
    from paper_1409_5254_gb300 import inputs

    d = P_MAIN + 1
    T = N_FULL * TAU
    forcing = inputs.Forcing.draw(np.random.default_rng(1), T)
    F = _sample_load_vector(P_MAIN, sample_N, T, forcing)
    t0 = time.perf_counter()
    _, hist = oracle.mg_solve(P_MAIN, LAM * TAU, F, U0, tol=TOL, max_cycles=100, nu1=NU[0], nu2=NU[1],
                              n_min=n_min_for(F.shape[0]))
    t_mg = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.fsub(P_MAIN, LAM * TAU, F, U0)
    t_fs = time.perf_counter() - t0
    out = {"value": sample_N * d / t_mg, "unit": "DoF/s", "cores": 1, "kind": "oracle",
           "sample": f"first {sample_N} of the 2^24 intervals, textbook V{NU} multigrid to 1e-10 ({len(hist) - 1} cycles), "
                     f"{t_mg:.2f} s",
           "fsub_value": sample_N * d / t_fs, "fsub_note": "exact forward substitution, same sample"}
    if batched:
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        b = {}
        lam, amps, freqs = inputs.heat_modes_batch(2, 256, 4096, 1)
        sel = range(0, len(lam), 32)
        b["heat_modes_65536x4096_p1"] = _oracle_batch(
            [(1, 4096, 1.0, float(lam[i]) / 4096, 0.0, amps[i], freqs[i]) for i in sel], cores,
            "every 32nd of the 65,536 heat modes")
        Nv, pv, z = inputs.uneven_batch(3, 10000)
        A, K = inputs.sinusoid_batch_params(3, len(Nv))
        b["uneven_10000"] = _oracle_batch(
            [(int(pv[i]), int(Nv[i]), 1.0, float(z[i]), 1.0, A[i], K[i]) for i in range(0, len(Nv), 10)], cores,
            "every 10th of the 10,000 uneven instances")
        lam, u0, _ = inputs.adjoint_problem(4, 4096, 16384, 2)
        A, K = inputs.sinusoid_batch_params(4, 4096)
        b["adjoint_4096x16384_p2_forward"] = _oracle_batch(
            [(2, 16384, 1.0, float(lam[i]) / 16384, float(u0[i]), A[i], K[i]) for i in range(0, 4096, 64)], cores,
            "forward solves of every 64th of the 4096 gradient instances")
        out["batched"] = b
    return out


def _sample_load_vector(p, n, T, forcing):
    """Load vector of the first n intervals of the 2^24-interval mesh (same step)."""
    from paper_1409_5254_gb300 import inputs
    return inputs.load_vector(p, N_FULL, T, forcing, n_stop=n)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_1409_5254_gb300 import inputs

    n = 1 << 16
    d = P_MAIN + 1
    T = N_FULL * TAU
    forcing = inputs.Forcing.draw(np.random.default_rng(1), T)
    F = _sample_load_vector(P_MAIN, n, T, forcing)
    for _ in range(args.warmup):
        oracle.mg_solve(P_MAIN, LAM * TAU, F, U0, tol=TOL, max_cycles=100, nu1=NU[0], nu2=NU[1],
                        n_min=n_min_for(F.shape[0]))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, hist = oracle.mg_solve(P_MAIN, LAM * TAU, F, U0, tol=TOL, max_cycles=100, nu1=NU[0], nu2=NU[1],
                              n_min=n_min_for(F.shape[0]))
    dt = (time.perf_counter() - t0) / args.steps
    value = n * d / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_FULL, "p_t": P_MAIN, "tau": TAU, "lambda": LAM, "tol": TOL},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n} of the 2^24 intervals per step, textbook V{NU} multigrid "
                                       f"({len(hist) - 1} cycles)"},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the FP64-form and other-degree side runs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--traffic", type=float, default=None, help="ncu DRAM bytes per launch of the dominant kernel")
    ap.add_argument("--eager", action="store_true", help="host-driven cycle loop instead of the CUDA graph (profiling: "
                    "ncu does not profile the kernels of a graph with conditional nodes one by one)")
    ap.add_argument("--n-log2", type=int, default=24, help="intervals = 2^n (smaller cases for ncu captures)")
    ap.add_argument("--p-t", type=int, default=1, help="degree of the long-horizon line (profiling other degrees "
                    "with --quick; the benchmark line is p_t = 1)")
    ap.add_argument("--workload", default="all", choices=["all", "heat", "uneven", "gradients", "space_time_heat"],
                    help="all: the benchmark line; otherwise only that batched workload, or the space-time heat "
                         "equation (profiling)")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"],
                    help="forms of the batched workloads run with --workload")
    ap.add_argument("--heat-n-log2", type=int, default=12,
                    help="intervals of the space-time heat line = 2^k (smaller cases for ncu captures)")
    ap.add_argument("--batch-stride", type=int, default=1,
                    help="with --workload heat: every s-th mode only (smaller cases for ncu captures)")
    args = ap.parse_args()
    global BATCH_STRIDE
    BATCH_STRIDE = max(1, args.batch_stride) if args.workload == "heat" else 1
    global N_FULL, P_MAIN, HEAT_N
    N_FULL = 1 << args.n_log2
    HEAT_N = 1 << args.heat_n_log2
    P_MAIN = args.p_t
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "space_time_heat":
        run_space_time_heat(args)
    elif args.workload != "all":
        run_one_batched(args)
    else:
        run_ours(args)


def run_one_batched(args):
    """One batched workload alone, one GPU (for profiling its kernels)."""
    import torch
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    prec = ("mixed", "fp64") if args.precision == "both" else (args.precision,)
    out = run_batched_configs(dev, stream, args.steps, torch, only=(args.workload,), precisions=prec,
                              eager=args.eager)
    print(json.dumps(out))


def run_space_time_heat(args):
    """The space-time heat line alone, one GPU (for profiling its kernels)."""
    import torch
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()
    print(json.dumps(_space_time_heat(dev, stream, max(3, args.steps), torch, hbm_peak, peak_kind, args.eager)))


if __name__ == "__main__":
    main()
