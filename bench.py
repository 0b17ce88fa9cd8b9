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
METRIC = "time-DoFs/s solved to 1e-10 rel residual"
WORKLOAD = ("long horizon u'+lambda u=f, lambda=1, tau=1e-6, N=2^24, p_t=1, mixed FP32 cycles + FP64-accurate "
            "refinement, V(2,2), omega*, coarsest level 2^17 intervals solved by the parallel affine scan")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one k_updown0
# launch on the default workload, from one ncu capture; valid only for the
# kernel source it was taken with (first 16 hex digits of the SHA-256 of
# tmg_kernels.cuh), else null.
BATCH_STRIDE = 1          # every s-th heat mode (profiling of smaller cases only)
UPDOWN0_TRAFFIC = {"bytes_per_launch": 1.0180e9, "kernels_sha256": "34384092ae2de274"}


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


def time_solves(plan, F, u, steps: int, stream, torch):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        plan.solve(F, U0, u)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps


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
                    nu1=NU[0], nu2=NU[1], n_min=N_MIN)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    for _ in range(args.warmup):
        plan.solve(F, U0, u)
    st = plan.stats()
    info = plan.info()

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ms = time_solves(plan, F, u, args.steps, stream, torch)
    clk.stop()
    ms = replicas.max_over_ranks(ms, dev)
    st = plan.stats()
    value = replicas.aggregate_throughput([N_FULL * d] * world, ms)    # one replica per rank

    # accuracy of the timed result, in FP64 on the GPU (residual entry point)
    r = plan.residual(F, U0, u)
    Fh = torch.from_numpy(prob["F"].copy()).to(dev)
    Fh[0, 0] += U0
    Fh[0, 1] -= U0
    rel_fp64 = float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(Fh))
    del r, Fh

    # exact FP64 solve by the parallel affine scan: the error of the timed
    # result, and the direct solve as a throughput ceiling (one pass to reduce
    # each tile of F, one to replay it: reads F twice, writes u once)
    u_ex = plan.solve_direct(F, U0)
    err_vs_fp64 = float((u - u_ex).abs().max() / u_ex.abs().max())
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    n_dir = max(3, args.steps // 2)
    start.record(stream)
    for _ in range(n_dir):
        plan.solve_direct(F, U0, u_ex)
    end.record(stream)
    end.synchronize()
    ms_dir = start.elapsed_time(end) / n_dir
    dir_bytes = 3 * N_FULL * d * 8
    # FP64 operations (an FMA or an add counts one) per interval: pass 1 c^T f and
    # the map composition (d + 2), pass 3 c^T f, A^{-1} f + g e and the carry
    # (d^2 + 2d + 1); the peak is 2 FP64 FMA per clock per SM (1.25 TFLOP/s
    # nominal) at 152 SMs x 2.07 GHz
    fp64_ops = N_FULL * (d * d + 3 * d + 3)
    fp64_peak = 152 * 2 * 2.07e9
    direct = {"value": N_FULL * d / (ms_dir * 1e-3), "unit": "DoF/s", "ms_per_step": round(ms_dir, 4),
              "precision": "fp64", "bytes_per_dof": 24, "lower_bound_bytes_per_dof": 16,
              "hbm_frac": round(dir_bytes / (ms_dir * 1e-3) / 1e9 / hbm_peak, 4),
              "roofline": {"bound": "alu", "achieved": round(fp64_ops / (ms_dir * 1e-3) / 1e9, 1),
                           "peak": round(fp64_peak / 1e9, 1), "unit": "G FP64 ops/s",
                           "frac": round(fp64_ops / (ms_dir * 1e-3) / fp64_peak, 4), "peak_kind": "nominal"},
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
                "bytes_per_launch": cb["updown0"], "launch_ms": round(t_dom, 5), "launches_per_solve": st.cycles,
                "cycle_bytes": cb["cycle"], "cycle_ms": round(steady_ms, 5),
                "cycle_frac": round(cb["cycle"] / (steady_ms * 1e-3) / 1e9 / hbm_peak, 4),
                "solve_ms_per_cycle": round(ms / max(st.cycles, 1), 5),
                "kernel_ms": {"down0_confirm_once_per_solve": round(prof["down0"], 5),
                              "down_levels": round(prof["down_levels"], 5),
                              "coarsest_solve": round(prof["coarse_on_chip"], 5),
                              "up_levels": round(prof["up_levels"], 5), "updown0": round(prof["up0"], 5),
                              "cycle_events": round(prof["cycle"], 5)}}

    # every kernel of the graph body launches in each of the cycles + 1 loop iterations
    launches = args.steps * (st.cycles + 1) * plan.launches_per_cycle()

    extra = {}
    if rank == 0 and not args.quick:
        # plain FP64 form on the same problem
        with tmg.Plan(P_MAIN, TAU, LAM, N_FULL, precision="fp64", tol=TOL, stream=stream, nu1=NU[0], nu2=NU[1],
                      n_min=N_MIN, use_graph=not args.eager) as p64:
            p64.solve(F, U0, u)
            ms64 = time_solves(p64, F, u, max(2, args.steps // 4), stream, torch)
            s64 = p64.stats()
        extra["fp64_form"] = {"value": N_FULL * d / (ms64 * 1e-3), "ms_per_step": round(ms64, 4),
                              "cycles": s64.cycles, "rel_res": s64.rel_res}
        # the other degrees of the same long horizon, mixed precision
        per_p = {}
        for p in (0, 2, 3, 4, 5):
            pr = inputs.scalar_problem(1, N_FULL, p, lam=LAM, tau=TAU, u0=U0)
            Fp = torch.from_numpy(pr["F"]).to(dev)
            up = torch.empty_like(Fp)
            try:
                with tmg.Plan(p, TAU, LAM, N_FULL, precision="mixed", tol=TOL, stream=stream, max_cycles=300,
                              nu1=NU[0], nu2=NU[1], n_min=n_min_p(p),
                              use_graph=not args.eager) as pp:
                    pp.solve(Fp, U0, up)
                    msp = time_solves(pp, Fp, up, max(2, args.steps // 4), stream, torch)
                    sp = pp.stats()
                    per_p[str(p)] = {"value": N_FULL * (p + 1) / (msp * 1e-3), "ms_per_step": round(msp, 4),
                                     "cycles": sp.cycles, "rel_res": sp.rel_res, "cycle": f"V{NU}",
                                     "coarsest_intervals": pp.info()["tail_intervals"]}
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
            with tmg.Plan(P_MAIN, tau2, LAM, N_FULL, precision="mixed", tol=TOL, stream=stream, max_cycles=300,
                          nu1=NU[0], nu2=NU[1], n_min=N_MIN, use_graph=not args.eager) as pp:
                pp.solve(Fp, U0, up)
                msp = time_solves(pp, Fp, up, max(2, args.steps // 4), stream, torch)
                sp = pp.stats()
                extra["tau_1_1024"] = {"value": N_FULL * d / (msp * 1e-3), "ms_per_step": round(msp, 4),
                                       "cycles": sp.cycles, "rel_res": sp.rel_res, "z": LAM * tau2,
                                       "cycle": f"V{NU}"}
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
            key = f"p10_{prec}"
            try:
                with tmg.Plan(10, TAU, LAM, N_FULL, precision=prec, tol=TOL, stream=stream, max_cycles=300,
                              nu1=NU[0], nu2=NU[1], n_min=64, use_graph=not args.eager) as pp:
                    pp.solve(Fp, U0, up)
                    msp = time_solves(pp, Fp, up, 2, stream, torch)
                    sp = pp.stats()
                    extra[key] = {"value": N_FULL * 11 / (msp * 1e-3), "ms_per_step": round(msp, 4),
                                  "cycles": sp.cycles, "rel_res": sp.rel_res, "cycle": f"V{NU}",
                                  "levels": pp.info()["levels"],
                                  "coarsest_intervals": pp.info()["tail_intervals"]}
            except tmg.TmgError as e:
                extra[key] = {"error": str(e)}
        del Fp, up
        # other sweep counts on the headline problem (same solver, same tolerance)
        nus = {}
        for nu in ((1, 1), (1, 3), (2, 3), (3, 3)):
            with tmg.Plan(P_MAIN, TAU, LAM, N_FULL, precision="mixed", tol=TOL, stream=stream, nu1=nu[0],
                          nu2=nu[1], n_min=N_MIN, use_graph=not args.eager) as pn:
                pn.solve(F, U0, u)
                msn = time_solves(pn, F, u, max(2, args.steps // 4), stream, torch)
                sn = pn.stats()
            nus[f"V({nu[0]},{nu[1]})"] = {"value": N_FULL * d / (msn * 1e-3), "ms_per_step": round(msn, 4),
                                           "cycles": sn.cycles, "rel_res": sn.rel_res}
        extra["nu_variants"] = nus

    if not args.quick:
        # every rank solves its shard of the batched workloads
        extra_b = run_batched_configs(dev, stream, args.steps, torch, rank, world)
        if rank == 0:
            extra["batched"] = extra_b

    # end to end through the host-array entry point (pinned buffers, copies inside the call)
    F_h = torch.from_numpy(prob["F"]).pin_memory()
    u_h = torch.empty_like(F_h).pin_memory()
    plan.solve_host(F_h, U0, u_h)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    n_e2e = max(3, args.steps // 2)
    for _ in range(n_e2e):
        plan.solve_host(F_h, U0, u_h)
    t_e2e = replicas.max_over_ranks((time.perf_counter() - t0) / n_e2e, dev)
    nbytes = N_FULL * d * 8
    e2e = {"value": replicas.aggregate_throughput([N_FULL * d] * world, t_e2e * 1e3), "unit": "DoF/s",
           "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes, "ms_per_step": round(t_e2e * 1e3, 3)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    plan.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
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


def _time_batch(batch, f, u0, u, steps, stream, torch):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        batch.solve(f, u0, u)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps


def run_batched_configs(dev, stream, steps, torch, rank: int = 0, world: int = 1,
                        only=("heat", "uneven", "gradients"), precisions=("mixed", "fp64"), eager=False):
    """The batched workloads: decoupled 2-D heat modes, an uneven batch, and
    gradients through the adjoint.  One step = one batched solve (plus the
    adjoint for the gradient workload); inputs resident in HBM.  With several
    ranks each solves its shard of the instances (balanced by N (p_t+1)); the
    value is all instances' DoFs over the slowest rank's time.  `only` and
    `precisions` select workloads and forms (for profiling one of them)."""
    import numpy as np
    from paper_1409_5254_gb300 import inputs, replicas, tmg

    def shard(weights):
        return replicas.partition_instances(weights, world)[rank]

    out = {}
    if "heat" in only:
        out.update(_heat_modes(dev, stream, steps, torch, shard, precisions, eager))
    if "uneven" in only:
        out.update(_uneven(dev, stream, steps, torch, shard, precisions, eager))
    if "gradients" in only:
        out.update(_gradients(dev, stream, steps, torch, shard, eager))
    if world > 1:
        out["sharding"] = f"instances split over {world} ranks (no data exchange), weak in per-rank time"
    return out


def _heat_modes(dev, stream, steps, torch, shard, precisions, eager):
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
        with tmg.Batch([p] * n, 1.0 / N, lam, N, precision=prec, tol=TOL, max_cycles=200, stream=stream,
                       nu1=NU[0], nu2=NU[1], use_graph=not eager) as B:
            B.solve(f, u0, u)
            ms = _time_batch(B, f, u0, u, max(1, steps // 10) if prec == "mixed" else 1, stream, torch)
            cyc, rel, mx = B.stats()
        ms = replicas.max_over_ranks(ms, dev)
        mx = replicas.max_over_ranks(mx, dev)
        worst = replicas.max_over_ranks(float(rel.max()), dev)
        res[prec] = {"value": n_all * N * (p + 1) / (ms * 1e-3), "ms_per_step": round(ms, 3), "max_cycles": int(mx),
                     "max_rel_res": worst}
    out["heat_modes_65536x4096_p1" if BATCH_STRIDE == 1 else f"heat_modes_{n_all}x4096_p1"] = {"unit": "DoF/s", "instances": n_all, "N": N, "p_t": p,
                                       "lambda_range": [float(lam_all.min()), float(lam_all.max())], **res}
    del f, u, u0
    torch.cuda.empty_cache()
    return out


def _uneven(dev, stream, steps, torch, shard, precisions, eager):
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
        torch.cuda.synchronize()
        t_setup = time.perf_counter()
        with tmg.Batch(pv, tau, lamv, Nv, precision=prec, tol=TOL, max_cycles=300, stream=stream,
                       nu1=NU[0], nu2=NU[1], use_graph=not eager) as B:
            setup_ms = (time.perf_counter() - t_setup) * 1e3
            B.solve(f, u0, u)
            ms = _time_batch(B, f, u0, u, max(1, steps // 10), stream, torch)
            cyc, rel, mx = B.stats()
            info = B.info()
        ms = replicas.max_over_ranks(ms, dev)
        kinds = [g["schedule"] for g in info["group_info"]]
        res[prec] = {"value": dofs / (ms * 1e-3), "ms_per_step": round(ms, 3),
                     "max_cycles": int(replicas.max_over_ranks(mx, dev)),
                     "max_rel_res": replicas.max_over_ranks(float(rel.max()), dev),
                     "setup_ms_with_autotune": round(setup_ms, 1),
                     "groups_cta": kinds.count("cta"), "groups_grid": kinds.count("grid"),
                     "autotune_whole_batch_ms": {k: (round(v, 3) if v == v else None)
                                                 for k, v in info["whole_batch_ms"].items()}}
    out["uneven_10000"] = {"unit": "DoF/s", "instances": len(Nv_all), "dofs": dofs, "groups": info["groups"],
                           "padded_dofs": info["padded_values"], **res}
    del f, u, u0
    torch.cuda.empty_cache()
    return out


def _gradients(dev, stream, steps, torch, shard, eager):
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
        step()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        k = max(1, steps // 10)
        start.record(stream)
        for _ in range(k):
            step()
        end.record(stream)
        end.synchronize()
        ms = replicas.max_over_ranks(start.elapsed_time(end) / k, dev)
        cyc, rel, mx = B.stats()
    out["adjoint_4096x16384_p2"] = {"unit": "DoF/s (forward + adjoint)", "instances": n_all, "N": N, "p_t": p,
                                    "value": n_all * N * (p + 1) / (ms * 1e-3), "gradients_per_s": 1e3 / ms,
                                    "ms_per_step": round(ms, 3),
                                    "adjoint_max_cycles": int(replicas.max_over_ranks(mx, dev)),
                                    "precision": "mixed", "cycle": f"V{NU}"}
    del f, u, u0, y
    torch.cuda.empty_cache()
    return out


def cpu_baseline(sample_N: int = 1 << 21):
    """The FP64 oracle as it stands (textbook multigrid, one host thread) on the
    first sample_N intervals of the same workload (same tau, lambda, p_t, forcing)."""
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
    return {"value": sample_N * d / t_mg, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"first {sample_N} of the 2^24 intervals, textbook V{NU} multigrid to 1e-10 ({len(hist) - 1} cycles), "
                      f"{t_mg:.2f} s",
            "fsub_value": sample_N * d / t_fs, "fsub_note": "exact forward substitution, same sample"}


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
    ap.add_argument("--workload", default="all", choices=["all", "heat", "uneven", "gradients"],
                    help="all: the benchmark line; otherwise only that batched workload (profiling)")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"],
                    help="forms of the batched workloads run with --workload")
    ap.add_argument("--batch-stride", type=int, default=1,
                    help="with --workload heat: every s-th mode only (smaller cases for ncu captures)")
    args = ap.parse_args()
    global BATCH_STRIDE
    BATCH_STRIDE = max(1, args.batch_stride) if args.workload == "heat" else 1
    global N_FULL
    N_FULL = 1 << args.n_log2
    if args.impl == "reference":
        run_reference(args)
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


if __name__ == "__main__":
    main()
