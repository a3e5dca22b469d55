#!/usr/bin/env python
"""Seconds per time step of the NEAREST regularized-stokeslet swimming
problem on GB300.

One step = one explicit-midpoint (RK2) step of the single free undulating
swimmer (N = 800 force points, Q = 8000 quadrature points, eps = 0.005,
n = 2406 unknowns): twice (kinematics, nearest neighbours, segments, FP64
assembly, rigid-body border, explicit FP32 inverse by blocked Gauss-Jordan
with split-TF32 tensor-core updates, FP64 GMRES-based iterative refinement to
the FP64 answer as one cooperative launch) plus the state update, recorded once
into a CUDA graph and replayed.  Inputs are the seeded synthetic beat shapes of
`synth` (the paper's cited beat patterns are not available), resident in HBM
before the timed region.  Beside the headline: the same step launched kernel by
kernel, with the host-driven refinement loop, with factor reuse, with the
learned start, the plain FP64 path, and (N = 1) the batch workload of many
uneven problems in one graph.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nrs|reference]
                    [--prec tf32|fp32|fp64]
    python bench.py --profile-solve --workload swimmer_mid   # one solve, for ncu
    python bench.py --no-batch --no-cpu-baseline             # the C1 lines only
    python bench.py --batch-full                             # all 128 full-size batch problems

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the same workload.  Under torchrun each rank runs its own replica of the
problem ("replicas only": one dense solve does not shard across GPUs).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import geometry as g  # noqa: E402
from synth import mlp_init  # noqa: E402

METRIC = "s per timestep (assemble+solve) mixed-IR vs FP64 at 1e-10 rel err; pairs/s"
WORKLOAD = "single free undulating swimmer, N=800 force / Q=8000 quadrature points, eps=0.005, n=2406"
L2_FLUSH_BYTES = 512 << 20
FP64_NOMINAL_TFLOPS = 1.25       # GB300 FP64 (vector and tensor), nominal
TF32_OVER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor throughput
SM_COUNT_NOMINAL = 152
MLP_TRAIN_ITERS = 4              # Adam steps per stage for the learned starting vector
MLP_LR = 3e-3
FP32_LANES_PER_SM = 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest x over the ranks of the default process group (x itself
    on one rank): the whole job's time is that of its slowest rank."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _rank_share(costs, ws: int, rank: int):
    """The problems a rank steps when a batch is split over ws ranks: the
    longest-processing-time-first plan of the library (nrs_batch_plan) with
    one chain per rank, no collective in the data path."""
    from paper_2001_06468_gb300 import nrs
    chain_of, _ = nrs.batch_plan(list(costs), ws)
    return [i for i, ch in enumerate(chain_of) if ch == rank]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=float(max(smax)),
                       reasons=sorted(reasons), samples=len(sm))
        return out


def _visible_gpu_index(local: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if parts and parts[local if local < len(parts) else 0].strip().isdigit():
        return int(parts[local if local < len(parts) else 0])
    return local


def _shapes_host(pr, t):
    import torch
    d = g.pack_shapes(pr, t)
    return tuple(torch.from_numpy(d[k]).pin_memory() for k in ("x", "Xw", "xidot"))


# DRAM bytes per launch from one ncu capture (profiles/), valid while the
# kernel's source file is unchanged (first 12 hex digits of its SHA-1).
NCU_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch, from the captures summarised
    # in profiles/ (kept only while the kernel's source is the one captured)
    "k_gj_diag": {"bytes": 136832, "file": "paper_2001_06468_gb300/csrc/gj.cu",
                  "sha1": "d098875a34c5",
                  "scale": "none (the 64 x 64 block, the previous D^{-1} and two 64 x 64 tiles at any n)"},
    "k_tc_gj_update": {"bytes": 150743296 + 77540181, "n": 6006,
                       "file": "paper_2001_06468_gb300/csrc/tc_gemm.cu", "sha1": "e38e9748bdee",
                       "scale": "n^2 (captured at n = 6006)"},
    "k_gj_fused": {"bytes": None, "file": "paper_2001_06468_gb300/csrc/gj.cu",
                   "sha1": "", "scale": None},
    # captured at n = 6006 (matrices larger than L2): DRAM bytes = 1.003 x the algorithmic bytes;
    # at n = 2406 the matrices stay in L2, so that figure does not carry over: not reported
    "k_gmres_ir": {"bytes": None, "file": "paper_2001_06468_gb300/csrc/gmres_persistent.cu",
                   "sha1": "f0099c63014a", "scale": None},
    "k_assemble64": {"bytes": None, "file": "paper_2001_06468_gb300/csrc/assemble.cu",
                     "sha1": "fcf536ee0b72", "scale": None},
}


def _traffic(kernel, n):
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if not rec or rec["bytes"] is None:
        return None
    src = open(os.path.join(ROOT, rec["file"]), "rb").read()
    if hashlib.sha1(src).hexdigest()[:12] != rec["sha1"]:
        return None  # the kernel changed since the counters were taken
    if "n" in rec:
        return rec["bytes"] * (n / rec["n"]) ** 2
    return rec["bytes"]


def _rooflines(ph_ms, ph_spans, pr, peaks, peak_src, clocks, solve_stats=None):
    """Roofline records of the kernel families of the step, from the live
    per-phase CUDA-event times.  Algorithmic work per launch:
      k_gj_diag       2*64^3 flops (inverse) + 6*64^3 (lookahead: R = Dprev M[P,K],
                      D -= M[K,P] R, and the staged tile -M[K,P] Dprev); the first
                      block of a factorisation has no lookahead (2*64^3)
      k_tc_gj_update  8 n^2 bytes (read and write of the FP32 matrix), HBM-bound at K = 64
      k_assemble64    29 FP64 operations per (force point, quadrature point) pair
      k_gemv_part     8 n^2 bytes (FP64 matrix)
      k_gemv32_part   4 n^2 bytes (FP32 explicit inverse)
      k_gmres_ir      8 n^2 (outer + inner) + 4 n^2 (outer + inner + 1) bytes per solve"""
    n = pr.n
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    fp64_peak = FP64_NOMINAL_TFLOPS * sm_mhz / 2070.0
    tf32_peak = peaks["bf16_tflops_sustained"] * TF32_OVER_BF16

    def per_launch(ph):
        return ph_ms[ph] / 1e3 / max(ph_spans[ph], 1)

    recs = {}
    if ph_spans["lu_diag"] == 0 and ph_spans["lu_update"] > 0:
        # the fused factorisation: one cooperative launch per inversion, timed
        # as the lu_update phase; every block step reads and writes the FP32
        # matrix once (8 n^2 bytes), its critical path is the chain of the
        # nblk diagonal inverses on one CTA
        t = per_launch("lu_update")
        nblk = -(-n // 64)
        b = 8.0 * n * n * nblk
        recs["lu_update"] = {
            "kernel": "k_gj_fused (the whole Gauss-Jordan inversion in one cooperative launch: "
                      "the diagonal-inverse chain on one CTA, prep/finish and the tcgen05 "
                      "3xTF32 rank-64 updates on the others)",
            "bound": "hbm", "achieved": b / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": b / t / 1e9 / peaks["hbm_gbs"],
            "peak_source": peak_src + " (HBM copy; the FP32 matrix is L2-resident at this size)",
            "work_per_launch": b,
            "tensor_tflops": 2.0 * n * n * 64 * nblk / t / 1e12,
            "tensor_frac_of_tf32": 2.0 * n * n * 64 * nblk / t / 1e12 / tf32_peak,
            "us_per_block": t / nblk * 1e6, "blocks": nblk,
            "latency_bound": "the chain of diagonal inverses (64 dependent pivot steps each)",
            "launches": ph_spans["lu_update"], "traffic": _traffic("k_gj_fused", n)}
    else:
        _separate_factor_rooflines(recs, per_launch, ph_spans, n, peaks, peak_src, fp32_peak,
                                   tf32_peak, sm_mhz)
    _other_rooflines(recs, per_launch, ph_spans, pr, n, peaks, peak_src, fp64_peak, solve_stats)
    return recs


def _separate_factor_rooflines(recs, per_launch, ph_spans, n, peaks, peak_src, fp32_peak,
                               tf32_peak, sm_mhz):
    t = per_launch("lu_diag")
    nblk = -(-n // 64)
    w = (2.0 + 8.0 * (nblk - 1)) / nblk * 64 ** 3  # mean over one factorisation's launches
    sm_peak = fp32_peak / SM_COUNT_NOMINAL
    recs["lu_diag"] = {"kernel": "k_gj_diag (64 x 64 diagonal-block inverse, one CTA)",
                       "bound": "alu", "achieved": w / t / 1e12, "peak": sm_peak,
                       "unit": "TFLOP/s", "frac": w / t / 1e12 / sm_peak,
                       "peak_source": f"derived: ONE SM (the kernel is one CTA by construction: "
                                      f"64 dependent pivot steps), 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz; "
                                      f"{w / t / 1e12 / fp32_peak:.5f} of the whole GPU's FP32 peak",
                       "latency_bound": True,
                       "work_per_launch": w, "launches": ph_spans["lu_diag"],
                       "traffic": _traffic("k_gj_diag", n)}
    t = per_launch("lu_update")
    b = 8.0 * n * n
    recs["lu_update"] = {"kernel": "k_tc_gj_update (tcgen05 3xTF32 rank-64 update)",
                         "bound": "hbm", "achieved": b / t / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": b / t / 1e9 / peaks["hbm_gbs"],
                         "peak_source": peak_src + " (HBM copy)", "work_per_launch": b,
                         "tensor_tflops": 2.0 * n * n * 64 / t / 1e12,
                         "tensor_frac_of_tf32": 2.0 * n * n * 64 / t / 1e12 / tf32_peak,
                         "launches": ph_spans["lu_update"], "traffic": _traffic("k_tc_gj_update", n)}


def _other_rooflines(recs, per_launch, ph_spans, pr, n, peaks, peak_src, fp64_peak, solve_stats):
    t = per_launch("assemble")
    f = pr.pairs * 29.0
    recs["assemble"] = {"kernel": "k_assemble64 (NEAREST A_s, FP64)", "bound": "alu",
                        "achieved": f / t / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                        "frac": f / t / 1e12 / fp64_peak,
                        "peak_source": "nominal FP64 1.25 TFLOP/s at 2070 MHz, scaled to the clock",
                        "pairs_per_s": pr.pairs / t, "work_per_launch": f,
                        "launches": ph_spans["assemble"], "traffic": _traffic("k_assemble64", n)}
    if ph_spans["trsv"] > 0:  # host-driven refinement: separate product kernels
        t = per_launch("gemv")
        b = 8.0 * n * n
        recs["gemv"] = {"kernel": "k_gemv_part (FP64 residual / Arnoldi products)", "bound": "hbm",
                        "achieved": b / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": b / t / 1e9 / peaks["hbm_gbs"], "peak_source": peak_src,
                        "work_per_launch": b, "launches": ph_spans["gemv"], "traffic": None}
        t = per_launch("trsv")
        b = 4.0 * n * n
        recs["precond"] = {"kernel": "k_gemv32_part (explicit-inverse preconditioner)",
                           "bound": "hbm", "achieved": b / t / 1e9, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "frac": b / t / 1e9 / peaks["hbm_gbs"],
                           "peak_source": peak_src, "work_per_launch": b,
                           "launches": ph_spans["trsv"], "traffic": None}
    elif solve_stats and ph_spans["krylov"] > 0:
        # one persistent launch per solve: (outer + inner) FP64 products with A and
        # (outer + inner + 1) FP32 products with the explicit inverse per launch
        o, i = solve_stats["outer_mean"], solve_stats["inner_mean"]
        t = per_launch("krylov")
        b = 8.0 * n * n * (o + i) + 4.0 * n * n * (o + i + 1)
        recs["solve"] = {"kernel": "k_gmres_ir (persistent GMRES-IR, one cooperative launch per solve)",
                         "bound": "hbm", "achieved": b / t / 1e9, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": b / t / 1e9 / peaks["hbm_gbs"],
                         "peak_source": peak_src, "work_per_launch": b,
                         "fp64_tflops": 2.0 * n * n * (o + i) / t / 1e12,
                         "fp64_frac": 2.0 * n * n * (o + i) / t / 1e12 / fp64_peak,
                         "us_per_launch": t * 1e6,
                         "launches": ph_spans["krylov"], "traffic": _traffic("k_gmres_ir", n)}


def run_nrs(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2001_06468_gb300 import nrs

    pr = g.swimmer_config()
    dt = pr.dt
    K, W = args.steps, args.warmup
    total = K + W
    # body-frame beat shapes at t and t + dt/2 for every step, pinned on the host
    host = [(_shapes_host(pr, s * dt), _shapes_host(pr, (s + 0.5) * dt)) for s in range(total)]
    dev = [tuple(tuple(t.cuda() for t in st) for st in pair) for pair in host]
    Y0 = g.initial_state(pr)
    # the product path: the step recorded once into a CUDA graph and replayed
    # (graph mode); each step's shapes are first copied into the fixed
    # buffers the graph reads, inside the timed region
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, graph=True)
    ctx.set_state(Y0["x0"], Y0["B"])
    stream = ctx.stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    gbuf = tuple(tuple(torch.empty_like(t) for t in st) for st in dev[0])

    def do_step(ctx_, pair):
        s0 = nrs.Context.shapes(*pair[0])
        sh = nrs.Context.shapes(*pair[1])
        return ctx_.step(s0, sh, dt)

    def graph_step(ctx_, pair):
        for st_src, st_dst in zip(pair, gbuf):
            for src, dst in zip(st_src, st_dst):
                dst.copy_(src, non_blocking=True)
        return ctx_.step(nrs.Context.shapes(*gbuf[0]), nrs.Context.shapes(*gbuf[1]), dt,
                         report=False)

    def eager_step(ctx_, pair):
        return ctx_.step(nrs.Context.shapes(*pair[0]), nrs.Context.shapes(*pair[1]), dt,
                         report=False)

    reports = []
    for s in range(W):
        graph_step(ctx, dev[s])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]

    def timed_pass(ctx_, first, fn=do_step):
        ms = []
        for s in range(K):
            flush.fill_(float(s))  # evict L2 between timed steps (untimed)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                ev[s][0].record(stream)
                r = fn(ctx_, dev[first + s])
                ev[s][1].record(stream)
            if r is not None:
                reports.append(r)
            torch.cuda.synchronize()
            ms.append(ev[s][0].elapsed_time(ev[s][1]))
        return ms

    # the timed region: K steps, no instrumentation inside the library
    ctx.get_timing()  # clears the kernel count
    with ClockSampler(_visible_gpu_index(local)) as clk:
        step_ms = timed_pass(ctx, W, graph_step)
    clocks = clk.summary()
    _, launches = ctx.get_timing()
    # a second pass over the same inputs with CUDA events around every phase of
    # the step (on the stream each phase runs on): per-kernel durations for
    # the roofline, and the kernel count
    ctx_t = nrs.Context.from_problem(pr, factor_prec=args.prec)
    ctx_t.set_state(Y0["x0"], Y0["B"])
    for s in range(W):
        do_step(ctx_t, dev[s])
    torch.cuda.synchronize()
    ctx_t.set_timing(True)
    nrep_t = len(reports)
    step_ms_instr = timed_pass(ctx_t, W)
    phases, _ = ctx_t.get_timing()
    instr_reports = reports[nrep_t:]
    solve_stats = {
        "outer_mean": float(np.mean([r["stages"][i]["outer"] for r in instr_reports for i in (0, 1)])),
        "inner_mean": float(np.mean([r["stages"][i]["inner"] for r in instr_reports for i in (0, 1)]))}
    ctx_t.set_timing(False)
    t_local = sum(step_ms) / 1e3
    t_max = _max_over_ranks(t_local, ws)
    s_per_step = t_max / K / ws  # whole job: ws replicas each advance K steps

    # end to end through the C ABI from pinned host buffers: H2D of both
    # stages' shapes and D2H of the new state and both solutions, every step
    ctx_e = nrs.Context.from_problem(pr, factor_prec=args.prec, graph=True)
    ctx_e.set_state(Y0["x0"], Y0["B"])
    bufs = tuple(tuple(torch.empty_like(t, device="cuda") for t in st) for st in host[0])
    sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
    sol_h = torch.empty(2 * pr.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for st in host[0] for t in st)
    d2h = sol_h.numel() * 8 + pr.n_free * 12 * 8
    for s in range(W):
        for st_h, st_d in zip(host[s], bufs):
            for th, td in zip(st_h, st_d):
                td.copy_(th, non_blocking=True)
        ctx_e.step(nrs.Context.shapes(*bufs[0]), nrs.Context.shapes(*bufs[1]), dt, sol=sol,
                   report=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_ms = 0.0
    for s in range(K):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        with torch.cuda.stream(ctx_e.stream):
            e0.record(ctx_e.stream)
            for st_h, st_d in zip(host[W + s], bufs):
                for th, td in zip(st_h, st_d):
                    td.copy_(th, non_blocking=True)
            ctx_e.step(nrs.Context.shapes(*bufs[0]), nrs.Context.shapes(*bufs[1]), dt, sol=sol,
                       report=False)
            sol_h.copy_(sol, non_blocking=True)
            st = ctx_e.get_state()
            e1.record(ctx_e.stream)
        torch.cuda.synchronize()
        e_ms += e0.elapsed_time(e1)
    e2e_s = e_ms / 1e3 / K / ws

    # plain FP64 path (FP64 factor) on the same steps, for the mixed-vs-plain ratio
    ctx_p = nrs.Context.from_problem(pr, factor_prec="fp64")
    ctx_p.set_state(Y0["x0"], Y0["B"])
    Kp = min(K, 5)
    do_step(ctx_p, dev[0])
    torch.cuda.synchronize()
    p_ms = 0.0
    for s in range(Kp):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        with torch.cuda.stream(ctx_p.stream):
            e0.record(ctx_p.stream)
            do_step(ctx_p, dev[W + s])
            e1.record(ctx_p.stream)
        torch.cuda.synchronize()
        p_ms += e0.elapsed_time(e1)
    plain_s = p_ms / 1e3 / Kp

    # the same mixed path with the host-driven refinement loop (one host
    # synchronisation per GMRES iteration) instead of the persistent solve
    ctx_h = nrs.Context.from_problem(pr, factor_prec=args.prec, solve_mode="host")
    ctx_h.set_state(Y0["x0"], Y0["B"])
    for s in range(W):
        do_step(ctx_h, dev[s])
    torch.cuda.synchronize()
    host_loop_s = float(np.sum(timed_pass(ctx_h, W))) / 1e3 / K / ws
    ctx_h.close()

    # the same step without the graph (kernels launched one by one)
    ctx_eg = nrs.Context.from_problem(pr, factor_prec=args.prec)
    ctx_eg.set_state(Y0["x0"], Y0["B"])
    for s in range(W):
        eager_step(ctx_eg, dev[s])
    torch.cuda.synchronize()
    eager_s = float(np.sum(timed_pass(ctx_eg, W, eager_step))) / 1e3 / K / ws
    ctx_eg.close()

    # factor reuse across stages + warm start (same inputs, same timing rules)
    ctx_r = nrs.Context.from_problem(pr, factor_prec=args.prec, reuse_factor=True, warm_start=True)
    ctx_r.set_state(Y0["x0"], Y0["B"])
    for s in range(W):
        do_step(ctx_r, dev[s])
    torch.cuda.synchronize()
    nrep = len(reports)
    r_ms = timed_pass(ctx_r, W)
    reuse_reports = reports[nrep:]
    reuse_s = float(np.sum(r_ms)) / 1e3 / K / ws

    # starting vectors of the refinement: cold (M^{-1} b), the previous stage's
    # solution, and the MLP prediction (trained during the run, on every
    # stage's solution; the timed steps include its training and selection)
    starts = {}
    for reuse in (False, True):
        for mode in ("cold", "previous", "learned"):
            ctx_s = nrs.Context.from_problem(pr, factor_prec=args.prec, reuse_factor=reuse,
                                             warm_start=(mode == "previous"))
            ctx_s.set_state(Y0["x0"], Y0["B"])
            if mode == "learned":
                ctx_s.mlp_set_params(mlp_init(0))
                ctx_s.mlp_config(train_iters=MLP_TRAIN_ITERS, predict=False, lr=MLP_LR)
            for s in range(W):
                do_step(ctx_s, dev[s])
            if mode == "learned":
                ctx_s.mlp_config(train_iters=MLP_TRAIN_ITERS, predict=True, lr=MLP_LR)
            torch.cuda.synchronize()
            nrep = len(reports)
            m_ms = timed_pass(ctx_s, W)
            reps = reports[nrep:]
            kinds = [k for r in reps for k in r["start"]]
            starts[("reuse_" if reuse else "fresh_") + mode] = {
                "s_per_step": float(np.sum(m_ms)) / 1e3 / K / ws,
                "inner_mean": float(np.mean([r["stages"][i]["inner"] for r in reps for i in (0, 1)])),
                "starts_used": {k: kinds.count(k) for k in sorted(set(kinds))},
                "mlp_rel_err_last": reps[-1]["mlp_rel_err"] if mode == "learned" else None,
            }
            ctx_s.close()

    # the first steps from the initial state, kept for the accuracy check
    # (fresh factor every stage, and factor reuse)
    sols = {}
    for name, kw in (("fresh", {}), ("reuse", {"reuse_factor": True, "warm_start": True})):
        ctx_a = nrs.Context.from_problem(pr, factor_prec=args.prec, **kw)
        ctx_a.set_state(Y0["x0"], Y0["B"])
        out = []
        for s in range(3):
            sol_a = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
            ctx_a.step(nrs.Context.shapes(*dev[s][0]), nrs.Context.shapes(*dev[s][1]), dt, sol=sol_a)
            out.append(sol_a.cpu().numpy())
        sols[name] = out

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    peaks, peak_src = _peaks()
    ph_ms = {k: v[0] for k, v in phases.items()}
    ph_spans = {k: v[1] for k, v in phases.items()}
    tot = sum(ph_ms.values())
    recs = _rooflines(ph_ms, ph_spans, pr, peaks, peak_src, clocks, solve_stats)
    top = max(recs, key=lambda p: ph_ms[{"precond": "trsv", "solve": "krylov"}.get(p, p)])
    roof = recs[top]
    asm = recs["assemble"]
    line = {
        "metric": METRIC,
        "value": s_per_step,
        "unit": "s/step",
        "n_gpus": ws,
        "steps": K,
        "warmup": W,
        "ms_per_step": t_max / K * 1e3,
        "ms_per_step_instrumented": float(np.mean(step_ms_instr)),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 residual + " + {"tf32": "split-TF32 tensor-core", "fp32": "fp32",
                                     "fp64": "fp64", "bf16": "bf16"}[args.prec] + " factor",
        "data": "synthetic (seeded undulating-tube beat shapes)",
        "config": {"workload": WORKLOAD, "factor": args.prec, "refinement": "GMRES-IR, FP64 residual",
                   "rk2_stages_per_step": 2, "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas x{ws}"},
        "pairs_per_s": asm.get("pairs_per_s"),
        "plain_fp64_s_per_step": plain_s,
        "mixed_vs_plain_speedup": plain_s / (t_max / K),
        "host_loop_refinement_s_per_step": host_loop_s,
        "eager_s_per_step": eager_s,
        "value_factor_reuse": reuse_s,
        "factor_reuse": {"s_per_step": reuse_s, "vs_plain_speedup": plain_s / (reuse_s * ws),
                         "factorizations_per_step": float(np.mean([r["factorizations"] for r in reuse_reports])),
                         "inner_mean": float(np.mean([r["stages"][i]["inner"] for r in reuse_reports for i in (0, 1)])),
                         "note": "the previous stages' factor preconditions the refinement until its GMRES "
                                 "count exceeds 8 or 16 stages pass; each solve from the previous solution"},
        "starts": starts,
        "starts_note": ("fresh_*: factor every stage; reuse_*: factor reuse. learned: "
                        f"{MLP_TRAIN_ITERS} Adam steps per stage (lr {MLP_LR}) on each stage's "
                        "solution, prediction used only where its residual beats the cold start's; "
                        "mlp_rel_err_last = held-out relative RMS error of the prediction of f"),
        "phases_ms_per_step": {k: v / K for k, v in ph_ms.items()},
        "phase_share": {k: (v / tot if tot else 0.0) for k, v in ph_ms.items()},
        "phase_note": ("the whole factorisation is one fused launch, timed as lu_update"
                       if ph_spans["lu_diag"] == 0 else
                       "lu_diag runs on a second stream, overlapping lu_update and lu_panel"),
        "refinement": {"outer_mean": solve_stats["outer_mean"], "inner_mean": solve_stats["inner_mean"],
                       "backward_err_max": float(max(r["stages"][i]["backward_err"] for r in instr_reports for i in (0, 1))),
                       "from": "the instrumented eager pass (same kernels, same inputs)"},
        "roofline": roof,
        "rooflines": recs,
        "e2e": {"value": e2e_s, "unit": "s/step", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "gpu_launches_note": "kernels of the recorded step graph replayed in the timed region, counted by the library",
        "clocks": clocks,
    }
    if not args.no_batch and ws == 1:
        line["batch"] = batch_bench(nrs, args)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(pr, sols)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def _oracle_step_timing(pr, max_steps, budget_s):
    import oracle as O
    Y = g.initial_state(pr)
    times, all_stages = [], []
    for s in range(max_steps):
        t0 = time.perf_counter()
        Yn, stages = O.rk2_step(pr, Y, s * pr.dt, pr.dt, return_stages=True)
        times.append(time.perf_counter() - t0)
        all_stages.append(stages)
        Y = Yn
        if sum(times) > budget_s:
            break
    return times, all_stages, O.threads()


def _batch_case(nrs, probs, prec, steps, tune=True, plan=None, seq_steps=None):
    """Seconds per batch step of ``probs`` through one recorded graph (K and G
    from the autotuner), and the same problems stepped one after the other
    on eager contexts, from the same initial states and inputs."""
    import torch
    dt = probs[0].dt
    host = [[tuple(torch.from_numpy(np.ascontiguousarray(sh[k])).cuda() for k in ("x", "Xw", "xidot"))
             for sh in (g.pack_shapes(pr, s * dt), g.pack_shapes(pr, (s + 0.5) * dt))]
            for s in range(steps + 2) for pr in probs]
    nprob = len(probs)

    def pairs_at(s):
        return [tuple(host[s * nprob + i]) for i in range(nprob)]

    batch = nrs.Batch(probs, factor_prec=prec)
    for c, pr in zip(batch.contexts, probs):
        Y = g.initial_state(pr)
        c.set_state(Y["x0"], Y["B"])
    bufs = [tuple(tuple(torch.empty_like(t) for t in st) for st in pair) for pair in pairs_at(0)]

    def load(s):
        for pair, buf in zip(pairs_at(s), bufs):
            for st_src, st_dst in zip(pair, buf):
                for src, dst in zip(st_src, st_dst):
                    dst.copy_(src, non_blocking=True)
        return bufs

    batch.step(load(0), dt)  # first step: nearest-neighbour maps, eager
    if plan is not None:
        batch.config(*plan)
    tuned = batch.tune(load(1), dt) if tune else batch.info()
    batch.step(load(1), dt)  # records the graph with the tuned plan
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream()
    ms = 0.0
    for s in range(steps):
        torch.cuda.synchronize()
        e0.record(st)
        batch.step(load(2 + s), dt)
        e1.record(st)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    info = batch.info()
    batch.close()
    # eager, one problem after the other
    ctxs = []
    for pr in probs:
        c = nrs.Context.from_problem(pr, factor_prec=prec)
        Y = g.initial_state(pr)
        c.set_state(Y["x0"], Y["B"])
        ctxs.append(c)
    seq_steps = steps if seq_steps is None else seq_steps
    for s in range(2):
        for i, c in enumerate(ctxs):
            a, b = pairs_at(s)[i]
            c.step(nrs.Context.shapes(*a), nrs.Context.shapes(*b), dt, report=False)
    torch.cuda.synchronize()
    ms_seq = 0.0
    for s in range(seq_steps):
        torch.cuda.synchronize()
        e0.record(st)
        for i, c in enumerate(ctxs):
            a, b = pairs_at(2 + s)[i]
            c.step(nrs.Context.shapes(*a), nrs.Context.shapes(*b), dt, report=False)
        e1.record(st)
        torch.cuda.synchronize()
        ms_seq += e0.elapsed_time(e1)
    for c in ctxs:
        c.close()
    ns = [pr.n for pr in probs]
    return {"problems": nprob, "n_min": min(ns), "n_max": max(ns), "n_mean": float(np.mean(ns)),
            "pairs": int(sum(pr.pairs for pr in probs)),
            "s_per_batch_step": ms / 1e3 / steps,
            "problem_steps_per_s": nprob * steps / (ms / 1e3),
            "sequential_eager_s_per_batch_step": ms_seq / 1e3 / seq_steps,
            "speedup_vs_sequential": (ms_seq / seq_steps) / (ms / steps), "steps": steps,
            "chains": info["chains"], "solve_grid": info["grid"],
            "graph_kernels": info["graph_kernels"],
            "tuned_ms": tuned.get("ms")}


def batch_bench(nrs, args):
    """The batch workload: 128 ventral-node-like problems at reduced sizes
    (all of them), and the first 8 at the full sizes."""
    small = [g.node_config(i, cilia=(4, 12), floor=(160, 500), n_rod=10, q_rod=100, n_sphere=2,
                           q_sphere=8) for i in range(128)]
    full = [g.node_config(i) for i in range(8)]
    return {"workload": "ventral-node batch: cilia rotating on tilted cones, static floor disc, "
                        "5 free spheres; eps 0.005",
            "reduced_128": dict(_batch_case(nrs, small, args.prec, 3),
                                recipe="cilia 4-12 (10/100 points), floor 160-500 (x10), spheres 26/386"),
            "full_first8": dict(_batch_case(nrs, full, args.prec, 2),
                                recipe="the batch recipe at full size, problems 0-7")}


def batch_full(args):
    """The whole batch workload at full size (128 ventral-node problems, n 5322-15771,
    about 173 GB of FP64 + FP32 matrices on the device): seconds per batch step through
    one graph with a fixed plan (K = 8 chains, G = 38: the autotuner's choice on the
    first 8 problems; tuning all 128 would take minutes), and one step of the same
    problems one after the other.  Not part of the default run."""
    import torch
    from paper_2001_06468_gb300 import nrs
    torch.cuda.set_device(0)
    t0 = time.time()
    probs = g.node_batch(128)
    gen_s = time.time() - t0
    res = _batch_case(nrs, probs, args.prec, 2, tune=False, plan=(8, 38), seq_steps=1)
    res.update({"workload": "ventral-node batch, all 128 problems at full size",
                "generator_s": gen_s,
                "matrix_bytes": int(sum(12 * pr.n * pr.n for pr in probs))})
    print(json.dumps(res), flush=True)


def cpu_baseline(pr, sols):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same
    workload (three RK2 steps from the initial state); also the largest
    relative error, over those steps' stage solutions, of the GPU paths
    (forces f and rigid velocities V separately)."""
    times, stages, cores = _oracle_step_timing(pr, 3, 1e9)
    n, n3 = pr.n, 3 * pr.N

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    errs = {}
    for name, gpu in sols.items():
        ef, eV = 0.0, 0.0
        for s, st in enumerate(stages[:len(gpu)]):
            for half, ref in ((0, st["sol1"]), (1, st["sol2"])):
                g_ = gpu[s][half * n:(half + 1) * n]
                ef = max(ef, rel(g_[:n3], ref[:n3]))
                eV = max(eV, rel(g_[n3:], ref[n3:]))
        errs[name] = {"f": ef, "V": eV}
    return {"value": float(np.mean(times)), "unit": "s/step", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} RK2 steps of the same workload from the initial state",
            "gpu_max_rel_err_vs_oracle": errs}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    pr = g.swimmer_config()
    W = min(args.warmup, 1)
    K = min(args.steps, 10)
    import oracle as O
    O.build()
    times, _, cores = _oracle_step_timing(pr, W + K, 1e9)
    t = times[W:]
    v = float(np.mean(t))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/step", "n_gpus": ws,
            "steps": len(t), "warmup": W, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "solver": "FP64 partial-pivoting LU + double-double refinement"},
            "cpu_baseline": {"value": v, "unit": "s/step", "cores": cores, "kind": "oracle",
                             "sample": f"{len(t)} RK2 steps after {W} warm-up (steps capped at 10)"},
            "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PROFILE_WORKLOADS = {
    "swimmer": lambda: g.swimmer_config(),
    # n = 6006: FP64 matrix 289 MB, FP32 copy 144 MB, both larger than L2
    "swimmer_mid": lambda: g.swimmer_config(ns_f=200, nth_f=10, ns_q=1000, nth_q=20),
    "swimmers4": lambda: g.swimmers_config(),
    "sperm_channel": lambda: g.sperm_channel_config(),
}


def profile_solve(args):
    """One solve of one stage (no timing loop): the command ncu captures."""
    import torch
    from paper_2001_06468_gb300 import nrs
    torch.cuda.set_device(0)
    pr = PROFILE_WORKLOADS[args.workload]()
    sh = g.pack_shapes(pr, 0.25)
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = nrs.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)
    ctx.factor(args.prec)
    _, rep = ctx.solve(b, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "n": pr.n, "prec": args.prec, "report": rep[0]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nrs", choices=["nrs", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp32", "tf32", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch workload section")
    ap.add_argument("--batch-full", action="store_true",
                    help="only the full-size batch of 128 problems (one JSON line)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="one kinematics + nearest + assemble + factor + solve on --workload, "
                         "then exit (for ncu captures)")
    ap.add_argument("--workload", default="swimmer", choices=sorted(PROFILE_WORKLOADS))
    args = ap.parse_args()
    if args.profile_solve:
        profile_solve(args)
        return
    if args.batch_full:
        batch_full(args)
        return
    if args.warmup < 3 and args.impl == "nrs":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nrs(args)


if __name__ == "__main__":
    main()
