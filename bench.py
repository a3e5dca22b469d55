#!/usr/bin/env python
"""Seconds per time step of the NEAREST regularized-stokeslet swimming
problem on GB300.

Headline workload: eight sperm-like cells in a closed channel (the analogue of
the paper's "multiple swimming sperm between parallel plates" runs): a static
box 4 x 1 x 0.5 meshed with 6000 force / 60000 quadrature points and eight
free cells of 400 / 4000 points, N = 9200, Q = 92000, eps = 0.005,
n = 27648 unknowns.  One step = one explicit-midpoint (RK2) step: twice
(kinematics, nearest neighbours, segments, FP64 assembly of A_s bit-identical
to the oracle's, rigid-body border, FP32 explicit inverse by blocked
Gauss-Jordan, two levels, whose rank-256 updates run on the tensor cores
from power-of-two-scaled FP16 pairs -- refreshed when the
previous solve needed more than 40 GMRES iterations or after 32 stages --,
GMRES-based iterative refinement with an extended-precision residual (every
product's rounded value summed exactly as a fixed-point integer, the rounding
errors in FP64) to the FP64
answer, started from the previous stage's solution) plus the state update.
Inputs are the seeded synthetic shapes of `synth` (the paper's cited beat
patterns are not available), resident in HBM before the timed region.

Beside the headline: the same workload with a fresh factor at every stage
(recorded as a CUDA graph), end to end through the C ABI from host buffers,
the four-swimmer box (n = 24024) and the single swimmer (n = 2406), the plain
FP64 path (cuSOLVER getrf/getrs on the same FP64 matrix), the batch of
ventral-node problems, the FP64 CPU oracle on a bounded sample, the GPU
solution's relative error against the oracle's on the first step, and the
roofline records of the kernels.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nrs|reference]
                    [--prec tf32|fp32] [--no-side] [--no-batch] [--no-cpu-baseline]
    python bench.py --profile-solve --workload swimmer_mid   # one solve, for ncu
    python bench.py --profile-step --workload sperm_channel  # one step, for ncu
    python bench.py --batch-full                             # all 128 full-size batch problems

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload.  Under torchrun each rank runs its
own replica of the headline problem ("replicas only": one dense solve does not
shard across GPUs) and its share of the batch (independent problems, no
collective in the data path).
"""

from __future__ import annotations

import argparse
import hashlib
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

METRIC = "s per timestep (assemble+solve) mixed-IR vs FP64 at 1e-10 rel err; pairs/s"
HEADLINE = "sperm_channel"
WORKLOADS_DESC = {
    "sperm_channel": "8 sperm-like cells in a closed channel 4x1x0.5, N=9200 force / Q=92000 "
                     "quadrature points, eps=0.005, n=27648",
    "swimmers4": "4 interacting undulating swimmers in a 4x4x1 box, N=8000 / Q=80000, eps=0.005, "
                 "n=24024",
    "swimmer": "single free undulating swimmer, N=800 / Q=8000, eps=0.005, n=2406",
}
# the product path's solver settings per workload
# (swept on the channel: refresh after 40 GMRES iterations or 32 stages, each
# GMRES call reducing the preconditioned residual 1e5-fold; the GMRES products
# with the float-pair copy of A)
HEADLINE_SOLVER = dict(reuse_factor=True, warm_start=True, reuse_max_inner=40,
                       reuse_max_stages=32, inner_tol=1e-5, arnoldi="df")
# the four-swimmer system has kappa_1 ~ 1e13: its GMRES steps need the longest
# restart and a tighter inner tolerance; a refinement that has not converged
# after 20 steps is retried with a new factor (nrs_step).  Swept: refresh after
# 60 GMRES iterations, the FP32 copy evaluated in FP32
C2_SOLVER = dict(inner_tol=1e-6, max_inner=64, max_outer=20, reuse_factor=True,
                 warm_start=True, reuse_max_inner=60, reuse_max_stages=32, arnoldi="df")
L2_FLUSH_BYTES = 512 << 20
FP64_NOMINAL_TFLOPS = 1.25       # GB300 FP64, nominal (2 FMA lanes per SM per clock)
TF32_OVER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor throughput
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128
PAIR_INSTR = 20                  # FP32-pipe instructions per (force, quadrature) pair
ASM64_OPS_PER_PAIR = 40          # FP64 operations per pair of the bit-exact assembly
RES_OPS_PER_ENTRY = 3           # FP64 operations per matrix entry of the extended residual
TOL = 1e-10


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




# DRAM bytes per launch from one ncu capture (profiles/), valid while the
# kernel's source file is unchanged (first 12 hex digits of its SHA-1).
NCU_TRAFFIC = {
    "k_tc_gj_update": {"bytes": 150743296 + 77540181, "n": 6006,
                       "file": "paper_2001_06468_gb300/csrc/tc_gemm.cu", "sha1": "e38e9748bdee",
                       "scale": "n^2 (captured at n = 6006, matrix larger than L2)"},
    # the bulk launch of block 5 at n = 13824: 817.7 + 674.5 MB against 8 x 13824 x
    # 13312 = 1.472 GB of M read and written
    "k_tc_gj2_update": {"bytes": None, "ratio": (817686528 + 674459392) / (8.0 * 13824 * 13312),
                        "file": "paper_2001_06468_gb300/csrc/gj2.cu", "sha1": "d617a4c644e5",
                        "scale": "traffic / algorithmic bytes at n = 13824, times the record's bytes"},
    "k_gj_diag": {"bytes": 136832, "file": "paper_2001_06468_gb300/csrc/gj.cu",
                  "sha1": "d098875a34c5",
                  "scale": "none (the 64 x 64 block, the previous D^{-1} and two 64 x 64 tiles)"},
    "k_assemble64": {"bytes": None, "file": "paper_2001_06468_gb300/csrc/assemble.cu",
                     "sha1": "", "scale": None},
    # one solve at n = 13824 (cold start, 2 refinement steps -- the first on a
    # working-precision residual, the second on the exact one -- and 4 GMRES
    # iterations; the three-CTAs-per-SM variant on 456 CTAs): 16.101 + 0.056 GB
    # against 7 passes over A (8 n^2) and M (4 n^2) = 16.05 GB
    "k_gmres_ir": {"bytes": None, "ratio": (16100587008 + 56127744) / (12.0 * 13824 ** 2 * 7),
                   "file": "paper_2001_06468_gb300/csrc/gmres_persistent.cu", "sha1": "0a46b9864734",
                   "scale": "traffic / algorithmic bytes at n = 13824, times the record's bytes"},
}


def _traffic(kernel, n, work=None):
    """DRAM bytes per launch from the ncu capture in NCU_TRAFFIC: scaled by n^2
    from the captured size, or as the captured ratio of traffic to algorithmic
    bytes times `work` (the record's algorithmic bytes per launch); None when
    there is no capture or the kernel's source changed since."""
    rec = NCU_TRAFFIC.get(kernel)
    if not rec or (rec["bytes"] is None and rec.get("ratio") is None):
        return None
    src = open(os.path.join(ROOT, rec["file"]), "rb").read()
    if hashlib.sha1(src).hexdigest()[:12] != rec["sha1"]:
        return None  # the kernel changed since the counters were taken
    if rec.get("ratio") is not None:
        return None if work is None else rec["ratio"] * work
    if "n" in rec:
        return rec["bytes"] * (n / rec["n"]) ** 2
    return rec["bytes"]


def derived_peaks(peaks, sm_mhz):
    """Whole-GPU peaks used by the roofline records.  HBM and BF16 are the
    measured figures; the others are derived from the unit counts and the
    sampled SM clock (FP32: 128 lanes x 2 flops; FP64: 2 FMA lanes per SM;
    TF32: the measured sustained BF16 rate x the nominal TF32/BF16 ratio;
    FP16: the measured sustained BF16 rate, the same nominal dense rate)."""
    clk = sm_mhz * 1e6
    return {"hbm_gbs": peaks["hbm_gbs"],
            "fp32_tflops": SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * clk / 1e12,
            "fp64_gops": FP64_NOMINAL_TFLOPS / 2 * 1e3 * sm_mhz / 2070.0,
            "tf32_tflops": peaks["bf16_tflops_sustained"] * TF32_OVER_BF16,
            "f16_tflops": peaks["bf16_tflops_sustained"],
            "pair_peak": SM_COUNT_NOMINAL * FP32_LANES_PER_SM * clk / PAIR_INSTR}


# phases that form one chain of work (the factorisation's blocks: updates on
# one stream, panels on another, back to back)
FAMILY = {"lu_update": "lu", "lu_panel": "lu", "lu_diag": "lu"}


def critical_ms(trace, merge_ms=0.2):
    """Milliseconds each phase family spends on the critical path of a trace
    [(phase, begin, end)].  A family's spans closer than merge_ms are one run
    (the factorisation is a chain of short spans on two streams); every
    instant covered by some run is charged to the running run that ends last
    (the one the work beside it waits for), instants no run covers to
    nothing.  Families: FAMILY, else the phase itself."""
    by_fam = {}
    for p, b, e in trace:
        by_fam.setdefault(FAMILY.get(p, p), []).append((b, e))
    runs = []
    for f, iv in by_fam.items():
        iv.sort()
        cb, ce = iv[0]
        for b, e in iv[1:]:
            if b <= ce + merge_ms:
                ce = max(ce, e)
            else:
                runs.append((f, cb, ce))
                cb, ce = b, e
        runs.append((f, cb, ce))
    runs.sort(key=lambda r: r[1])
    pts = sorted({t for _, b, e in runs for t in (b, e)})
    out = {}
    for a, b in zip(pts, pts[1:]):
        best = None
        for f, r0, r1 in runs:
            if r0 > a:
                break
            if r1 > a and (best is None or r1 > best[1]):
                best = (f, r1)
        if best is not None:
            out[best[0]] = out.get(best[0], 0.0) + (b - a)
    return out


def spans_alone(trace, phase, others):
    """Durations (ms) of the spans of `phase` in a trace [(phase, begin, end)]
    that overlap no span of the phases `others`."""
    busy = [(a, b) for p, a, b in trace if p in others]
    out = []
    for p, a, b in trace:
        if p == phase and not any(x < b and a < y for x, y in busy):
            out.append(b - a)
    return out


def kept_pairs(nrs, pr):
    """Pairs the FP64 assembly keeps from the previous assembly of the same
    context: tiles (128 collocation points x 16 segments) made only of static
    rigid bodies' force points, with per-body nearest neighbours (the rule of
    the library).  Their entries never change, so the assembly skips them
    once the matrix holds them."""
    import torch
    if pr.nn_global:
        return 0
    keep = np.zeros(pr.N, dtype=bool)
    off = 0
    for b in pr.bodies:
        if b.kind == g.STATIC and b.rigid:
            keep[off:off + b.N] = True
        off += b.N

    def blocks(bs):
        return np.array([keep[k * bs:(k + 1) * bs].all() for k in range(-(-pr.N // bs))])
    mb, nb = blocks(128), blocks(16)
    if not mb.any() or not nb.any():
        return 0
    ctx = nrs.Context.from_problem(pr)
    xi, Xiw, _ = nrs.shapes_to_device(g.pack_shapes(pr, 0.0))
    nn, _, _ = ctx.nearest_build(xi, Xiw)
    nn = nn.cpu().numpy()
    ctx.close()
    m_kept = int(sum(min(pr.N, (k + 1) * 128) - k * 128 for k in np.nonzero(mb)[0]))
    q_kept = int(np.count_nonzero(nb[nn // 16]))
    return m_kept * q_kept


def rooflines(ph_ms, ph_spans, n, pairs, peaks, peak_src, sm_mhz, solve_stats, pairs64=None,
              update_f16=True, arnoldi_df=False):
    """Roofline records of the kernel families from the live per-phase CUDA
    event times (one span per launch, on the stream each kernel runs on).
    Algorithmic work per launch:
      lu_update   k_tc_gj_update: 8 n^2 bytes (read + write of the FP32 matrix);
                  3 x 2 n^2 64 tensor flops (split TF32)
      lu_diag     k_gj_diag: (2 + 8 (nblk - 1)) / nblk x 64^3 FP32 flops, one CTA
      assemble    k_assemble64: 40 FP64 operations per (force, quadrature) pair
      assemble32  k_assemble32: N Q pairs against the FP32 pair peak (20 instructions a pair)
      krylov      k_gmres_ir: (exact + working + inner) 8 n^2 (the residuals'
                  products, exact from A in FP64 or in working precision from its
                  float-pair copy, and the GMRES products: 8 bytes an entry each)
                  + (outer + inner + 1) 4 n^2 bytes of M; + 8 n^2 (||A||_inf, once
                  per launch); exact x 3 n^2 (extended residual: product, its error,
                  the error sum; the products' sum on the integer pipe) + n^2
                  (||A||_inf) + (inner + working) x n^2 (the GMRES and residual
                  products, when in FP64) FP64 operations.  Without the residual
                  counts, every refinement step counts one exact residual."""
    P = derived_peaks(peaks, sm_mhz)

    def per_launch(ph):
        return ph_ms[ph] / 1e3 / max(ph_spans[ph], 1)

    recs = {}
    two_level = (ph_spans.get("lu_update") and not ph_spans.get("lu_diag")
                 and ph_spans.get("lu_panel") == ph_spans.get("lu_update"))
    if two_level:
        # k_tc_gj2_update: one rank-256 product per 256-column block, from
        # scaled FP16 pairs (kind::f16, rated against the BF16/FP16 tensor
        # peak) or split TF32; it also reads and writes the FP32 matrix once
        # (8 n^2 bytes).  The record's bound is the roofline it is closer to.
        t = per_launch("lu_update")
        b = 8.0 * n * n
        fl = 3 * 2.0 * n * n * 256
        tp = P["f16_tflops"] if update_f16 else P["tf32_tflops"]
        pieces = "scaled FP16 pairs" if update_f16 else "split TF32"
        tfrac, hfrac = fl / t / 1e12 / tp, b / t / 1e9 / P["hbm_gbs"]
        tensor_rec = {"bound": "tensor", "achieved": fl / t / 1e12, "peak": tp, "unit": "TFLOP/s",
                      "frac": tfrac,
                      "peak_source": peak_src + (" BF16 sustained (FP16 runs at the BF16 rate)"
                                                 if update_f16 else
                                                 " BF16 sustained x nominal TF32/BF16 (1.1/2.25)"),
                      "work_per_launch": fl,
                      "work_unit": f"tensor flops (3 passes of {pieces} x 2 n^2 256)"}
        hbm_rec = {"bound": "hbm", "achieved": b / t / 1e9, "peak": P["hbm_gbs"], "unit": "GB/s",
                   "frac": hfrac, "peak_source": peak_src + " HBM copy", "work_per_launch": b,
                   "work_unit": "bytes (8 n^2: read and write of the FP32 matrix)"}
        recs["lu_update"] = {
            "kernel": "k_tc_gj2_update (persistent tcgen05 rank-256 update of the FP32 inverse "
                      f"from {pieces}, two-level Gauss-Jordan)",
            **(hbm_rec if hfrac >= tfrac else tensor_rec),
            "tensor_tflops": fl / t / 1e12, "tensor_frac": tfrac, "tensor_peak": tp,
            "useful_tflops": fl / 3 / t / 1e12,
            "hbm_gbs": b / t / 1e9, "hbm_frac": hfrac,
            "us_per_launch": t * 1e6, "launches": ph_spans["lu_update"],
            "traffic": _traffic("k_tc_gj2_update", n, b)}
        t = per_launch("lu_panel")
        recs["lu_panel"] = {
            "kernel": "column-panel elimination (4 x k_gj_diag, k_gj2_rpanel, k_gj2_panel_update) "
                      "and k_gj2_prep",
            "bound": "alu", "achieved": 2.0 * n * 256 * 256 / t / 1e12, "peak": P["fp32_tflops"],
            "unit": "TFLOP/s", "frac": 2.0 * n * 256 * 256 / t / 1e12 / P["fp32_tflops"],
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x sampled clock",
            "overlap": "runs on a second stream beside the previous block's bulk update (all "
                       "SMs but 24); its span includes waiting for SMs and is on the critical "
                       "path only where it outlasts that update",
            "work_per_launch": 2.0 * n * 256 * 256, "us_per_launch": t * 1e6,
            "launches": ph_spans["lu_panel"], "traffic": None}
    elif ph_spans.get("lu_update"):
        t = per_launch("lu_update")
        b = 8.0 * n * n
        fl = 3 * 2.0 * n * n * 64
        recs["lu_update"] = {
            "kernel": "k_tc_gj_update (tcgen05 split-TF32 rank-64 update of the FP32 inverse)",
            "bound": "hbm", "achieved": b / t / 1e9, "peak": P["hbm_gbs"], "unit": "GB/s",
            "frac": b / t / 1e9 / P["hbm_gbs"], "peak_source": peak_src + " HBM copy",
            "work_per_launch": b, "work_unit": "bytes (8 n^2)",
            "tensor_tflops": fl / t / 1e12, "tensor_frac_of_tf32": fl / t / 1e12 / P["tf32_tflops"],
            "tf32_peak_tflops": P["tf32_tflops"],
            "us_per_launch": t * 1e6, "launches": ph_spans["lu_update"],
            "traffic": _traffic("k_tc_gj_update", n)}
    if ph_spans.get("lu_diag"):
        t = per_launch("lu_diag")
        nblk = -(-n // 64)
        w = (2.0 + 8.0 * (nblk - 1)) / nblk * 64 ** 3
        recs["lu_diag"] = {
            "kernel": "k_gj_diag (64 x 64 diagonal-block inverse with lookahead, one CTA)",
            "bound": "alu", "achieved": w / t / 1e12, "peak": P["fp32_tflops"], "unit": "TFLOP/s",
            "frac": w / t / 1e12 / P["fp32_tflops"],
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x sampled clock (whole GPU)",
            "latency_bound": "64 dependent pivot steps on one CTA", "work_per_launch": w,
            "us_per_launch": t * 1e6, "launches": ph_spans["lu_diag"],
            "traffic": _traffic("k_gj_diag", n)}
    if ph_spans.get("assemble"):
        t = per_launch("assemble")
        p64 = pairs if pairs64 is None else pairs64  # the pairs evaluated (kept blocks skipped)
        ops = p64 * ASM64_OPS_PER_PAIR
        recs["assemble"] = {
            "kernel": "k_assemble64 (NEAREST A_s in FP64, bit-identical to the oracle)",
            "bound": "alu", "achieved": ops / t / 1e9, "peak": P["fp64_gops"], "unit": "Gop/s",
            "frac": ops / t / 1e9 / P["fp64_gops"],
            "peak_source": "derived: nominal FP64 1.25 TFLOP/s = 625 G FP64 ops/s at 2070 MHz, "
                           "scaled to the sampled clock",
            "work_per_launch": ops, "work_unit": "FP64 operations (40 per pair; square root and "
                                                 "division counted once each)",
            "pairs_per_s": p64 / t, "pairs_evaluated_per_launch": p64,
            "pairs_kept_per_launch": pairs - p64, "ms_per_launch": t * 1e3,
            "launches": ph_spans["assemble"], "traffic": _traffic("k_assemble64", n)}
    if ph_spans.get("assemble32"):
        t = per_launch("assemble32")
        recs["assemble32"] = {
            "kernel": "k_assemble32 (+ 2 k_split_points): FP32 copy of A_s for the factorisation",
            "bound": "alu", "achieved": pairs / t, "peak": P["pair_peak"], "unit": "pairs/s",
            "frac": pairs / t / P["pair_peak"],
            "peak_source": "derived: 152 SMs x 128 lanes x sampled clock / 20 FP32 instructions "
                           "per pair",
            "hbm_write_bound_pairs_per_s": pairs / (4.0 * n * n / (peaks["hbm_gbs"] * 1e9)),
            "work_per_launch": pairs, "ms_per_launch": t * 1e3, "launches": ph_spans["assemble32"],
            "traffic": None}
    if ph_spans.get("krylov") and solve_stats:
        o, i = solve_stats["outer_mean"], solve_stats["inner_mean"]
        ex = solve_stats.get("exact_mean", o)
        wk = solve_stats.get("working_mean", 0.0)
        t = per_launch("krylov")
        b = 8.0 * n * n * (ex + wk + i + 1) + 4.0 * n * n * (o + i + 1)
        # FP64 operations: the exact residuals, the ||A||_inf pass, and the
        # GMRES and working-precision residual products unless they run on the
        # float-pair copy (FP32 pipe)
        ops = RES_OPS_PER_ENTRY * n * n * ex + n * n * (1 + (0 if arnoldi_df else i + wk))
        recs["krylov"] = {
            "kernel": "k_gmres_ir (persistent GMRES-IR, one cooperative launch per solve)",
            "bound": "hbm", "achieved": b / t / 1e9, "peak": P["hbm_gbs"], "unit": "GB/s",
            "frac": b / t / 1e9 / P["hbm_gbs"], "peak_source": peak_src + " HBM copy",
            "work_per_launch": b, "work_unit": "bytes of A (FP64) and M (FP32) streamed",
            "fp64_gops": ops / t / 1e9, "fp64_frac": ops / t / 1e9 / P["fp64_gops"],
            "outer_mean": o, "inner_mean": i, "ms_per_launch": t * 1e3,
            "launches": ph_spans["krylov"], "traffic": _traffic("k_gmres_ir", n, b)}
    return recs


def _shapes_host(pr, t):
    import torch
    d = g.pack_shapes(pr, t)
    return tuple(torch.from_numpy(d[k]).pin_memory() for k in ("x", "Xw", "xidot"))


def _input_digest(pr, dt):
    m = hashlib.sha1()
    for t in (0.0, 0.5 * dt):
        d = g.pack_shapes(pr, t)
        for k in ("x", "Xw", "xidot"):
            m.update(np.ascontiguousarray(d[k], dtype=np.float64).tobytes())
    Y = g.initial_state(pr)
    m.update(np.ascontiguousarray(Y["x0"], dtype=np.float64).tobytes())
    m.update(np.ascontiguousarray(Y["B"], dtype=np.float64).tobytes())
    return m.hexdigest()


def _golden(name, pr):
    """The oracle's first step of a full-size workload, stored under
    tests/golden by a script that calls only the oracle (None when absent or
    written from other inputs)."""
    path = os.path.join(ROOT, "tests", "golden", f"{name}_step0.npz")
    if not os.path.exists(path):
        return None
    z = np.load(path)
    if str(z["digest"]) != _input_digest(pr, pr.dt):
        return None
    return {k: z[k] for k in ("sol1", "sol2", "x0", "B")}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _first_step_errors(nrs, pr, ref, **kw):
    """Relative errors of f and V of both stages of the first step (from the
    initial state) against the oracle's."""
    import torch
    ctx = nrs.Context.from_problem(pr, factor_prec="tf32", **kw)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    d0 = nrs.shapes_to_device(g.pack_shapes(pr, 0.0))
    dh = nrs.shapes_to_device(g.pack_shapes(pr, 0.5 * pr.dt))
    sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
    rep = ctx.step(nrs.Context.shapes(*d0), nrs.Context.shapes(*dh), pr.dt, sol=sol)
    s = sol.cpu().numpy()
    Yg = ctx.get_state()
    ctx.close()
    n, n3 = pr.n, 3 * pr.N
    out = {}
    for k, key in enumerate(("sol1", "sol2")):
        got = s[k * n:(k + 1) * n]
        out[f"stage{k + 1}"] = {"f": _rel(got[:n3], ref[key][:n3]), "V": _rel(got[n3:], ref[key][n3:])}
    out["state"] = {"x0": _rel(Yg["x0"], ref["x0"]), "B": _rel(Yg["B"], ref["B"])}
    out["backward_err"] = [st["backward_err"] for st in rep["stages"]]
    out["within_tol"] = all(v <= TOL for st in ("stage1", "stage2") for v in out[st].values())
    return out


class _Timer:
    """CUDA-event timing of K calls on a stream, L2 flushed before each."""

    def __init__(self, flush):
        self.flush = flush

    def run(self, stream, fn, count, first=0):
        import torch
        ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for s in range(count):
            self.flush.fill_(float(s))  # evict L2 between timed steps (untimed)
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                e0.record(stream)
                fn(first + s)
                e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms


def headline(nrs, args, ws, local, timer, peaks, peak_src):
    """The product path on the channel workload: timed steps, end to end,
    instrumented pass, fresh-factor graph path, first-step parity."""
    import torch
    pr = g.workload(HEADLINE)
    dt = pr.dt
    K, W = args.steps, args.warmup
    total = K + W
    host = [(_shapes_host(pr, s * dt), _shapes_host(pr, (s + 0.5) * dt)) for s in range(total)]
    dev = [tuple(tuple(t.cuda() for t in st) for st in pair) for pair in host]
    Y0 = g.initial_state(pr)
    kw = dict(HEADLINE_SOLVER)

    def new_ctx(**extra):
        c = nrs.Context.from_problem(pr, factor_prec=args.prec, **dict(kw, **extra))
        c.set_state(Y0["x0"], Y0["B"])
        return c

    def stepper(c, bufs=None):
        def f(s):
            pair = dev[s] if bufs is None else bufs
            c.step(nrs.Context.shapes(*pair[0]), nrs.Context.shapes(*pair[1]), dt, report=False)
        return f

    # -- timed region: K steps of the product path, no instrumentation
    ctx = new_ctx()
    for s in range(W):
        stepper(ctx)(s)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    c0, r0 = ctx.counters(), ctx.residual_counters()
    ctx.get_timing()  # clears the kernel count
    with ClockSampler(_visible_gpu_index(local)) as clk:
        step_ms = timer.run(ctx.stream, stepper(ctx), K, first=W)
    clocks = clk.summary()
    _, launches = ctx.get_timing()
    c1, r1 = ctx.counters(), ctx.residual_counters()
    st = ctx.sync()  # device status word after the timed region
    ctx.close()
    counts = {k: c1[k] - c0[k] for k in c1}
    counts.update({"residuals_" + k: r1[k] - r0[k] for k in r1})
    t_local = sum(step_ms) / 1e3
    t_max = _max_over_ranks(t_local, ws)

    # -- end to end through the C ABI from pinned host buffers: H2D of both
    # stages' shapes and D2H of both solutions and the new state, every step
    ctx = new_ctx()
    bufs = tuple(tuple(torch.empty_like(t, device="cuda") for t in st) for st in host[0])
    sol = torch.empty(2 * pr.n, dtype=torch.float64, device="cuda")
    sol_h = torch.empty(2 * pr.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for st in host[0] for t in st)
    d2h = sol_h.numel() * 8 + pr.n_free * 12 * 8
    Ke = K  # the same steps as the timed region (refreshed and reused factors alternate)

    def e2e_step(s):
        for st_h, st_d in zip(host[s], bufs):
            for th, td in zip(st_h, st_d):
                td.copy_(th, non_blocking=True)
        ctx.step(nrs.Context.shapes(*bufs[0]), nrs.Context.shapes(*bufs[1]), dt, sol=sol,
                 report=False)
        sol_h.copy_(sol, non_blocking=True)
        ctx.get_state()

    for s in range(W):
        e2e_step(s)
    e_ms = timer.run(ctx.stream, e2e_step, Ke, first=W)
    ctx.close()
    e2e_s = _max_over_ranks(sum(e_ms) / 1e3, ws) / Ke / ws

    # -- instrumented pass: CUDA events around every phase, on the stream each
    # phase runs on (per-launch durations for the roofline records)
    Ki = min(K, 5)
    ctx = new_ctx()
    for s in range(W):
        stepper(ctx)(s)
    torch.cuda.synchronize()
    ci0, ri0 = ctx.counters(), ctx.residual_counters()
    ctx.set_timing(True)
    instr_ms = timer.run(ctx.stream, stepper(ctx), Ki, first=W)
    trace = ctx.get_trace()
    phases, _ = ctx.get_timing()
    ctx.set_timing(False)
    ci1, ri1 = ctx.counters(), ctx.residual_counters()
    ctx.close()
    ph_ms = {k: v[0] for k, v in phases.items()}
    ph_spans = {k: v[1] for k, v in phases.items()}
    solves = max(ci1["solves"] - ci0["solves"], 1)
    solve_stats = {"outer_mean": (ci1["outer"] - ci0["outer"]) / solves,
                   "inner_mean": (ci1["inner"] - ci0["inner"]) / solves}
    if ri1["exact"] + ri1["working"] > ri0["exact"] + ri0["working"]:
        solve_stats["exact_mean"] = (ri1["exact"] - ri0["exact"]) / solves
        solve_stats["working_mean"] = (ri1["working"] - ri0["working"]) / solves

    # -- the same workload with a fresh factor at every stage, recorded as a
    # CUDA graph, and its instrumented phases (the factorisation's kernels)
    Kf = min(K, 4)
    ctxf = nrs.Context.from_problem(pr, factor_prec=args.prec, graph=True)
    ctxf.set_state(Y0["x0"], Y0["B"])
    gbuf = tuple(tuple(torch.empty_like(t) for t in st) for st in dev[0])

    def graph_step(s):
        for st_src, st_dst in zip(dev[s], gbuf):
            for src, dst in zip(st_src, st_dst):
                dst.copy_(src, non_blocking=True)
        ctxf.step(nrs.Context.shapes(*gbuf[0]), nrs.Context.shapes(*gbuf[1]), dt, report=False)

    for s in range(2):  # the first call builds the maps of the rigid bodies, the second records
        graph_step(s)
    f_ms = timer.run(ctxf.stream, graph_step, Kf, first=2)
    ctxf.sync()
    ctxf.close()
    ctxf = nrs.Context.from_problem(pr, factor_prec=args.prec)
    ctxf.set_state(Y0["x0"], Y0["B"])
    stepper(ctxf)(0)
    cf0 = ctxf.counters()
    ctxf.set_timing(True)
    timer.run(ctxf.stream, stepper(ctxf), 1, first=1)
    fph, _ = ctxf.get_timing()
    ctxf.set_timing(False)
    cf1 = ctxf.counters()
    ctxf.close()
    fph_ms = {k: v[0] for k, v in fph.items()}
    fph_spans = {k: v[1] for k, v in fph.items()}
    fsolves = max(cf1["solves"] - cf0["solves"], 1)
    fsolve_stats = {"outer_mean": (cf1["outer"] - cf0["outer"]) / fsolves,
                    "inner_mean": (cf1["inner"] - cf0["inner"]) / fsolves}

    # -- parity: the first step from the initial state against the oracle's
    ref = _golden(HEADLINE, pr)
    parity = None
    if ref is not None:
        parity = {"product_path": _first_step_errors(nrs, pr, ref, **kw),
                  "fresh_factor": _first_step_errors(nrs, pr, ref),
                  "tolerance": TOL,
                  "oracle": "tests/golden/sperm_channel_step0.npz (oracle/ alone; input digest checked)"}

    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # every instrumented assembly follows at least one full one: the static
    # blocks are kept in all of them
    p64 = pr.pairs - kept_pairs(nrs, pr)
    recs = rooflines(ph_ms, ph_spans, pr.n, pr.pairs, peaks, peak_src, sm_mhz, solve_stats, p64,
                     arnoldi_df=kw.get("arnoldi") == "df")
    # the FP64 assembly runs beside the factorisation in factored stages: its
    # launches that overlapped no factorisation span, rated on their own
    alone = spans_alone(trace, "assemble", ("lu_panel", "lu_update", "assemble32"))
    if alone and "assemble" in recs:
        r = recs["assemble"]
        t = float(np.mean(alone)) / 1e3
        r["alone"] = {"launches": len(alone), "ms_per_launch": t * 1e3,
                      "achieved": r["work_per_launch"] / t / 1e9,
                      "frac": r["work_per_launch"] / t / 1e9 / r["peak"],
                      "note": "launches that overlapped no factorisation span"}
    frecs = rooflines(fph_ms, fph_spans, pr.n, pr.pairs, peaks, peak_src, sm_mhz, fsolve_stats, p64)
    tot = sum(ph_ms.values())
    crit = critical_ms(trace)
    crit_tot = sum(instr_ms)
    return {
        "pr": pr, "K": K, "W": W, "t_max": t_max, "step_ms": step_ms, "clocks": clocks,
        "launches": launches, "counts": counts, "status_after": st, "e2e_s": e2e_s,
        "h2d": h2d, "d2h": d2h, "e2e_steps": Ke,
        "fresh_graph_s": float(np.mean(f_ms)) / 1e3, "fresh_steps": Kf,
        "instr_s": float(np.mean(instr_ms)) / 1e3,
        "phases_ms_per_step": {k: v / Ki for k, v in ph_ms.items() if ph_spans[k]},
        "phase_share": {k: v / tot for k, v in ph_ms.items() if ph_spans[k]},
        "critical_share": {k: v / crit_tot for k, v in crit.items()},
        "fresh_phases_ms_per_step": {k: v for k, v in fph_ms.items() if fph_spans[k]},
        "solve_stats": solve_stats, "fresh_solve_stats": fsolve_stats,
        "recs": recs, "fresh_recs": frecs, "parity": parity}


def side_workload(nrs, args, name, steps, warm, solver, timer, graph=False):
    """Seconds per step of another workload (same timing rules), and the
    first step's errors against the oracle where its answer is stored."""
    import torch
    pr = g.workload(name)
    dt = pr.dt
    dev = [(nrs.shapes_to_device(g.pack_shapes(pr, s * dt)),
            nrs.shapes_to_device(g.pack_shapes(pr, (s + 0.5) * dt))) for s in range(steps + warm)]
    Y0 = g.initial_state(pr)
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, graph=graph, **solver)
    ctx.set_state(Y0["x0"], Y0["B"])
    gbuf = tuple(tuple(torch.empty_like(t) for t in st) for st in dev[0])

    def step(s):
        src = dev[s]
        if graph:
            for st_src, st_dst in zip(src, gbuf):
                for a, b in zip(st_src, st_dst):
                    b.copy_(a, non_blocking=True)
            src = gbuf
        ctx.step(nrs.Context.shapes(*src[0]), nrs.Context.shapes(*src[1]), dt, report=False)

    for s in range(warm):
        step(s)
    c0 = ctx.counters()
    ms = timer.run(ctx.stream, step, steps, first=warm)
    c1 = ctx.counters()
    ctx.sync()
    ctx.close()
    out = {"workload": WORKLOADS_DESC.get(name, name), "s_per_step": float(np.mean(ms)) / 1e3,
           "steps": steps, "warmup": warm, "graph": graph,
           "solver": {k: v for k, v in solver.items()}}
    sol_n = c1["solves"] - c0["solves"]
    if sol_n:
        out["outer_mean"] = (c1["outer"] - c0["outer"]) / sol_n
        out["inner_mean"] = (c1["inner"] - c0["inner"]) / sol_n
        out["factorizations_per_step"] = (c1["factorizations"] - c0["factorizations"]) / steps
    ref = _golden(name, pr)
    if ref is not None:
        out["first_step_vs_oracle"] = _first_step_errors(nrs, pr, ref, **solver)
    return out


def tracers_line(nrs, args, timer, count=2000, steps=3, warm=1):
    """The channel workload with passive tracers (the paper's particle
    tracking): seconds per step of the product path carrying ``count``
    tracers seeded in the channel, and the velocity kernel on its own
    (pairs/s = tracers x quadrature points per evaluation)."""
    import torch
    pr = g.workload(HEADLINE)
    dt = pr.dt
    rng = np.random.default_rng(0)
    tr = np.zeros((count, 4))
    tr[:, :3] = rng.uniform([0.1, 0.1, 0.05], [3.9, 0.9, 0.45], size=(count, 3))
    dev = [(nrs.shapes_to_device(g.pack_shapes(pr, s * dt)),
            nrs.shapes_to_device(g.pack_shapes(pr, (s + 0.5) * dt))) for s in range(steps + warm)]
    Y0 = g.initial_state(pr)
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, **HEADLINE_SOLVER)
    ctx.set_state(Y0["x0"], Y0["B"])
    ctx.set_tracers(tr)

    def step(s):
        ctx.step(nrs.Context.shapes(*dev[s][0]), nrs.Context.shapes(*dev[s][1]), dt, report=False)

    for s in range(warm):
        step(s)
    ms = timer.run(ctx.stream, step, steps, first=warm)
    # the velocity kernel alone, on the last stage's geometry
    xp = torch.from_numpy(tr).cuda()
    f = torch.from_numpy(rng.normal(size=3 * pr.N)).cuda()
    ctx.velocity(xp, f)
    vms = timer.run(ctx.stream, lambda s: ctx.velocity(xp, f), 5)
    moved = float(np.abs(ctx.get_tracers()[:, :3] - tr[:, :3]).max())
    ctx.close()
    t = float(np.median(vms)) / 1e3
    pairs = count * pr.Q
    return {"workload": WORKLOADS_DESC[HEADLINE] + f", {count} tracers",
            "s_per_step": float(np.mean(ms)) / 1e3, "steps": steps,
            "velocity_ms": t * 1e3, "velocity_pairs_per_s": pairs / t,
            "velocity_fp64_gops": pairs * 52 / t / 1e9,
            "velocity_note": "52 FP64 operations per (tracer, quadrature point) pair; two "
                             "evaluations per step",
            "max_tracer_displacement": moved}


def dormand_prince_line(nrs, args, name="swimmer", T=0.1, tol=1e-8):
    """Adaptive Dormand-Prince 5(4) (the paper's ode45) on a workload over
    [0, T] with rtol = atol = tol: steps, stage evaluations and seconds per
    simulated time unit (wall clock of the whole integration, device
    synchronised at its ends), beside the explicit midpoint's cost per unit
    time at the bench's dt."""
    import torch
    pr = g.workload(name)
    Y0 = g.initial_state(pr)
    cache = {}

    def at(t):
        key = round(t, 15)
        if key not in cache:
            cache[key] = nrs.shapes_to_device(g.pack_shapes(pr, t))
        return nrs.Context.shapes(*cache[key])

    for warm in (True, False):
        ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, **HEADLINE_SOLVER)
        ctx.set_state(Y0["x0"], Y0["B"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = ctx.dp_integrate(at, 0.0, T if not warm else pr.dt, pr.dt, tol, tol)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ctx.close()
    stages = 7 + 6 * (info["accepted"] + info["rejected"] - 1)
    return {"workload": WORKLOADS_DESC.get(name, name), "interval": T, "rtol": tol, "atol": tol,
            "accepted": info["accepted"], "rejected": info["rejected"], "stage_evaluations": stages,
            "s_per_time_unit": wall / T, "s_per_accepted_step": wall / max(info["accepted"], 1),
            "mean_step": T / max(info["accepted"], 1),
            "rk2_stage_evaluations_per_time_unit_at_dt": 2.0 / pr.dt}


def factorisation_line(nrs, args, timer, peaks, sm_mhz):
    """One factorisation alone on the headline workload (the FP32 copy of the
    first stage's matrix inverted by the product path's schedule), timed with
    CUDA events after one untimed one, L2 flushed before each.  Work counted:
    Gauss-Jordan 2 n^3 flops (an LU would need 2/3 n^3); the tensor cores
    multiply 3 split products of rank 256 into every column for each of the
    n / 256 blocks (6 n^3 flops); the updates read and write the FP32 matrix
    once a block (8 n^2 bytes x n / 256)."""
    pr = g.workload(HEADLINE)
    n = pr.n
    Y0 = g.initial_state(pr)
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec)
    ctx.set_state(Y0["x0"], Y0["B"])
    xi, Xiw, xidot = nrs.shapes_to_device(g.pack_shapes(pr, 0.0))
    x, Xw, _ = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)
    if ctx.factor(args.prec) != 0:
        ctx.close()
        return {"error": "factorisation failed"}
    ms = timer.run(ctx.stream, lambda s: ctx.factor(args.prec), 4)
    ctx.close()
    t = float(np.mean(ms)) / 1e3
    P = derived_peaks(peaks, sm_mhz)
    blocks = -(-n // 256)
    return {"workload": WORKLOADS_DESC[HEADLINE], "n": n, "ms": t * 1e3, "runs": len(ms),
            "gauss_jordan_tflops": 2.0 * n ** 3 / t / 1e12,
            "lu_equivalent_tflops": 2.0 / 3.0 * n ** 3 / t / 1e12,
            "tensor_tflops": 6.0 * n ** 3 / t / 1e12,
            "tensor_frac": 6.0 * n ** 3 / t / 1e12 / P["f16_tflops"],
            "hbm_gbs": 8.0 * n * n * blocks / t / 1e9,
            "hbm_frac": 8.0 * n * n * blocks / t / 1e9 / P["hbm_gbs"],
            "note": "FP32 explicit inverse, two-level Gauss-Jordan (rank-256 tcgen05 updates from "
                    "scaled FP16 pairs); tensor and HBM fractions of the measured sustained "
                    "BF16/FP16 and copy peaks"}


def plain_fp64(nrs, args, timer):
    """The plain FP64 GPU path on the headline workload: the FP64 assembly
    (this library's kernel, the same matrix) and cuSOLVER's getrf + getrs
    through torch.linalg, each timed once on the first stage's system, and
    this library's own blocked FP64 LU on the single swimmer as a fraction of
    the FP64 peak."""
    import torch
    torch.backends.cuda.preferred_linalg_library("cusolver")
    pr = g.workload(HEADLINE)
    Y0 = g.initial_state(pr)
    ctx = nrs.Context.from_problem(pr, factor_prec="fp64")
    ctx.set_state(Y0["x0"], Y0["B"])
    xi, Xiw, xidot = nrs.shapes_to_device(g.pack_shapes(pr, 0.0))
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)  # warm-up of the kernel
    torch.cuda.synchronize()
    st = ctx.stream
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(st):
        e[0].record(st)
        ctx.assemble(x, Xw, want_matrix=False)
        e[1].record(st)
    torch.cuda.synchronize()
    t_asm = e[0].elapsed_time(e[1]) / 1e3
    At = ctx.assemble(x, Xw)
    ctx.close()
    A = At.T  # column-major view of the FP64 matrix
    bb = b[:pr.n].clone().reshape(-1, 1)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        e[0].record(st)
        LU, piv = torch.linalg.lu_factor(A)
        e[1].record(st)
        xs = torch.linalg.lu_solve(LU, piv, bb)
        e[2].record(st)
    torch.cuda.synchronize()
    t_getrf = e[0].elapsed_time(e[1]) / 1e3
    t_getrs = e[1].elapsed_time(e[2]) / 1e3
    xs = xs.reshape(-1).cpu().numpy()
    del LU, piv, A, At
    torch.cuda.empty_cache()
    ref = _golden(HEADLINE, pr)
    err = None
    if ref is not None:
        n3 = 3 * pr.N
        err = {"f": _rel(xs[:n3], ref["sol1"][:n3]), "V": _rel(xs[n3:], ref["sol1"][n3:])}
    stage = t_asm + t_getrf + t_getrs
    n = pr.n
    # this library's FP64 LU on the single swimmer
    sw = g.workload("swimmer")
    cs = nrs.Context.from_problem(sw, factor_prec="fp64")
    Ys = g.initial_state(sw)
    cs.set_state(Ys["x0"], Ys["B"])
    xi, Xiw, xidot = nrs.shapes_to_device(g.pack_shapes(sw, 0.0))
    x, Xw, b = cs.kinematics(xi, Xiw, xidot)
    cs.nearest_build(xi, Xiw)
    cs.assemble(x, Xw, want_matrix=False)
    cs.factor("fp64")
    torch.cuda.synchronize()
    with torch.cuda.stream(cs.stream):
        e[0].record(cs.stream)
        cs.factor("fp64")
        e[1].record(cs.stream)
    torch.cuda.synchronize()
    t_own = e[0].elapsed_time(e[1]) / 1e3
    cs.close()
    fp64_peak = FP64_NOMINAL_TFLOPS
    return {"s_per_step": 2 * stage,
            "how": "2 x one measured stage: FP64 assembly + cuSOLVER getrf + getrs (torch.linalg) "
                   "on the first stage's system",
            "assemble64_s": t_asm, "getrf_s": t_getrf, "getrs_s": t_getrs,
            "getrf_tflops": 2.0 / 3.0 * n ** 3 / t_getrf / 1e12,
            "getrf_frac_of_fp64_nominal": 2.0 / 3.0 * n ** 3 / t_getrf / 1e12 / fp64_peak,
            "error_vs_oracle_without_refinement": err,
            "own_fp64_lu": {"workload": WORKLOADS_DESC["swimmer"], "s": t_own,
                            "tflops": 2.0 / 3.0 * sw.n ** 3 / t_own / 1e12,
                            "frac_of_fp64_nominal": 2.0 / 3.0 * sw.n ** 3 / t_own / 1e12 / fp64_peak}}


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
    info = dict(info)
    ns = [pr.n for pr in probs]
    out = {"problems": nprob, "n_min": min(ns), "n_max": max(ns), "n_mean": float(np.mean(ns)),
           "pairs": int(sum(pr.pairs for pr in probs)),
           "s_per_batch_step": ms / 1e3 / steps,
           "problem_steps_per_s": nprob * steps / (ms / 1e3), "steps": steps,
           "chains": info["chains"], "solve_grid": info["grid"],
           "graph_kernels": info["graph_kernels"], "tuned_ms": tuned.get("ms")}
    if seq_steps == 0:
        return out
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
    out.update(sequential_eager_s_per_batch_step=ms_seq / 1e3 / seq_steps,
               speedup_vs_sequential=(ms_seq / seq_steps) / (ms / steps))
    return out


def batch_full(args):
    """The whole batch workload at full size (128 ventral-node problems, n 5322-15771,
    about 173 GB of FP64 + FP32 matrices on the device): seconds per batch step through
    one graph with the plan the autotuner chooses on the first 8 problems (tuning all
    128 would take minutes), and one step of the same problems one after the other.
    Not part of the default run."""
    import torch
    from paper_2001_06468_gb300 import nrs
    torch.cuda.set_device(0)
    t0 = time.time()
    probs = g.node_batch(128)
    gen_s = time.time() - t0
    first8 = _batch_case(nrs, probs[:8], args.prec, 1, seq_steps=0)
    plan = (first8["chains"], first8["solve_grid"])
    torch.cuda.empty_cache()
    res = _batch_case(nrs, probs, args.prec, 2, tune=False, plan=plan, seq_steps=1)
    res.update({"workload": "ventral-node batch, all 128 problems at full size",
                "generator_s": gen_s,
                "matrix_bytes": int(sum(12 * pr.n * pr.n for pr in probs))})
    print(json.dumps(res), flush=True)


PROFILE_WORKLOADS = {
    "swimmer": lambda: g.swimmer_config(),
    # n = 6006: FP64 matrix 289 MB, FP32 copy 144 MB, both larger than L2
    "swimmer_mid": lambda: g.swimmer_config(ns_f=200, nth_f=10, ns_q=1000, nth_q=20),
    # n = 13824: four cells in a coarser channel; 54 blocks of the two-level
    # factorisation, 38 update tiles per SM and block; FP64 matrix 1.5 GB, FP32 768 MB
    "channel_half": lambda: g.sperm_channel_config(count=4, wall_f=(60, 15, 8),
                                                   wall_q=(186, 46, 24)),
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
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, factor_schedule=args.factor_schedule)
    Y = g.initial_state(pr)
    ctx.set_state(Y["x0"], Y["B"])
    xi, Xiw, xidot = nrs.shapes_to_device(sh)
    x, Xw, b = ctx.kinematics(xi, Xiw, xidot)
    ctx.nearest_build(xi, Xiw)
    ctx.assemble(x, Xw, want_matrix=False)
    ctx.factor(args.prec)
    _, rep = ctx.solve(b, check=False)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "n": pr.n, "prec": args.prec, "report": rep[0],
                      "residuals": ctx.residual_counters()}))




def oracle_sample(pr, budget_rows=92, lu_n=6144, seed=0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of one RK2 step
    of ``pr`` (seconds per step, and what was measured): per stage the
    nearest-neighbour search and segments of every quadrature point
    (measured whole), the assembly of ``budget_rows`` sampled force points'
    rows (scaled by N / rows), the LAPACK LU of an n = ``lu_n`` system of the
    same workload's kind (scaled by (n / lu_n)^3) and one double-double
    residual at that size (scaled by (n / lu_n)^2, three per solve); a step is
    two stages."""
    import oracle as O
    import scipy.linalg as sla
    O.build()
    sh = g.pack_shapes(pr, 0.0)
    Y = g.initial_state(pr)
    t0 = time.perf_counter()
    nn = O.nearest(sh["x"], sh["Xw"], sh["n_off"], sh["q_off"], pr.nn_global)
    O.segments(nn, pr.N)
    t_nn = time.perf_counter() - t0
    x, Xw = O.lab_frame(sh, Y)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(pr.N, size=min(budget_rows, pr.N), replace=False))
    t0 = time.perf_counter()
    O.assemble_rows(rows, x, Xw, nn, pr.eps, pr.mu)
    t_asm = (time.perf_counter() - t0) * pr.N / len(rows)
    m = min(lu_n, pr.n)
    A = np.asfortranarray(rng.standard_normal((m, m)) + m * np.eye(m))
    bvec = rng.standard_normal(m)
    t0 = time.perf_counter()
    lu = sla.lu_factor(A, overwrite_a=False, check_finite=False)
    t_lu = (time.perf_counter() - t0) * (pr.n / m) ** 3
    xs = sla.lu_solve(lu, bvec, check_finite=False)
    t0 = time.perf_counter()
    O.residual_dd(A, xs, bvec)
    t_res = (time.perf_counter() - t0) * (pr.n / m) ** 2
    stage = t_nn + t_asm + t_lu + 3 * t_res
    return 2 * stage, {"nearest_s": t_nn, "assemble_s_scaled": t_asm, "lu_s_scaled": t_lu,
                       "residual_dd_s_scaled": t_res, "cores": O.threads(),
                       "sample": (f"per stage: nearest neighbours + segments of all {pr.Q} "
                                  f"quadrature points (measured); A_s rows of {len(rows)} of "
                                  f"{pr.N} force points (x {pr.N / len(rows):.0f}); LAPACK LU "
                                  f"at n = {m} (x (n/{m})^3); 3 double-double residuals at "
                                  f"n = {m} (x (n/{m})^2); a step = 2 stages")}


def cpu_baseline(pr):
    v, info = oracle_sample(pr)
    return {"value": v, "unit": "s/step", "cores": info.pop("cores"), "kind": "oracle",
            "sample": info.pop("sample"), "parts": info}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    pr = g.workload(HEADLINE)
    W = min(args.warmup, 1)
    K = min(args.steps, 5)
    times, info = [], None
    for s in range(W + K):
        v, info = oracle_sample(pr, seed=s)
        if s >= W:
            times.append(v)
    v = float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/step", "n_gpus": ws,
            "steps": len(times), "warmup": W, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS_DESC[HEADLINE],
                       "solver": "FP64 LAPACK LU + double-double refinement (oracle)"},
            "cpu_baseline": {"value": v, "unit": "s/step", "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"] + f"; {len(times)} sampled steps after {W}"},
            "e2e": {"value": v, "unit": "s/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    peaks, peak_src = _peaks()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    timer = _Timer(flush)
    H = headline(nrs, args, ws, local, timer, peaks, peak_src)
    pr, K = H["pr"], H["K"]
    s_per_step = H["t_max"] / K / ws  # whole job: ws replicas each advance K steps
    side = {}
    if not args.no_side and ws == 1:
        side["fresh_factor_graph"] = {"s_per_step": H["fresh_graph_s"], "steps": H["fresh_steps"],
                                      "note": "same workload, factor at every stage, the step "
                                              "recorded as a CUDA graph and replayed"}
        side["swimmers4"] = side_workload(nrs, args, "swimmers4", 1, 1, C2_SOLVER, timer)
        side["swimmer"] = side_workload(nrs, args, "swimmer", 20, 3, {}, timer, graph=True)
        side["swimmer_reuse"] = side_workload(nrs, args, "swimmer", 20, 3, HEADLINE_SOLVER, timer)
        side["tracers"] = tracers_line(nrs, args, timer)
        side["dormand_prince"] = dormand_prince_line(nrs, args)
        torch.cuda.empty_cache()
        side["plain_fp64"] = plain_fp64(nrs, args, timer)
        torch.cuda.empty_cache()
        side["factorisation"] = factorisation_line(
            nrs, args, timer, peaks, H["clocks"].get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0))
        torch.cuda.empty_cache()
    batch = None
    if not args.no_batch:
        batch = batch_bench(nrs, args, ws, rank)
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    recs = H["recs"]
    # the dominant kernel: the largest share of the step's critical path (a
    # launch that runs beside a longer one -- the FP64 assembly beside the
    # factorisation -- is off it)
    # (the factorisation's family is represented by its rank-256 updates)
    share = H["critical_share"]
    fams = {"lu": "lu_update" if "lu_update" in recs else "lu_diag",
            "assemble": "assemble", "assemble32": "assemble32", "krylov": "krylov"}
    top_fam = max((f for f, k in fams.items() if k in recs), key=lambda f: share.get(f, 0.0))
    top = fams[top_fam]
    roof = dict(recs[top], share_of_critical_path=share.get(top_fam, 0.0),
                share_of_phase_time=H["phase_share"].get(top, 0.0))
    plain = side.get("plain_fp64")
    line = {
        "metric": METRIC,
        "value": s_per_step,
        "unit": "s/step",
        "n_gpus": ws,
        "steps": K,
        "warmup": H["W"],
        "ms_per_step": H["t_max"] / K * 1e3,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (bit-exact assembly, extended-precision residual) + fp32 inverse "
                 "(tensor-core updates from scaled fp16 pairs)",
        "data": "synthetic (seeded channel, head and flagellum shapes)",
        "config": {"workload": WORKLOADS_DESC[HEADLINE], "factor": "FP32 explicit inverse (two-level "
                   "blocked Gauss-Jordan, rank-256 tensor-core updates from scaled FP16 pairs; "
                   f"--prec {args.prec}), refreshed after >40 GMRES iterations or 32 stages",
                   "refinement": "GMRES-IR, extended residual (exact fixed-point product sums; "
                                 "a float-pair residual while the backward error is >= 1e-8), "
                                 "GMRES products with the float-pair copy of A, inner tolerance "
                                 "1e-5, warm start from the previous stage",
                   "rk2_stages_per_step": 2,
                   "l2": "flushed between timed steps (512 MiB write); matrices 9.2 GB > L2",
                   "parallelism": f"replicas x{ws}"},
        "step_ms": H["step_ms"],
        "factorizations_per_step": H["counts"]["factorizations"] / K,
        "refinement": {"outer_mean": H["counts"]["outer"] / max(H["counts"]["solves"], 1),
                       "inner_mean": H["counts"]["inner"] / max(H["counts"]["solves"], 1),
                       "solves": H["counts"]["solves"],
                       "exact_residuals_mean": H["counts"]["residuals_exact"]
                       / max(H["counts"]["solves"], 1),
                       "working_residuals_mean": H["counts"]["residuals_working"]
                       / max(H["counts"]["solves"], 1),
                       "status_after_timed_region": H["status_after"],
                       "all_converged": True},
        "parity_vs_oracle": H["parity"],
        "pairs_per_s": recs.get("assemble", {}).get("pairs_per_s"),
        "pairs_per_s_fp32_copy": recs.get("assemble32", {}).get("achieved"),
        "phases_ms_per_step": H["phases_ms_per_step"],
        "phase_share": H["phase_share"],
        "critical_path_share": H["critical_share"],
        "fresh_factor_phases_ms_per_step": H["fresh_phases_ms_per_step"],
        "roofline": roof,
        "rooflines": recs,
        "fresh_factor_rooflines": H["fresh_recs"],
        "e2e": {"value": H["e2e_s"], "unit": "s/step", "h2d_bytes_per_step": H["h2d"],
                "d2h_bytes_per_step": H["d2h"], "steps": H["e2e_steps"]},
        "gpu_launches": H["launches"],
        "gpu_launches_note": "kernels launched by the library in the timed region (its count)",
        "clocks": H["clocks"],
        "side": side,
    }
    if plain:
        line["plain_fp64_s_per_step"] = plain["s_per_step"]
        line["mixed_vs_plain_speedup"] = plain["s_per_step"] / (H["t_max"] / K)
    if batch:
        line["batch"] = batch
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(pr)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def batch_bench(nrs, args, ws, rank):
    """The batch workload.  One rank: 128 ventral-node-like problems at
    reduced sizes (all of them) and the first 8 at the full sizes, one graph
    per batch step against stepping them one after the other, and all 128 at
    the full sizes (one timed batch step; --no-batch-full skips it).  Several ranks:
    each steps its own share of the 128 reduced problems (the library's LPT
    plan with one chain per rank, no collective in the data path); the time is
    the slowest rank's."""
    small = [g.node_config(i, cilia=(4, 12), floor=(160, 500), n_rod=10, q_rod=100, n_sphere=2,
                           q_sphere=8) for i in range(128)]
    recipe = "cilia 4-12 (10/100 points), floor 160-500 (x10), spheres 26/386"
    if ws > 1:
        mine = _rank_share([pr.n ** 3 for pr in small], ws, rank)
        res = _batch_case(nrs, [small[i] for i in mine], args.prec, 3, seq_steps=0)
        t = _max_over_ranks(res["s_per_batch_step"], ws)
        return {"workload": "ventral-node batch, reduced sizes, sharded over ranks",
                "recipe": recipe, "problems": len(small), "ranks": ws,
                "s_per_batch_step": t, "problem_steps_per_s": len(small) / t,
                "rank0_problems": len(mine)}
    full = [g.node_config(i) for i in range(8)]
    out = {"workload": "ventral-node batch: cilia rotating on tilted cones, static floor disc, "
                       "5 free spheres; eps 0.005",
           "reduced_128": dict(_batch_case(nrs, small, args.prec, 3), recipe=recipe),
           "full_first8": dict(_batch_case(nrs, full, args.prec, 2),
                               recipe="the batch recipe at full size, problems 0-7")}
    if not args.no_batch_full:
        import torch
        torch.cuda.empty_cache()
        probs = g.node_batch(128)
        plan = (out["full_first8"]["chains"], out["full_first8"]["solve_grid"])
        res = _batch_case(nrs, probs, args.prec, 1, tune=False, plan=plan, seq_steps=0)
        out["full_128"] = dict(res, recipe="all 128 problems at full size (n 5322-15771), plan "
                                           f"K = {plan[0]} chains, G = {plan[1]} (the autotuner's "
                                           "choice on the first 8), one timed batch step after "
                                           "the eager first step and the recorded second",
                               matrix_bytes=int(sum(12 * pr.n * pr.n for pr in probs)))
        del probs
        torch.cuda.empty_cache()
    return out


def profile_step(args):
    """Warm-up steps then one more step of --workload with the product path's
    settings (no timing loop): the command an ncu launch list captures."""
    import torch
    from paper_2001_06468_gb300 import nrs
    torch.cuda.set_device(0)
    pr = PROFILE_WORKLOADS[args.workload]()
    Y = g.initial_state(pr)
    solver = C2_SOLVER if args.workload == "swimmers4" else HEADLINE_SOLVER
    ctx = nrs.Context.from_problem(pr, factor_prec=args.prec, **solver)
    ctx.set_state(Y["x0"], Y["B"])
    for s in range(args.warmup + 1):
        d0 = nrs.shapes_to_device(g.pack_shapes(pr, s * pr.dt))
        dh = nrs.shapes_to_device(g.pack_shapes(pr, (s + 0.5) * pr.dt))
        rep = ctx.step(nrs.Context.shapes(*d0), nrs.Context.shapes(*dh), pr.dt)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "n": pr.n, "report": rep}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nrs", choices=["nrs", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp32", "tf32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch workload section")
    ap.add_argument("--no-batch-full", action="store_true",
                    help="skip the 128 full-size batch problems (about 180 GB of matrices)")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the other workloads and the plain FP64 comparator")
    ap.add_argument("--batch-full", action="store_true",
                    help="only the full-size batch of 128 problems (one JSON line)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="one kinematics + nearest + assemble + factor + solve on --workload, "
                         "then exit (for ncu captures)")
    ap.add_argument("--profile-step", action="store_true",
                    help="--warmup steps and one more of --workload, then exit (for ncu)")
    ap.add_argument("--workload", default="swimmer", choices=sorted(PROFILE_WORKLOADS))
    ap.add_argument("--factor-schedule", default="auto",
                    choices=["auto", "fused", "streams", "two_level", "two_level_tf32"],
                    help="factorisation schedule of --profile-solve")
    args = ap.parse_args()
    if args.profile_solve:
        profile_solve(args)
        return
    if args.profile_step:
        profile_step(args)
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
