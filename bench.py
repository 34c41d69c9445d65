#!/usr/bin/env python
"""Benchmark of the selected-inversion hot path on one GB300 (or N replicas).

Default workload: the block-sparse DG operator of 16^3 elements x 64 unknowns
(n = 262,144, FP64), nested dissection on the element grid, supernodes of
at most 256 columns: the largest single-GPU workload of the benchmark set.
One step = pselinv_selinv (normalisation + the whole root-to-leaf sweep) +
extraction of the selected entries on the pattern of A, with the LU factors
resident in HBM.  The factorisation is timed separately (and inside the
end-to-end figure).  ``--config 2`` runs the 40^3 upwind convection-diffusion
matrix instead (``--config 3`` / ``4``: the complex and pole-batch workloads).

Metric: FP64-equivalent GFLOP/s of selected inversion, counting
sum_K 4 c^2 s + 4 c s^2 + 4/3 s^3 over the strict (unrelaxed) supernodes.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(the single-matrix path has no exchange step); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "selinv_fp64_equiv_gflops"
UNIT = "GFLOP/s"
HEADLINE_CONFIG = 5
WORKLOADS = {
    1: "2D 5-point convection-diffusion {m}^2 (n={n}), FP64, nested dissection, max supernode 64",
    2: "3D 7-point upwind convection-diffusion {m}^3 (n={n}), FP64, nested dissection, "
       "max supernode 256, relaxed supernodes (<=20% explicit zeros)",
    3: "3D 27-point complex operator A = H - zS + 0.2N on a {m}^3 grid (n={n}), complex128, "
       "nested dissection, max supernode 256",
    4: "pole-expansion batch: 40 complex shifts of a 3D 7-point {m}^3 operator (n={n}), "
       "complex128, one sweep for all shifts, max supernode 256",
    5: "block-sparse DG operator: {m}^3 elements x 64 unknowns (n={n}), dense element and "
       "upwind face blocks, FP64, nested dissection on the element grid, max supernode 256, "
       "relaxed supernodes (<=20% explicit zeros)",
}
DEFAULT_SIZE = {1: 31, 2: 40, 3: 60, 4: 32, 5: 16}
# unknowns of the leading nested-dissection subdomain the CPU oracle is timed on
SAMPLE_TARGET_N = {1: 961, 2: 4000, 3: 2000, 4: 4000, 5: 2048}
# smaller matrices of the same family whose tuner records train the cost model
TRAIN_SIZES = {2: (20, 24, 28), 5: (8, 10, 12)}
SLICES = 6


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--schedule", default="level", choices=["level", "per_supernode"])
    ap.add_argument("--precision", default="ozaki", choices=["fp64", "ozaki"],
                    help="ozaki: FP16-sliced tensor-core products (default); fp64: every product in FP64")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 level-batched / per-supernode comparison and error report")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned cost model against the exhaustive tuner and the heuristic")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="end-to-end steps (default 5; 1 for the DG operator, whose "
                         "factorisation dominates)")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the launch-by-launch replay (roofline fields become null)")
    ap.add_argument("--tune", default="exhaustive", choices=["none", "exhaustive"],
                    help="launch-shape autotuning before the timed region (untimed, like the factorisation)")
    ap.add_argument("--plan-out", default=None,
                    help="write the tuned launch shapes (JSON triples) to this path")
    ap.add_argument("--plan-in", default=None,
                    help="replay launch shapes written by --plan-out instead of tuning "
                         "(profiling runs: timings under a profiler would mislead the tuner)")
    ap.add_argument("--dump-profile", default=None,
                    help="write the launch-by-launch profile (JSON) to this path")
    ap.add_argument("--factor-precision", default="auto", choices=["auto", "fp64", "ozaki"],
                    help="Schur products of the factorisation: auto = the sweep's precision")
    ap.add_argument("--slices", type=int, default=0, choices=[0, 4, 5, 6],
                    help="FP16 slices per operand of the split products (0: the library's "
                         "default, 6)")
    ap.add_argument("--ozaki-a-tmem", action="store_true",
                    help="sliced GEMM reads its A slices from tensor memory (default: from "
                         "shared memory)")
    ap.add_argument("--capture", action="store_true",
                    help="profiler runs: one factorisation and one sweep (plan from --plan-in, "
                         "or the untuned heuristic), nothing timed, no JSON line")
    ap.add_argument("--split-normalise", action="store_true",
                    help="also slice the normalisation and D_K (by default they stay FP64)")
    ap.add_argument("--size", type=int, default=None,
                    help="grid side (elements per side for the DG operator; default: the "
                         "configuration's own; smaller for profiling captures)")
    ap.add_argument("--config", type=int, default=HEADLINE_CONFIG, choices=[1, 2, 3, 4, 5],
                    help="5: 16^3 x 64 DG operator (default); 1: 31^2 convection-diffusion; "
                         "2: 40^3 upwind; 3: 60^3 complex 27-point; 4: 40 complex shifts of a "
                         "32^3 operator and 64 uneven 2D grids in one sweep")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def leading_subdomain(p, target):
    """The leading nested-dissection subdomain of ``p`` with at most ``target``
    unknowns, as a Problem in the permuted ordering (identity perm).

    The factor of a leading principal submatrix of the permuted matrix is the
    leading block of the whole factor, so the elimination tree of the first
    M = 4 target columns, analysed alone, gives the subtree sizes there."""
    import scipy.sparse as sp

    import gen
    import oracle

    n = p.n
    M = min(n, 4 * target)
    cols = np.repeat(np.arange(n), np.diff(p.colptr))
    iperm = np.empty(n, dtype=np.int64)
    iperm[p.perm] = np.arange(n)
    r, c = iperm[p.rowind], iperm[cols]
    keep = (r < M) & (c < M)
    vals = p.values if p.values.ndim == 1 else p.values[0]
    a = sp.csc_matrix((vals[keep], (r[keep], c[keep])), shape=(M, M))
    a.sort_indices()
    lead = gen.Problem(f"{p.name}_prefix{M}", M, a.indptr.astype(np.int64),
                       a.indices.astype(np.int64), a.data.copy(), np.arange(M, dtype=np.int64),
                       p.max_supernode)
    s = oracle.analyze(lead, relax_pct=0)
    size = np.ones(M, dtype=np.int64)
    for j in range(M):
        if s.parent[j] >= 0:
            size[s.parent[j]] += size[j]
    # walk up from column 0: the largest complete subtree that is exactly the
    # leading columns [0, m) with m <= target
    m, j = 1, 0
    while j >= 0 and size[j] <= target:
        if size[j] == j + 1:
            m = j + 1
        j = int(s.parent[j])
    b = a[:m, :m].tocsc()
    b.sort_indices()
    return gen.Problem(f"{p.name}_lead{m}", m, b.indptr.astype(np.int64),
                       b.indices.astype(np.int64), b.data.copy(), np.arange(m, dtype=np.int64),
                       p.max_supernode)


def exact_flops(sym):
    w = np.diff(sym.supptr).astype(float)
    c = np.array([sym.supernode_rows(k).size for k in range(sym.nsup)], dtype=float)
    return float(np.sum(4 * c * c * w + 4 * c * w * w + 4.0 / 3.0 * w ** 3))


class OracleSample:
    def __init__(self, p, target):
        import oracle
        self.q = leading_subdomain(p, target)
        self.sym = oracle.analyze(self.q, relax_pct=0)
        self.fac = oracle.lu(self.sym, self.q.colptr, self.q.rowind, self.q.values)
        self.flops = exact_flops(self.sym) * (4.0 if np.iscomplexobj(self.q.values) else 1.0)
        self.desc = (f"selected inversion (Theorem 1 oracle) of the leading nested-dissection "
                     f"subdomain of the same matrix: n={self.q.n}, {self.flops:.3e} flop; "
                     f"LU untimed")

    def step(self, threads=1):
        import oracle
        t0 = time.perf_counter()
        if threads == 1:
            oracle.selinv(self.fac)
        else:
            oracle.selinv_parallel(self.fac, threads)
        return time.perf_counter() - t0


def cpu_baseline(p, target, min_seconds=6.0, max_reps=5):
    """The oracle on every host core (independent columns of one depth, or one
    column's dot products, in parallel), with its single-thread time beside it."""
    smp = OracleSample(p, target)
    cores = host_cores()
    single = smp.step(1)
    times = []
    while len(times) < max_reps and (sum(times) < min_seconds or len(times) < 1):
        times.append(smp.step(cores))
    t = statistics.median(times)
    return {"value": smp.flops / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": smp.desc, "seconds_per_sample": t, "reps": len(times),
            "single_thread": {"value": smp.flops / single / 1e9, "cores": 1,
                              "seconds_per_sample": single}}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


GEMM_TEMPLATES = {0: "64,64,16", 1: "32,32,16", 2: "128,64,8"}  # tile config -> BM,BN,BK (3: row panels)


def roofline_from_profile(prof, slices, fp64_peak):
    """Roofline record of the kernel kind with the largest share of the step."""
    kinds = {}
    for r in prof:
        k = kinds.setdefault(r["kind"], {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0})
        k["launches"] += 1
        k["ms"] += r["ms"]
        k["flops"] += r["flops"]
        k["bytes"] += r["bytes"]
    tot = sum(k["ms"] for k in kinds.values())
    for k in kinds.values():
        k["share"] = k["ms"] / tot if tot else 0.0
    if not kinds:
        return None, kinds
    top = max(kinds, key=lambda k: kinds[k]["ms"])
    k = kinds[top]
    by_param = {}
    for r in prof:
        if r["kind"] == top:
            by_param[r.get("param", -1)] = by_param.get(r.get("param", -1), 0.0) + r["ms"]
    main_param = max(by_param, key=by_param.get) if by_param else -1
    sec = k["ms"] * 1e-3
    peaks = measured_peaks()
    if top == "gemm":
        achieved = k["flops"] / sec / 1e12
        if main_param == 3:  # row panels (the normalisation's triangular products)
            name, tkey = "rows_gemm_kernel<double> (FP64 DFMA)", "rows_gemm_kernel_f64"
        else:
            tile = GEMM_TEMPLATES.get(main_param, "?")
            name, tkey = f"gemm_kernel<double,{tile}> (FP64 DFMA)", "gemm_kernel_f64"
        rec = {"bound": "alu", "kernel": name,
               "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
               "peak_source": "measured in this run: pselinv_measure_fp64_peak (FP64 FMA loop "
                              "on every SM; mma.sync f64 measured slower on GB300)",
               "traffic": traffic_from_profiles(tkey)}
    elif top == "ozaki_gemm":
        pairs = slices * (slices + 1) // 2
        achieved = pairs * k["flops"] / sec / 1e12
        peak = float(peaks.get("bf16_tflops", 1925.5))
        rec = {"bound": "tensor", "kernel": f"ozaki_gemm_kernel<{slices}> (tcgen05 kind::f16)",
               "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "peak_source": "measured bf16 dense peak (MEASURED_PEAKS.json) x 1.0 nominal "
                              "fp16/bf16 ratio",
               "tensor_flops_per_fp64_flop": pairs,
               # captured with the default six slices
               "traffic": traffic_from_profiles("ozaki_gemm") if slices == SLICES else None}
    else:
        achieved = k["bytes"] / sec / 1e9
        peak = float(peaks.get("hbm_gbs", 6778.7))
        rec = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
               "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
               "traffic": traffic_from_profiles(top)}
    rec["frac"] = rec["achieved"] / rec["peak"]
    rec["share_of_step"] = k["share"]
    rec["launches_per_step"] = k["launches"]
    return rec, {n: {"launches": v["launches"], "ms": v["ms"], "share": v["share"]}
                 for n, v in kinds.items()}


def path_roofline(st, cplx, nbatch, ms_step, fp64_peak, split, slices=SLICES):
    """Path-level roofline of one sweep from its level structure.

    Per supernode (width s, c = |R_K|, relaxed structure): products of steps
    3-5 P = 4 c^2 s + 2 c s^2, FP64 normalisation and diagonal block
    F = 2 c s^2 + 4/3 s^3, algorithmic bytes (c^2 + 2 (2 c s + s^2)) w (G read
    once, panels read and written).  FP64 roofline of level l:
    min(P_fp64, AI_l x HBM) over all its flops; split roofline: the sliced
    products at the tensor peak (21 slice products each) or HBM, whichever
    is slower, plus F at the FP64 peak (S (S + 1) / 2 slice products for S
    slices).  frac = roofline time / measured."""
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6778.7)) * 1e9
    tensor = float(peaks.get("bf16_tflops", 1925.5)) * 1e12
    p64 = fp64_peak * 1e12
    mult = (4.0 if cplx else 1.0) * nbatch
    w = (16.0 if cplx else 8.0)
    width = np.asarray(st["sn_width"], dtype=float)
    c = np.diff(np.asarray(st["rows_ptr"])).astype(float)
    depth = np.asarray(st["sn_depth"])
    prod = (4 * c * c * width + 2 * c * width * width) * mult
    norm = (2 * c * width * width + 4.0 / 3.0 * width ** 3) * mult
    byts = (c * c + 2 * (2 * c * width + width * width)) * w * nbatch
    t64 = tsplit = 0.0
    pairs = slices * (slices + 1) // 2
    for lev in range(int(st["nlevels"])):
        m = depth == lev
        f, b = float((prod[m] + norm[m]).sum()), float(byts[m].sum())
        if f <= 0:
            continue
        t64 += f / min(p64, f / b * hbm)
        tsplit += max(float(prod[m].sum()) * pairs / tensor, b / hbm) + float(norm[m].sum()) / p64
    sec = ms_step * 1e-3
    out = {"fp64_roofline_ms": t64 * 1e3, "frac_vs_fp64_roofline": t64 / sec,
           "definition": "sum over depth levels of flops_l / min(P_fp64, AI_l x HBM), over the "
                         "measured step (the split path may exceed 1)"}
    if split:
        out.update({"split_roofline_ms": tsplit * 1e3, "frac_vs_split_roofline": tsplit / sec,
                    "split_definition": "per level max(21 x products / tensor peak, bytes / HBM) "
                                        "+ FP64 normalisation / P_fp64, over the measured step"})
    return out


def _supernode_blocks(st, K):
    """(offset, s, first column, R_K) of supernode K of the storage."""
    s = int(st["sn_width"][K])
    f = int(st["sn_first"][K])
    R = st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]]
    return int(st["sn_offset"][K]), s, f, R


def selected_error_supernodal(st, x, r):
    """Error of the supernodal storage x against r (device tensors of one
    instance): max over every stored entry (i, j) of |x_ij - r_ij| /
    max(max_k |r_ik|, max_k |r_kj|), the maxima over the stored entries of
    row i and column j; and the normwise error max |x - r| / max |r|.
    Computed supernode by supernode on the device."""
    import torch
    n = int(st["n"])
    dev = r.device
    ra = r.abs() if not r.is_complex() else r.abs()
    rowmax = torch.zeros(n, dtype=torch.float64, device=dev)
    colmax = torch.zeros(n, dtype=torch.float64, device=dev)
    views = []
    for K in range(int(st["nsuper"])):
        o, s, f, R = _supernode_blocks(st, K)
        c = R.size
        Rd = torch.from_numpy(np.ascontiguousarray(R)).to(dev)
        d = ra[o:o + s * s].view(s, s)                    # [col][row]: (f+i, f+j) at i + j s
        rowmax[f:f + s] = torch.maximum(rowmax[f:f + s], d.amax(dim=0))
        colmax[f:f + s] = torch.maximum(colmax[f:f + s], d.amax(dim=1))
        if c:
            lp = ra[o + s * s:o + s * s + c * s].view(s, c)   # [t][p] = (R[p], f+t)
            up = ra[o + s * s + c * s:o + s * s + 2 * c * s].view(s, c)  # [t][p] = (f+t, R[p])
            rowmax[Rd] = torch.maximum(rowmax[Rd], lp.amax(dim=0))
            colmax[f:f + s] = torch.maximum(colmax[f:f + s], lp.amax(dim=1))
            rowmax[f:f + s] = torch.maximum(rowmax[f:f + s], up.amax(dim=1))
            colmax[Rd] = torch.maximum(colmax[Rd], up.amax(dim=0))
        views.append((o, s, f, c, Rd))
    worst = torch.zeros((), dtype=torch.float64, device=dev)
    for o, s, f, c, Rd in views:
        rm, cm = rowmax[f:f + s], colmax[f:f + s]
        e = (x[o:o + s * s] - r[o:o + s * s]).abs().view(s, s)
        rho = torch.maximum(rm[None, :], cm[:, None])
        worst = torch.maximum(worst, (e / torch.where(rho > 0, rho, 1.0)).max())
        if c:
            a, b = o + s * s, o + s * s + c * s
            e = (x[a:b] - r[a:b]).abs().view(s, c)
            rho = torch.maximum(rowmax[Rd][None, :], cm[:, None])
            worst = torch.maximum(worst, (e / torch.where(rho > 0, rho, 1.0)).max())
            e = (x[b:b + c * s] - r[b:b + c * s]).abs().view(s, c)
            rho = torch.maximum(rm[:, None], colmax[Rd][None, :])
            worst = torch.maximum(worst, (e / torch.where(rho > 0, rho, 1.0)).max())
    normwise = float((x - r).abs().max() / ra.max())
    return float(worst), normwise


def time_steps(h, prec, stream, steps, out_dev, warm=True):
    """Mean ms of `steps` sweeps + extractions (CUDA events on `stream`)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        if warm:
            h.selinv(precision=prec, stream=stream)
            h.get_selected(out_dev, stream=stream)
        e0.record(stream)
        for _ in range(steps):
            h.selinv(precision=prec, stream=stream)
            h.get_selected(out_dev, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def comparison(p, h, stream, out_dev, flops, big, refactor=None, option_arm=True):
    """FP64 level-batched and FP64 per-supernode sweeps of the same matrix,
    and the error of the split-precision result against the FP64 one.

    big: the FP64 arms take about a minute each, so they run the built-in
    heuristic plan once (no tuning, no repeat; the plan is built before the
    timed call).  refactor: the values, when the handle's factors came from
    split Schur products; the FP64 arms then run on an FP64 factorisation
    (timed), and the error covers both split stages."""
    import torch
    import paper_1708_04539_gb300 as ps
    st = h.structure()
    cplx = np.iscomplexobj(p.values)
    odt = torch.complex128 if cplx else torch.float64
    total = int(st["storage_size"])
    split = torch.empty(total, dtype=odt, device="cuda")
    ref = torch.empty(total, dtype=odt, device="cuda")
    with torch.cuda.stream(stream):
        h.selinv(precision=ps.PREC_OZAKI_FP16, stream=stream)
        h.get_selected(split, layout=ps.LAYOUT_SUPERNODAL, stream=stream)
    torch.cuda.synchronize()
    fp64_factor_ms = None
    if refactor is not None:
        h.set_factor_precision(ps.PREC_FP64)
        with torch.cuda.stream(stream):
            h.factor(refactor, stream=stream)  # builds the FP64 factorisation plan
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.factor(refactor, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        fp64_factor_ms = e0.elapsed_time(e1)
    h.tune(precision=ps.PREC_FP64, mode=ps.TUNE_RESET if big else ps.TUNE_EXHAUSTIVE,
           stream=stream)
    fp64_level_ms = time_steps(h, ps.PREC_FP64, stream, 1 if big else 3, out_dev, warm=not big)
    with torch.cuda.stream(stream):
        h.get_selected(ref, layout=ps.LAYOUT_SUPERNODAL, stream=stream)
    torch.cuda.synchronize()
    err, normwise = selected_error_supernodal(st, split, ref)
    split_sweep_err = None
    if refactor is not None:  # the split sweep alone, on the FP64 factors
        with torch.cuda.stream(stream):
            h.selinv(precision=ps.PREC_OZAKI_FP16, stream=stream)
            h.get_selected(split, layout=ps.LAYOUT_SUPERNODAL, stream=stream)
        torch.cuda.synchronize()
        split_sweep_err, _ = selected_error_supernodal(st, split, ref)
    del split
    h.set_schedule(ps.SCHED_PER_SUPERNODE)
    h.tune(precision=ps.PREC_FP64, mode=ps.TUNE_RESET, stream=stream)  # builds its plan
    per_sn_ms = time_steps(h, ps.PREC_FP64, stream, 1 if big else 2, out_dev, warm=not big)
    h.set_schedule(ps.SCHED_LEVEL)
    out = {"fp64_level_batched_ms": fp64_level_ms,
           "fp64_level_batched_gflops": flops / (fp64_level_ms * 1e-3) / 1e9,
           "fp64_level_plan": "heuristic" if big else "exhaustive",
           "fp64_per_supernode_ms": per_sn_ms,
           "fp64_per_supernode_gflops": flops / (per_sn_ms * 1e-3) / 1e9,
           "split_vs_fp64_selected_error": err, "split_vs_fp64_normwise_error": normwise,
           "split_covers": "factorisation Schur products and sweep" if refactor is not None
                           else "sweep",
           "error_metric": "max |x - r| / max(max_k |r_ik|, max_k |r_kj|) over every entry "
                           "of the pattern of L+U; r = FP64 GPU result (FP64 factorisation "
                           "and FP64 sweep)"}
    if refactor is not None:
        out.update({"fp64_factor_ms": fp64_factor_ms,
                    "split_sweep_on_fp64_factors_selected_error": split_sweep_err})
    if not big and option_arm:
        # option: normalisation and D_K as sliced products too
        q = ps.SelInv.from_problem(p, relax_pct=20, split_normalise=True)
        with torch.cuda.stream(stream):
            q.factor(torch.from_numpy(p.values).cuda(), stream=stream)
            q.tune(precision=ps.PREC_OZAKI_FP16, mode=ps.TUNE_EXHAUSTIVE, stream=stream)
        sn_ms = time_steps(q, ps.PREC_OZAKI_FP16, stream, 5, out_dev)
        qx = torch.empty(total, dtype=odt, device="cuda")
        with torch.cuda.stream(stream):
            q.get_selected(qx, layout=ps.LAYOUT_SUPERNODAL, stream=stream)
        torch.cuda.synchronize()
        sn_err, _ = selected_error_supernodal(st, qx, ref)
        q.close()
        out.update({"split_normalise_option_ms": sn_ms,
                    "split_normalise_option_gflops": flops / (sn_ms * 1e-3) / 1e9,
                    "split_normalise_option_error": sn_err})
    del ref
    return out


def train_cost_model(config, prec, stream):
    """A cost model trained on the exhaustive tuner's records of smaller
    matrices of the same family (never on the benchmark matrix itself)."""
    import torch

    import gen
    import paper_1708_04539_gb300 as ps
    recs, names = [], []
    for size in TRAIN_SIZES[config]:
        if config == 5:
            q = gen.dg_blocks(size, 64, 1708045390 + 50 + size, max_sn=256)
        else:
            q = gen.upwind_3d(size, 1708045390 + 80 + size, max_sn=256)
        g = ps.SelInv.from_problem(q, relax_pct=20)
        with torch.cuda.stream(stream):
            g.factor(torch.from_numpy(q.values).cuda(), stream=stream)
            g.tune(precision=prec, mode=ps.TUNE_EXHAUSTIVE, stream=stream)
        recs += g.tune_records()
        names.append(f"n={q.n}")
        g.close()
    m = ps.CostModel(hidden=32, seed=5)
    loss = m.train(recs, epochs=4000, lr=3e-3, stream=stream)
    return m, {"records": len(recs), "matrices": names, "final_loss": loss,
               "network": "16 -> 32 -> 32 -> 1 tanh MLP, full-batch Adam, 4000 epochs"}


def learned_vs_exhaustive(h, prec, stream, out_dev, model, info, exhaustive_ms, triples):
    """Sweep time of the heuristic plan, the model-tuned plan and the
    exhaustive plan (already timed); the exhaustive plan is restored after."""
    import paper_1708_04539_gb300 as ps
    h.tune(precision=prec, mode=ps.TUNE_RESET, stream=stream)
    heur = time_steps(h, prec, stream, 3, out_dev)
    h.tune(precision=prec, mode=ps.TUNE_MODEL, model=model, stream=stream)
    mod = time_steps(h, prec, stream, 3, out_dev)
    h.plan_set(triples, prec)
    return dict(info, heuristic_ms=heur, model_ms=mod, exhaustive_ms=exhaustive_ms,
                regret_vs_exhaustive=(mod - exhaustive_ms) / exhaustive_ms,
                gain_over_heuristic=heur / mod)


def max_over_ranks(value, dist, device):
    """Largest value over all ranks (the job's time is its slowest replica)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(flops_per_rank, elapsed_ms_max, steps, world):
    """Whole-job throughput (GFLOP/s) of `world` replicas that each ran `steps`
    steps of `flops_per_rank` in at most `elapsed_ms_max` ms."""
    ms_per_step = elapsed_ms_max / steps
    return world * flops_per_rank / (ms_per_step * 1e-3) / 1e9, ms_per_step


def traffic_from_profiles(kernel):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel)
    if not ent:
        return None
    import hashlib
    src = os.path.join(ROOT, "paper_1708_04539_gb300", "csrc", ent["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return ent["bytes_per_launch"] if sha == ent.get("source_sha") else None


def group_problem(fam, grids):
    """The pole-expansion batch as one direct sum: each shift of `fam` and
    each grid a member, in member order (the pattern the library's
    pselinv_group forms; the values concatenated the same way)."""
    import gen
    patterns = [fam] + list(grids)
    member_of = [0] * fam.nbatch + list(range(1, len(grids) + 1))
    cps, ris, vals = [np.zeros(1, dtype=np.int64)], [], []
    n = nnz = 0
    for k, i in enumerate(member_of):
        q = patterns[i]
        cps.append(q.colptr[1:] + nnz)
        ris.append(q.rowind + n)
        vals.append(fam.values[k] if i == 0 else q.values)
        n += q.n
        nnz += q.nnz
    return gen.Problem("pole_batch", n, np.concatenate(cps), np.concatenate(ris),
                       np.concatenate([np.asarray(v, dtype=np.complex128) for v in vals]),
                       np.arange(n, dtype=np.int64), fam.max_supernode,
                       meta={"members": patterns, "member_of": member_of, "family_n": fam.n})


_T0 = time.perf_counter()


def log(msg):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def workload_name(config, size, n):
    return WORKLOADS[config].format(m=size, n=n)


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gen
    config = args.config
    size = args.size or DEFAULT_SIZE[config]
    p = gen.make_config(config, size=args.size)
    if config == 4:
        p = p[0]
    smp = OracleSample(p, SAMPLE_TARGET_N[config])
    cores = host_cores()
    for _ in range(args.warmup):
        smp.step(cores)
    times = [smp.step(cores) for _ in range(args.steps)]
    t = sum(times) / len(times)
    value = smp.flops / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if np.iscomplexobj(p.values) else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(config, size, p.n), "sample": smp.desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": smp.desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    import gen
    import paper_1708_04539_gb300 as ps
    from paper_1708_04539_gb300.binding import measure_fp64_peak

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    from paper_1708_04539_gb300 import build as libbuild
    if rank == 0 or world == 1:
        libbuild.build()
    if dist is not None:
        dist.barrier()
    ps.load_library()

    config = args.config
    p = gen.make_config(config, size=args.size)
    nmat = 1
    sample_p = p
    if config == 4:
        # the pole-expansion batch: every shift of the 3D operator and every
        # uneven 2D grid is a member of one group (pselinv_group), so one
        # sweep with one launch per kernel kind and level covers all of them
        fam, grids = p[0], p[1:]
        sample_p = fam
        p = group_problem(fam, grids)
        nmat = fam.nbatch + len(grids)
    size = args.size or DEFAULT_SIZE[config]
    workload = workload_name(config, size, p.n if config != 4 else p.meta["family_n"])
    big = config == 5 and size >= 14
    headline = config in (2, 5)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else (1 if big else 5)
    cplx = np.iscomplexobj(p.values)
    nbatch = p.nbatch
    sched = ps.SCHED_PER_SUPERNODE if args.schedule == "per_supernode" else ps.SCHED_LEVEL
    log(f"workload generated: n={p.n} nnz={p.nnz}")
    fprec_name = args.precision if args.factor_precision == "auto" else args.factor_precision
    fprec = ps.PREC_OZAKI_FP16 if fprec_name == "ozaki" else ps.PREC_FP64
    hkw = dict(relax_pct=20, schedule=sched, use_graph=not args.no_graph,
               split_normalise=args.split_normalise, factor_precision=fprec,
               slices=args.slices, ozaki_a_tmem=args.ozaki_a_tmem)
    if config == 4:
        members = [ps.SelInv.from_problem(q, host_only=True, relax_pct=20)
                   for q in p.meta["members"]]
        h = ps.SelInv.group([members[i] for i in p.meta["member_of"]], max_supernode=256, **hkw)
        for m in members:
            m.close()
    else:
        h = ps.SelInv.from_problem(p, **hkw)
    st = h.structure()
    log(f"analysed: {int(st['nsuper'])} supernodes, {int(st['nlevels'])} levels")
    # FP64-equivalent flops of one sweep over every instance (x4 for complex)
    flops = float(st["flops_selinv_exact"]) * (4.0 if cplx else 1.0) * nbatch
    stream = torch.cuda.Stream()
    vals_dev = torch.from_numpy(p.values).cuda()
    odt = torch.complex128 if cplx else torch.float64
    out_dev = torch.zeros((nbatch, p.nnz), dtype=odt, device="cuda")

    # factorisation: the first call builds its plan (untimed); it is timed
    # inside the end-to-end step below (and here when there is none)
    with torch.cuda.stream(stream):
        h.factor(vals_dev, stream=stream)
    torch.cuda.synchronize()
    if args.capture:  # one sweep for a profiler
        prec = ps.PREC_OZAKI_FP16 if args.precision == "ozaki" else ps.PREC_FP64
        if args.plan_in:
            with open(args.plan_in) as f:
                h.plan_set([tuple(t) for t in json.load(f)["triples"]], prec)
        with torch.cuda.stream(stream):
            h.selinv(precision=prec, stream=stream)
            h.get_selected(out_dev[0], stream=stream)
        torch.cuda.synchronize()
        if args.dump_profile:  # the plan's launches with their algorithmic work
            with open(args.dump_profile, "w") as f:
                json.dump({"config": config, "size": size,
                           "steps": h.profile(0, stream=stream)}, f)
        h.close()
        log("capture run done")
        return 0
    factor_ms = None
    if e2e_steps <= 0:
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.factor(vals_dev, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        factor_ms = e0.elapsed_time(e1)
    fp64_peak, _ = measure_fp64_peak(stream)
    log(f"factorised; FP64 peak {fp64_peak:.3f} TFLOP/s")

    prec = ps.PREC_OZAKI_FP16 if args.precision == "ozaki" else ps.PREC_FP64
    learned = (not args.no_learned and rank == 0 and world == 1 and headline and
               args.tune == "exhaustive" and not args.plan_in and config in TRAIN_SIZES)
    model = model_info = None
    if learned:
        model, model_info = train_cost_model(config, prec, stream)
        log(f"cost model trained on {model_info['records']} records")
    tune_s = 0.0
    tuning = args.tune
    if args.plan_in:
        with open(args.plan_in) as f:
            h.plan_set([tuple(t) for t in json.load(f)["triples"]], prec)
        tuning = "replayed"
    elif args.tune == "exhaustive":
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            h.tune(precision=prec, mode=ps.TUNE_EXHAUSTIVE, stream=stream)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
    triples = h.plan_get(prec)
    log(f"tuned in {tune_s:.1f} s")
    if args.plan_out:
        with open(args.plan_out, "w") as f:
            json.dump({"precision": args.precision, "config": config, "size": size,
                       "triples": triples}, f)

    def step():
        h.selinv(precision=prec, stream=stream)
        for b in range(nbatch):
            h.get_selected(out_dev[b], batch=b, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        time.sleep(0.25)
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    h.sync(stream=stream)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    value, ms_per_step = aggregate_throughput(flops, elapsed_ms, args.steps, world)
    log(f"timed: {ms_per_step:.3f} ms per step, {value:.1f} GFLOP/s")

    # launch-by-launch replay with CUDA events on the same stream
    prof = [] if args.no_profile else h.profile(0, stream=stream)
    nslices = args.slices or SLICES
    roofline, kinds = roofline_from_profile(prof, nslices, fp64_peak)
    if roofline is not None:
        roofline["path"] = path_roofline(st, cplx, nbatch, ms_per_step / 1.0, fp64_peak,
                                         prec == ps.PREC_OZAKI_FP16, nslices)
    if args.dump_profile and rank == 0:
        with torch.cuda.stream(stream):
            fprof = [] if big else h.profile(1, stream=stream)
            h.profile(2, stream=stream)  # warm the multi-stream timeline once
            timeline = h.profile(2, stream=stream)
        with open(args.dump_profile, "w") as f:
            json.dump({"precision": args.precision, "config": config, "size": size, "steps": prof,
                       "factor_steps": fprof, "timeline": timeline}, f)

    # the learned cost model against the exhaustive tuner and the heuristic
    learned_rec = None
    if learned:
        learned_rec = learned_vs_exhaustive(h, prec, stream, out_dev[0], model, model_info,
                                            ms_per_step, triples)
        model.close()
        log("learned vs exhaustive done")

    # end to end through the C ABI with host buffers: H2D values, factor,
    # selected inversion, D2H of the selected entries
    e2e = None
    if e2e_steps > 0:
        vals_host = torch.from_numpy(p.values.copy()).pin_memory()
        out_host = torch.zeros((nbatch, p.nnz), dtype=odt).pin_memory()
        fe0, fe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def e2e_step(time_factor):
            if time_factor:
                fe0.record(stream)
            h.factor(vals_host, stream=stream)
            if time_factor:
                fe1.record(stream)
            h.selinv(precision=prec, stream=stream)
            for b in range(nbatch):
                h.get_selected(out_host[b], batch=b, stream=stream)

        # one untimed step: a plan rebuilt by the tuning above records its
        # CUDA graph on its first call
        with torch.cuda.stream(stream):
            e2e_step(False)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(e2e_steps):
                e2e_step(i == 0)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, "cuda")
        factor_ms = fe0.elapsed_time(fe1)
        io_bytes = int(p.nnz * nbatch * (16 if cplx else 8))
        e2e = {"value": world * flops / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
               "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
               "includes": "H2D values, factor, selinv, extract, D2H"}
        del vals_host, out_host
        log(f"end to end {e2e_s * 1e3:.1f} ms")

    stats = h.plan_stats()
    nl = stats["launches_selinv"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("c128" if cplx else "f64") + ("" if args.precision == "fp64" else "+f16-slices"),
        "data": "synthetic (seeded generator, nested dissection)",
        "precision": args.precision,
        "config": {"workload": workload, "n": p.n, "nnz": p.nnz, "instances": nbatch * nmat,
                   "supernodes": int(st["nsuper"]), "levels": int(st["nlevels"]),
                   "flops_per_matrix": flops / nbatch,
                   "flops_relaxed_structure": st["flops_selinv"] * (4.0 if cplx else 1.0),
                   "schedule": args.schedule, "cuda_graph": not args.no_graph,
                   "normalisation": "split" if args.split_normalise else "fp64",
                   "factor_schur_products": fprec_name,
                   "tuning": tuning, "tuning_seconds": tune_s,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (%.0f MB of factors read per step)"
                         % (st["storage_size"] * (16 if cplx else 8) * nbatch / 1e6)},
        "time_per_matrix_ms": ms_per_step / (nbatch * nmat),
        "matrices_per_step": nbatch * nmat,
        "factor_ms": factor_ms,
        "e2e": e2e,
        "gpu_launches": int((nl + nbatch) * args.steps),
        "launches_per_sweep": int(nl),
        "launches_factor": int(stats["launches_factor"]),
        "fp64_peak_tflops": fp64_peak,
        "roofline": roofline,
        "kernel_shares": kinds,
        "clocks": clk.summary(),
    }
    if not prof:
        line["roofline"] = None
    if learned_rec is not None:
        line["learned"] = learned_rec
    if not args.no_compare and args.precision == "ozaki" and rank == 0:
        line["comparison"] = comparison(p, h, stream, out_dev[0], flops, big,
                                        vals_dev if fprec == ps.PREC_OZAKI_FP16 else None,
                                        option_arm=config != 4)
        log("comparison done")
    h.close()
    if rank == 0 and world == 1 and not args.skip_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sample_p, SAMPLE_TARGET_N[config])
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
