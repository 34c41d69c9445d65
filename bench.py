#!/usr/bin/env python
"""Benchmark of the selected-inversion hot path on one GB300 (or N replicas).

Workload: 3D 7-point upwind convection-diffusion on a 40^3 grid
(n = 64,000, FP64), nested-dissection ordering, supernodes of at most 256
columns.  One step = pselinv_selinv (normalisation + the whole root-to-leaf
sweep) + extraction of the selected entries on the pattern of A, with the
LU factors resident in HBM.  The factorisation is timed separately.

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
WORKLOAD = ("3D 7-point upwind convection-diffusion 40^3 (n=64000), FP64, nested dissection, "
            "max supernode 256, relaxed supernodes (<=20% explicit zeros)")
OTHER_WORKLOADS = {
    3: "3D 27-point complex operator A = H - zS + 0.2N on a {m}^3 grid (n={n}), complex128, "
       "nested dissection, max supernode 256",
    4: "pole-expansion batch: 40 complex shifts of a 3D 7-point {m}^3 operator (n={n}), "
       "complex128, one sweep for all shifts, max supernode 256",
    5: "block-sparse DG operator: {m}^3 elements x 64 unknowns (n={n}), dense element and "
       "upwind face blocks, FP64, nested dissection on the element grid, max supernode 256",
}
# FP64 DFMA pipe of GB300: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.07 GHz max SM clock
FP64_ALU_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
SAMPLE_TARGET_N = 4000  # unknowns of the leading nested-dissection subdomain timed on the CPU


def parse():
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
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
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
    ap.add_argument("--split-normalise", action="store_true",
                    help="also slice the normalisation and D_K (by default they stay FP64)")
    ap.add_argument("--size", type=int, default=None,
                    help="grid side (default: the configuration's own; 40 for the benchmark "
                         "workload; smaller for profiling captures)")
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5],
                    help="2: 40^3 upwind (the benchmark workload); 3: 60^3 complex 27-point; "
                         "4: 40 complex shifts of a 32^3 operator; 5: 16^3 x 64 DG operator")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def leading_subdomain(p, target):
    """The leading nested-dissection subdomain of ``p`` with at most ``target``
    unknowns, as a Problem in the permuted ordering (identity perm)."""
    import scipy.sparse as sp

    import gen
    import oracle

    s = oracle.analyze(p, relax_pct=0)
    n = p.n
    size = np.ones(n, dtype=np.int64)
    for j in range(n):
        if s.parent[j] >= 0:
            size[s.parent[j]] += size[j]
    # walk up from column 0: the largest complete subtree that is exactly the
    # leading columns [0, m) with m <= target
    m, j = 1, 0
    while j >= 0 and size[j] <= target:
        if size[j] == j + 1:
            m = j + 1
        j = int(s.parent[j])
    iperm = np.empty(n, dtype=np.int64)
    iperm[p.perm] = np.arange(n)
    cols = np.repeat(np.arange(n), np.diff(p.colptr))
    a = sp.csc_matrix((p.values, (iperm[p.rowind], iperm[cols])), shape=(n, n))[:m, :m].tocsc()
    a.sort_indices()
    return gen.Problem(f"{p.name}_lead{m}", m, a.indptr.astype(np.int64),
                       a.indices.astype(np.int64), a.data.copy(), np.arange(m, dtype=np.int64),
                       p.max_supernode)


def exact_flops(sym):
    w = np.diff(sym.supptr).astype(float)
    c = np.array([sym.supernode_rows(k).size for k in range(sym.nsup)], dtype=float)
    return float(np.sum(4 * c * c * w + 4 * c * w * w + 4.0 / 3.0 * w ** 3))


class OracleSample:
    def __init__(self, p):
        import oracle
        self.q = leading_subdomain(p, SAMPLE_TARGET_N)
        self.sym = oracle.analyze(self.q, relax_pct=0)
        self.fac = oracle.lu(self.sym, self.q.colptr, self.q.rowind, self.q.values)
        self.flops = exact_flops(self.sym)
        self.desc = (f"selected inversion (Theorem 1 oracle, single thread) of the leading "
                     f"nested-dissection subdomain of the same matrix: n={self.q.n}, "
                     f"{self.flops:.3e} flop; LU untimed")

    def step(self):
        import oracle
        t0 = time.perf_counter()
        oracle.selinv(self.fac)
        return time.perf_counter() - t0


def cpu_baseline(p, min_seconds=10.0, max_reps=5):
    smp = OracleSample(p)
    times = []
    while len(times) < max_reps and (sum(times) < min_seconds or len(times) < 1):
        times.append(smp.step())
    t = statistics.median(times)
    return {"value": smp.flops / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": smp.desc, "seconds_per_sample": t, "reps": len(times)}


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


def roofline_from_profile(prof, slices):
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
               "achieved": achieved, "peak": FP64_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
               "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
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
               "traffic": traffic_from_profiles("ozaki_gemm")}
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


def selected_error(x, r, rows, cols, n):
    """max |x - r| / max(row max, column max of |r|) over the entries given."""
    a = np.abs(r)
    rowmax = np.zeros(n)
    colmax = np.zeros(n)
    np.maximum.at(rowmax, rows, a)
    np.maximum.at(colmax, cols, a)
    rho = np.maximum(rowmax[rows], colmax[cols])
    rho[rho == 0] = 1.0
    return float(np.max(np.abs(x - r) / rho))


def time_steps(h, prec, stream, steps, out_dev):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        h.selinv(precision=prec, stream=stream)
        h.get_selected(out_dev, stream=stream)
        e0.record(stream)
        for _ in range(steps):
            h.selinv(precision=prec, stream=stream)
            h.get_selected(out_dev, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def comparison(p, h, stream, out_dev, flops):
    """FP64 level-batched and FP64 per-supernode sweeps of the same matrix,
    and the error of the split-precision result against the FP64 one."""
    import torch
    import paper_1708_04539_gb300 as ps
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    st = h.structure()
    rows, cols = supernodal_coordinates(st)
    h.selinv(precision=ps.PREC_OZAKI_FP16, stream=stream)
    split = h.get_selected(layout=ps.LAYOUT_SUPERNODAL, stream=stream)
    h.tune(precision=ps.PREC_FP64, mode=ps.TUNE_EXHAUSTIVE, stream=stream)
    fp64_level_ms = time_steps(h, ps.PREC_FP64, stream, 3, out_dev)
    ref = h.get_selected(layout=ps.LAYOUT_SUPERNODAL, stream=stream)
    err = selected_error(split, ref, rows, cols, p.n)
    normwise = float(np.max(np.abs(split - ref)) / np.max(np.abs(ref)))
    g = ps.SelInv.from_problem(p, relax_pct=20, schedule=ps.SCHED_PER_SUPERNODE)
    with torch.cuda.stream(stream):
        g.factor(torch.from_numpy(p.values).cuda(), stream=stream)
    per_sn_ms = time_steps(g, ps.PREC_FP64, stream, 2, out_dev)
    g.close()
    # option: normalisation and D_K as sliced products too
    q = ps.SelInv.from_problem(p, relax_pct=20, split_normalise=True)
    with torch.cuda.stream(stream):
        q.factor(torch.from_numpy(p.values).cuda(), stream=stream)
        q.tune(precision=ps.PREC_OZAKI_FP16, mode=ps.TUNE_EXHAUSTIVE, stream=stream)
    sn_ms = time_steps(q, ps.PREC_OZAKI_FP16, stream, 5, out_dev)
    sn_err = selected_error(q.get_selected(layout=ps.LAYOUT_SUPERNODAL, stream=stream), ref,
                            rows, cols, p.n)
    q.close()
    return {"fp64_level_batched_ms": fp64_level_ms,
            "fp64_level_batched_gflops": flops / (fp64_level_ms * 1e-3) / 1e9,
            "fp64_per_supernode_ms": per_sn_ms,
            "fp64_per_supernode_gflops": flops / (per_sn_ms * 1e-3) / 1e9,
            "split_vs_fp64_selected_error": err, "split_vs_fp64_normwise_error": normwise,
            "split_normalise_option_ms": sn_ms,
            "split_normalise_option_gflops": flops / (sn_ms * 1e-3) / 1e9,
            "split_normalise_option_error": sn_err,
            "error_metric": "max |x - r| / max(max_k |r_ik|, max_k |r_kj|) over every entry "
                            "of the pattern of L+U; r = FP64 GPU result"}


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


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import gen
    p = gen.make_config(2)
    smp = OracleSample(p)
    for _ in range(args.warmup):
        smp.step()
    times = [smp.step() for _ in range(args.steps)]
    t = sum(times) / len(times)
    value = smp.flops / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": smp.desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": smp.desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    import gen
    import paper_1708_04539_gb300 as ps

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

    p = gen.make_config(args.config, size=args.size)
    if args.config == 4:
        p = p[0]  # the shift family (the uneven grids are a parity case)
    size = args.size or {2: 40, 3: 60, 4: 32, 5: 16}[args.config]
    if args.config == 2:
        workload = WORKLOAD if size == 40 else WORKLOAD.replace(
            "40^3 (n=64000)", f"{size}^3 (n={size ** 3})")
    else:
        workload = OTHER_WORKLOADS[args.config].format(m=size, n=p.n)
    cplx = np.iscomplexobj(p.values)
    nbatch = p.nbatch
    headline = args.config == 2
    sched = ps.SCHED_PER_SUPERNODE if args.schedule == "per_supernode" else ps.SCHED_LEVEL
    h = ps.SelInv.from_problem(p, relax_pct=20, schedule=sched, use_graph=not args.no_graph,
                               split_normalise=args.split_normalise)
    st = h.structure()
    # FP64-equivalent flops of one sweep over every instance (x4 for complex)
    flops = float(st["flops_selinv_exact"]) * (4.0 if cplx else 1.0) * nbatch
    stream = torch.cuda.Stream()
    vals_dev = torch.from_numpy(p.values).cuda()
    odt = torch.complex128 if cplx else torch.float64
    out_dev = torch.zeros((nbatch, p.nnz), dtype=odt, device="cuda")

    # factorisation (timed separately)
    with torch.cuda.stream(stream):
        h.factor(vals_dev, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.factor(vals_dev, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    factor_ms = e0.elapsed_time(e1)

    prec = ps.PREC_OZAKI_FP16 if args.precision == "ozaki" else ps.PREC_FP64
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
    if args.plan_out:
        with open(args.plan_out, "w") as f:
            json.dump({"precision": args.precision, "config": args.config, "size": size,
                       "triples": h.plan_get(prec)}, f)

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

    # launch-by-launch replay with CUDA events on the same stream
    prof = [] if args.no_profile else h.profile(0, stream=stream)
    roofline, kinds = roofline_from_profile(prof, slices=6)
    if args.dump_profile and rank == 0:
        with torch.cuda.stream(stream):
            fprof = h.profile(1, stream=stream)
            h.profile(2, stream=stream)  # warm the multi-stream timeline once
            timeline = h.profile(2, stream=stream)
        with open(args.dump_profile, "w") as f:
            json.dump({"precision": args.precision, "config": args.config, "size": size, "steps": prof,
                       "factor_steps": fprof, "timeline": timeline}, f)

    # end to end through the C ABI with host buffers: H2D values, factor,
    # selected inversion, D2H of the selected entries
    e2e = None
    if args.e2e_steps > 0:
        vals_host = torch.from_numpy(p.values.copy()).pin_memory()
        out_host = torch.zeros((nbatch, p.nnz), dtype=odt).pin_memory()

        def e2e_step():
            h.factor(vals_host, stream=stream)
            h.selinv(precision=prec, stream=stream)
            for b in range(nbatch):
                h.get_selected(out_host[b], batch=b, stream=stream)

        with torch.cuda.stream(stream):
            e2e_step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for _ in range(args.e2e_steps):
                e2e_step()
        torch.cuda.synchronize()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, "cuda")
        io_bytes = int(p.nnz * nbatch * (16 if cplx else 8))
        e2e = {"value": world * flops / e2e_s / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
               "ms_per_step": e2e_s * 1e3,
               "includes": "H2D values, factor, selinv, extract, D2H"}

    stats = h.plan_stats()
    nl = stats["launches_selinv"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("c128" if cplx else "f64") + ("" if args.precision == "fp64" else "+f16-slices"),
        "data": "synthetic (seeded generator, nested dissection)",
        "precision": args.precision,
        "config": {"workload": workload, "n": p.n, "nnz": p.nnz, "instances": nbatch,
                   "supernodes": int(st["nsuper"]), "levels": int(st["nlevels"]),
                   "flops_per_matrix": flops / nbatch,
                   "flops_relaxed_structure": st["flops_selinv"] * (4.0 if cplx else 1.0),
                   "schedule": args.schedule, "cuda_graph": not args.no_graph,
                   "normalisation": "split" if args.split_normalise else "fp64",
                   "tuning": tuning, "tuning_seconds": tune_s,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (%.0f MB of factors read per step)"
                         % (st["storage_size"] * 8 / 1e6)},
        "time_per_matrix_ms": ms_per_step / nbatch,
        "factor_ms": factor_ms,
        "e2e": e2e,
        "gpu_launches": int((nl + 1) * args.steps),
        "launches_factor": int(stats["launches_factor"]),
        "roofline": roofline,
        "kernel_shares": kinds,
        "clocks": clk.summary(),
    }
    if not prof:
        line["roofline"] = None
    if not args.no_compare and args.precision == "ozaki" and rank == 0 and headline:
        line["comparison"] = comparison(p, h, stream, out_dev[0], flops)
    h.close()
    if rank == 0 and world == 1 and not args.skip_cpu_baseline and headline and size == 40:
        line["cpu_baseline"] = cpu_baseline(p)
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
