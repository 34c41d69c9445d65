"""bench.py's host-side arithmetic on synthetic launch records (no GPU): the
dominant-kernel roofline counts S (S + 1) / 2 tensor products per FP64
flop for the slice count of the run, takes the DRAM traffic of the captured
six-slice kernel only for six slices, and reports every kind's share."""
from __future__ import annotations

import bench


def _records():
    # two sliced-GEMM launches (1e12 FP64 flops each, 2 ms + 3 ms), one
    # gather-slice launch (4e9 bytes, 1 ms), one FP64 row-panel launch
    return [
        {"kind": "ozaki_gemm", "ms": 2.0, "flops": 1e12, "bytes": 1e9, "param": 1},
        {"kind": "ozaki_gemm", "ms": 3.0, "flops": 1e12, "bytes": 1e9, "param": 1},
        {"kind": "gather_slice", "ms": 1.0, "flops": 0.0, "bytes": 4e9, "param": -1},
        {"kind": "gemm", "ms": 0.5, "flops": 5e8, "bytes": 1e8, "param": 3},
    ]


def test_roofline_counts_slice_pairs():
    for slices, pairs in ((6, 21), (5, 15), (4, 10)):
        rec, kinds = bench.roofline_from_profile(_records(), slices, 1.25)
        assert rec["kernel"].startswith(f"ozaki_gemm_kernel<{slices}>")
        assert rec["tensor_flops_per_fp64_flop"] == pairs
        # 2e12 FP64 flops in 5 ms, times the slice pairs, in TFLOP/s
        assert abs(rec["achieved"] - pairs * 2e12 / 5e-3 / 1e12) < 1e-6 * rec["achieved"]
        assert abs(rec["frac"] - rec["achieved"] / rec["peak"]) < 1e-12
        if slices != bench.SLICES:
            assert rec["traffic"] is None  # the capture was of six slices
        assert abs(sum(k["share"] for k in kinds.values()) - 1.0) < 1e-12
        assert kinds["ozaki_gemm"]["launches"] == 2


def test_roofline_of_an_fp64_dominated_step():
    recs = [{"kind": "gemm", "ms": 4.0, "flops": 4e9, "bytes": 1e8, "param": 3},
            {"kind": "ozaki_gemm", "ms": 1.0, "flops": 1e9, "bytes": 1e8, "param": 1}]
    rec, _ = bench.roofline_from_profile(recs, 6, 1.25)
    assert rec["bound"] == "alu" and rec["peak"] == 1.25
    assert abs(rec["achieved"] - 4e9 / 4e-3 / 1e12) < 1e-12


def test_aggregate_throughput_over_replicas():
    value, ms = bench.aggregate_throughput(7.5e13, 2000.0, 2, 4)
    assert ms == 1000.0
    assert abs(value - 4 * 7.5e13 / 1.0 / 1e9) < 1e-6
