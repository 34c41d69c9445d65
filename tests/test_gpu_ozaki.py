"""Split-precision (FP16-sliced, tensor-core) selected inversion against the
oracle and against the FP64 path.  Bound: selected-entry error below 1e-9
(each entry relative to the largest selected entry of its row and column)."""
from __future__ import annotations

import numpy as np
import pytest

import gen
from test_gpu_parity import TOL_FP64, compare_full, gpu_run, oracle_coo
from helpers import selected_error

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-9


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def force_split(h):
    """Every level on the sliced products (the default keeps small levels in
    FP64), so that the small test matrices exercise the tensor-core path."""
    import paper_1708_04539_gb300 as ps
    nlev = h.structure()["nlevels"]
    h.plan_set([(lev, 3, 0) for lev in range(nlev)], ps.PREC_OZAKI_FP16)


def run_split(torch, p, slices=0, all_levels=True, **kw):
    import paper_1708_04539_gb300 as ps
    h = ps.SelInv.from_problem(p, slices=slices, **kw)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    if all_levels:
        force_split(h)
    h.selinv(precision=ps.PREC_OZAKI_FP16)
    st = h.structure()
    sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    pa = h.get_selected()
    h.selinv(precision=ps.PREC_FP64)
    sn64 = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    h.sync()
    h.close()
    return st, sn, pa, sn64


CASES = [
    ("cfg1", lambda: gen.make_config(1)),
    ("upwind12", lambda: gen.upwind_3d(12, 61, max_sn=64)),
    ("upwind16_wide", lambda: gen.upwind_3d(16, 62, max_sn=256)),
    ("dg", lambda: gen.dg_blocks(3, 16, 63, max_sn=48)),
    ("random", lambda: gen.random_struct_sym(300, 0.02, 64, max_sn=24)),
    ("dense", lambda: gen.dense(200, 65, max_sn=40)),
]


@pytest.mark.parametrize("name,maker", CASES, ids=[c[0] for c in CASES])
def test_split_matches_oracle(torch, name, maker):
    p = maker()
    st, sn, pa, sn64 = run_split(torch, p)
    _, err = compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT)
    # and the FP64 path of the same handle
    scale = np.abs(sn64).max()
    assert np.abs(sn - sn64).max() <= 1e-9 * scale


@pytest.mark.parametrize("name,maker", CASES[1:4], ids=[c[0] for c in CASES[1:4]])
def test_split_normalise_option_matches_oracle(torch, name, maker):
    """Option: Lhat, Uhat^T and D_K as sliced products as well."""
    p = maker()
    st, sn, pa, sn64 = run_split(torch, p, split_normalise=True)
    compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT)
    assert np.abs(sn - sn64).max() <= 1e-9 * np.abs(sn64).max()


def test_default_level_mix_matches_oracle(torch):
    """The default per-level choice (small levels in FP64, the rest split)."""
    p = gen.upwind_3d(20, 72, max_sn=256)
    st, sn, pa, sn64 = run_split(torch, p, all_levels=False)
    compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT)


@pytest.mark.parametrize("name,maker", [CASES[0], CASES[2], CASES[3]],
                         ids=[CASES[0][0], CASES[2][0], CASES[3][0]])
@pytest.mark.parametrize("slices", [6, 5])
def test_a_operand_sources_agree(torch, name, maker, slices):
    """The sliced GEMM reading A straight from shared memory (default) and
    from tensor memory form the same exact integer sums: the sweeps agree to
    the order of the FP64 atomic accumulation onto D_K, and both meet the
    oracle."""
    p = maker()
    st, sn_t, _, _ = run_split(torch, p, slices=slices, ozaki_a_tmem=True)
    _, sn_s, _, _ = run_split(torch, p, slices=slices)
    scale = np.abs(sn_s).max()
    # the order of the FP64 atomic sums differs run to run and propagates
    # down the tree: agreement far below the split path's 1e-9 bound
    assert np.abs(sn_t - sn_s).max() <= 1e-12 * scale
    if slices == 6:
        compare_full(p, st, sn_t, 0, 20, tol=TOL_SPLIT)


@pytest.mark.parametrize("slices,bound", [(5, 1e-8), (4, 1e-6)])
def test_fewer_slices_lose_accuracy_gracefully(torch, slices, bound):
    p = gen.upwind_3d(10, 66, max_sn=64)
    st, sn, pa, sn64 = run_split(torch, p, slices=slices)
    err = np.abs(sn - sn64).max() / np.abs(sn64).max()
    assert err <= bound


def test_split_per_supernode_schedule(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_3d(9, 67, max_sn=64)
    st, sn, pa, sn64 = run_split(torch, p, schedule=ps.SCHED_PER_SUPERNODE)
    assert np.abs(sn - sn64).max() <= 1e-9 * np.abs(sn64).max()


COMPLEX_CASES = [
    ("stencil27_c", lambda: gen.stencil27_complex(8, 68, max_sn=64)),
    ("cfg3_small", lambda: gen.make_config(3, size=10)),
    ("grid2d_c", lambda: gen.conv_diff_2d(24, 69, imag_diag=0.1, max_sn=64)),
    ("random_c", lambda: gen.random_struct_sym(250, 0.03, 70, complex_values=True, max_sn=20)),
]


@pytest.mark.parametrize("name,maker", COMPLEX_CASES, ids=[c[0] for c in COMPLEX_CASES])
def test_split_complex_matches_oracle(torch, name, maker):
    """Complex products through the real embedding of the sliced GEMM."""
    p = maker()
    st, sn, pa, sn64 = run_split(torch, p)
    compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT)
    assert np.abs(sn - sn64).max() <= 1e-9 * np.abs(sn64).max()


def test_split_complex_shift_batch(torch):
    """Several complex shifts of one pattern (a pole-expansion batch)."""
    import paper_1708_04539_gb300 as ps
    p = gen.shifted_family(7, 71, nshift=4, max_sn=64)
    h = ps.SelInv.from_problem(p)
    h.factor(torch.from_numpy(p.values).cuda())
    force_split(h)
    h.selinv(precision=ps.PREC_OZAKI_FP16)
    st = h.structure()
    for b in range(p.nbatch):
        compare_full(p, st, h.get_selected(batch=b, layout=ps.LAYOUT_SUPERNODAL), b, 20,
                     tol=TOL_SPLIT)
    h.close()


@pytest.mark.slow
def test_split_config2_full_size(torch):
    p = gen.make_config(2)
    st, sn, pa, sn64 = run_split(torch, p, all_levels=False)
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    from helpers import selected_error
    rows, cols = supernodal_coordinates(st)
    err = selected_error(sn, sn64, rows, cols, p.n)
    assert err < TOL_SPLIT, err


@pytest.mark.parametrize("name,make", [CASES[2], CASES[3], ("upwind12_c", lambda: gen.stencil27_complex(8, 66, max_sn=64))],
                         ids=["upwind16_wide", "dg", "stencil27_c"])
@pytest.mark.parametrize("cfg", [1, 3], ids=["tiles32", "rows"])
def test_fp64_product_kernels_match_oracle(torch, name, make, cfg):
    """Every FP64 product of the sweep through one kernel -- 32 x 32 tiles or
    row panels (exact triangles for the normalisation's Lhat, Uhat^T and
    D_K; transposed G for step 5; atomic K chunks for step 4): the FP64 plan,
    and the split plan with every other level in FP64, over two sweeps of
    one handle."""
    import paper_1708_04539_gb300 as ps
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    p = make()
    h = ps.SelInv.from_problem(p)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    nlev = h.structure()["nlevels"]
    st = h.structure()
    h.plan_set([(lev, slot, cfg) for lev in range(nlev) for slot in (0, 1, 2)], ps.PREC_FP64)
    h.plan_set([(lev, slot, cfg) for lev in range(nlev) for slot in (0, 4, 5)] +
               [(lev, 3, lev % 2) for lev in range(nlev)], ps.PREC_OZAKI_FP16)
    _, orows, ocols, ovals = oracle_coo(p, 0, 20)
    grows, gcols = supernodal_coordinates(st)
    gi, oi = np.argsort(grows * p.n + gcols), np.argsort(orows * p.n + ocols)
    for rep in range(2):
        for prec, tol in ((ps.PREC_FP64, TOL_FP64), (ps.PREC_OZAKI_FP16, TOL_SPLIT)):
            h.selinv(precision=prec)
            sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
            err = selected_error(sn[gi], ovals[oi], orows[oi], ocols[oi], p.n)
            assert err < tol, (rep, prec, err)
    h.sync()
    h.close()


@pytest.mark.parametrize("name,maker", [CASES[3], COMPLEX_CASES[0]], ids=["dg", "stencil27_c"])
def test_split_checked_maps_match_oracle(torch, name, maker):
    """The gather of Ainv_CC with every index-map read bounds-checked
    (check_level = 1): same result, no error reported (h.sync())."""
    p = maker()
    st, sn, pa, sn64 = run_split(torch, p, check_level=1)
    compare_full(p, st, sn, 0, 20, tol=TOL_SPLIT)
