"""Split-precision factorisation: the Schur-complement products
L_{C,K} U_{K,C} of the supernodal LU (the factorisation that Algorithm 1
takes as given, Section 2) as sliced FP16 tensor-core products, against the
oracle LU and the oracle selected inverse.

Tolerances: factors 1e-10 and selected entries 1e-9 in the selected-entry
metric (each entry's error relative to the largest entry of its row and
column), the bar of the split-precision sweep; a slice set represents each
operand entry to 2^-42 of its row's maximum, so a Schur product of width s
errs by about s 2^-42 of the product of the row maxima.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from helpers import selected_error

pytestmark = pytest.mark.gpu

TOL_FACTOR = 1e-10
TOL_SPLIT = 1e-9


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def sorted_against_oracle(st, p, relax):
    from paper_1708_04539_gb300.binding import supernodal_coordinates
    s = oracle.analyze(p, relax_pct=relax)
    orows, ocols = s.lu_pattern()
    grows, gcols = supernodal_coordinates(st)
    gk, ok = grows * p.n + gcols, orows * p.n + ocols
    gi, oi = np.argsort(gk), np.argsort(ok)
    assert np.array_equal(gk[gi], ok[oi])
    return s, gi, oi, orows[oi], ocols[oi]


def run(torch, p, relax, split_factor, precision, mflops=-1):
    import paper_1708_04539_gb300 as ps
    kw = {}
    if split_factor:
        kw = {"factor_precision": ps.PREC_OZAKI_FP16, "factor_split_mflops": mflops}
    h = ps.SelInv.from_problem(p, relax_pct=relax, **kw)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    fac = h.get_selected(layout=ps.LAYOUT_FACTORS)
    if precision == ps.PREC_OZAKI_FP16:  # every level through the sliced products
        nlev = h.structure()["nlevels"]
        h.plan_set([(lev, 3, 0) for lev in range(nlev)], ps.PREC_OZAKI_FP16)
    h.selinv(precision=precision)
    sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    st = h.structure()
    h.sync()
    return h, st, fac, sn


CASES = [
    ("upwind12", lambda: gen.upwind_3d(12, 901, max_sn=64), 20),
    ("upwind16_wide", lambda: gen.upwind_3d(16, 902, max_sn=256), 20),
    ("stencil27_c", lambda: gen.stencil27_complex(8, 903, max_sn=64), 20),
    ("dg", lambda: gen.dg_blocks(3, 16, 904, max_sn=48), 20),
    ("random", lambda: gen.random_struct_sym(300, 0.02, 905, max_sn=24), 30),
    ("random_c", lambda: gen.random_struct_sym(250, 0.03, 906, complex_values=True, max_sn=20), 20),
]


@pytest.mark.parametrize("name,maker,relax", CASES, ids=[c[0] for c in CASES])
def test_split_factor_matches_oracle(torch, name, maker, relax):
    import paper_1708_04539_gb300 as ps
    p = maker()
    for prec in (ps.PREC_FP64, ps.PREC_OZAKI_FP16):
        h, st, fac, sn = run(torch, p, relax, True, prec)
        s, gi, oi, orows, ocols = sorted_against_oracle(st, p, relax)
        f = oracle.lu(s, p.colptr, p.rowind, p.values)
        ovals = np.concatenate([f.diag, f.low, f.up])[oi]
        err_f = selected_error(fac[gi], ovals, orows, ocols, p.n)
        assert err_f < TOL_FACTOR, err_f
        sel = oracle.selected_inverse(p, relax_pct=relax)
        rows, cols = sel.sym.lu_pattern()
        ok = rows * p.n + cols
        ref = sel.values_lu_order()[np.argsort(ok)]
        err = selected_error(sn[gi], ref, orows, ocols, p.n)
        assert err < TOL_SPLIT, (prec, err)
        # the factor plan ran sliced products on every level with work
        kinds = {s_["kind"] for s_ in h.profile(1)}
        assert "ozaki_gemm" in kinds
        h.close()


def test_split_factor_general_pattern(torch):
    """General pattern with static pivoting (C_L != C_U): the Schur products
    L_{R_L, K} U_{K, R_U} sliced, checked through the general oracle."""
    import paper_1708_04539_gb300 as ps
    from test_gpu_general import check_against_oracle
    for p in (gen.general_random(300, 0.01, 907, max_sn=16),
              gen.upwind_oneway_2d(30, 908, max_sn=32, complex_values=True)):
        h = ps.SelInv.from_general_problem(p, relax_pct=20, factor_precision=ps.PREC_OZAKI_FP16,
                                           factor_split_mflops=-1)
        h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
        fac = h.get_selected(layout=ps.LAYOUT_FACTORS)
        h.selinv(precision=ps.PREC_FP64)
        sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
        pa = h.get_selected()
        st = h.structure()
        h.sync()
        check_against_oracle(p, st, fac, sn, pa, tol=TOL_SPLIT, tol_factor=TOL_FACTOR)
        h.close()


def test_factor_precision_switch(torch):
    """Default threshold keeps a small matrix in FP64 (the FP64 plan, equal to
    the FP64 factorisation up to the order of the atomic scatter's sums);
    switching to every level split and back rebuilds the plan each time."""
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_3d(10, 909, max_sn=64)
    vals = torch.from_numpy(np.ascontiguousarray(p.values)).cuda()
    h = ps.SelInv.from_problem(p, relax_pct=20)
    h.factor(vals)
    f0 = h.get_selected(layout=ps.LAYOUT_FACTORS)
    h.set_factor_precision(ps.PREC_OZAKI_FP16)  # default threshold: too little work
    h.factor(vals)
    f1 = h.get_selected(layout=ps.LAYOUT_FACTORS)
    scale = np.abs(f0).max()
    assert np.abs(f1 - f0).max() <= 1e-13 * scale
    assert "ozaki_gemm" not in {s["kind"] for s in h.profile(1)}
    h.set_factor_precision(ps.PREC_OZAKI_FP16, -1)
    h.factor(vals)
    f2 = h.get_selected(layout=ps.LAYOUT_FACTORS)
    assert "ozaki_gemm" in {s["kind"] for s in h.profile(1)}
    assert 0 < np.abs(f2 - f0).max() <= 1e-10 * scale
    h.set_factor_precision(ps.PREC_FP64)
    h.factor(vals)
    assert np.abs(h.get_selected(layout=ps.LAYOUT_FACTORS) - f0).max() <= 1e-13 * scale
    assert "ozaki_gemm" not in {s["kind"] for s in h.profile(1)}
    with pytest.raises(ps.PselinvError):
        h.set_factor_precision(7)
    h.close()
