"""General patterns with static pivoting on the GPU (pselinv_analyze_general):
the factors and the selected inverse against the general oracle, element by
element (Section 2, Theorem 1 with C_L != C_U; Algorithm 1; Theorem 2 with
P != Q^T).  Tolerances as for the structurally symmetric path: factors 1e-12
normwise, selected entries 1e-10 in the selected-entry metric."""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from helpers import selected_error

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


CASES = [
    ("random", lambda: gen.general_random(300, 0.01, 601, max_sn=16)),
    ("random_c", lambda: gen.general_random(250, 0.012, 602, complex_values=True, max_sn=16)),
    ("oneway", lambda: gen.upwind_oneway_2d(30, 603, max_sn=32)),
    ("oneway_c", lambda: gen.upwind_oneway_2d(24, 604, max_sn=32, complex_values=True)),
    ("oneway_wide", lambda: gen.upwind_oneway_2d(40, 605, max_sn=128)),
    ("upper", lambda: gen.general_random(120, 0.05, 606, triangle="upper", row_scramble=False)),
    ("lower", lambda: gen.general_random(120, 0.05, 607, triangle="lower", row_scramble=False)),
    ("sym_pattern", lambda: gen.conv_diff_2d(20, 608, max_sn=32)),
]


def run_general(torch, p, relax=20, split=False, **kw):
    import paper_1708_04539_gb300 as ps
    h = ps.SelInv.from_general_problem(p, relax_pct=relax, **kw)
    h.factor(torch.from_numpy(np.ascontiguousarray(p.values)).cuda())
    fac = h.get_selected(layout=ps.LAYOUT_FACTORS)
    if split:  # every level through the sliced tensor-core products
        nlev = h.structure()["nlevels"]
        h.plan_set([(lev, 3, 0) for lev in range(nlev)], ps.PREC_OZAKI_FP16)
    h.selinv(precision=ps.PREC_OZAKI_FP16 if split else ps.PREC_FP64)
    sn = h.get_selected(layout=ps.LAYOUT_SUPERNODAL)
    pa = h.get_selected()
    st = h.structure()
    h.sync()
    return h, st, fac, sn, pa


def factor_coordinates(st):
    """(rows, cols) of the factor entry each storage slot holds: diagonal
    block (L below, U on and above), L panel L_{R_L, K}, U^T panel
    (U_{K, R_U})^T."""
    from paper_1708_04539_gb300.binding import inverse_coordinates
    r, c = inverse_coordinates(st)
    rows, cols = r.copy(), c.copy()
    for K in range(int(st["nsuper"])):
        o, s = int(st["sn_offset"][K]), int(st["sn_width"][K])
        cl = int(st["rows_ptr"][K + 1] - st["rows_ptr"][K])
        a, b = o + s * s, o + s * s + cl * s  # L panel: (K, R_L) -> (R_L, K)
        rows[a:b], cols[a:b] = c[a:b], r[a:b]
        e = b + int(st["urows_ptr"][K + 1] - st["urows_ptr"][K]) * s  # U^T: (R_U, K) -> (K, R_U)
        rows[b:e], cols[b:e] = c[b:e], r[b:e]
    return rows, cols


def check_against_oracle(p, st, fac, sn, pa, tol=TOL, tol_factor=1e-12):
    from paper_1708_04539_gb300.binding import inverse_coordinates
    n = p.n
    g = oracle.ganalyze(p)
    ofac = oracle.glu(g, p.colptr, p.rowind, p.values)
    osel = oracle.gselinv(ofac)
    # factors on the oracle's pattern of L+U
    frows, fcols = factor_coordinates(st)
    fkey = {k: i for i, k in enumerate((frows * n + fcols).tolist())}
    kl = np.repeat(np.arange(n), np.diff(g.lptr))
    ku = np.repeat(np.arange(n), np.diff(g.uptr))
    lr = np.concatenate([np.arange(n), g.lidx, ku])
    lc = np.concatenate([np.arange(n), kl, g.uidx])
    lv = np.concatenate([ofac.diag, ofac.low, ofac.up])
    idx = np.array([fkey[k] for k in (lr * n + lc).tolist()])
    assert np.max(np.abs(fac[idx] - lv)) <= tol_factor * np.max(np.abs(lv))
    # every slot outside the oracle's pattern holds an explicit zero of L + U
    rest = np.ones(fac.size, dtype=bool)
    rest[idx] = False
    assert np.max(np.abs(fac[rest]), initial=0.0) <= tol_factor * np.max(np.abs(lv))
    # selected inverse on the oracle's pattern of (L+U)^T
    rows, cols = inverse_coordinates(st)
    key = {k: i for i, k in enumerate((rows * n + cols).tolist())}
    orows, ocols = g.inverse_pattern()
    ov = osel.values()
    idx = np.array([key[k] for k in (orows * n + ocols).tolist()])
    err = selected_error(sn[idx], ov, orows, ocols, n)
    assert err < tol, err
    # extraction (Theorem 2): (A^{-1})_{x,y} for every entry A_{y,x}
    ref = oracle.gextract(osel, p.colptr, p.rowind)
    assert np.max(np.abs(pa - ref)) <= tol * np.max(np.abs(ref))
    return err


@pytest.mark.parametrize("relax", [0, 20])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_general_matches_oracle(torch, name, make, relax):
    p = make()
    h, st, fac, sn, pa = run_general(torch, p, relax=relax)
    assert st["general"]
    check_against_oracle(p, st, fac, sn, pa)
    h.close()


def test_general_per_supernode_schedule_and_checked_maps(torch):
    import paper_1708_04539_gb300 as ps
    p = gen.upwind_oneway_2d(20, 609, max_sn=32)
    h, st, fac, sn, pa = run_general(torch, p, schedule=ps.SCHED_PER_SUPERNODE, check_level=1)
    check_against_oracle(p, st, fac, sn, pa)
    h.close()


@pytest.mark.parametrize("name,make", [CASES[0], CASES[1], CASES[2], CASES[4], CASES[5]],
                         ids=["random", "random_c", "oneway", "oneway_wide", "upper"])
def test_general_split_matches_oracle(torch, name, make):
    """The sliced tensor-core products on every level: G_K = Ainv(R_U, R_L)
    gathered and sliced in both layouts, steps 3-5 as sliced products."""
    p = make()
    h, st, fac, sn, pa = run_general(torch, p, split=True)
    check_against_oracle(p, st, fac, sn, pa, tol=1e-9)
    h.close()


def test_general_trace(torch):
    """Tr[A A^{-1}] = n (Section 1) from the selected entries alone."""
    p = gen.general_random(200, 0.02, 610, max_sn=16)
    h, st, fac, sn, pa = run_general(torch, p)
    tr = h.trace(np.array([1.0]), p.values)
    assert abs(tr - p.n) <= 1e-10 * p.n
    h.close()
