"""Pins of the general-pattern oracle (oracle/oracle_general.c): patterns that
are not structurally symmetric, and static pivoting P A Q with P != Q^T
(Section 1, Eq. sel_entries; Section 2, Theorem 1 with C_L != C_U,
Algorithm 1; Theorem 2).

Each test pins it to something other than itself: brute-force boolean
elimination, the double-double dense inverse (pinned in test_oracle_pins.py),
the triangular special case the paper states (only the diagonal is
selected, (A^{-1})_ii = 1/A_ii), the structurally symmetric oracle on
symmetric patterns, the transpose invariance, the row and column identities
that generalise Tr[A A^{-1}] = N, and planted mistakes.  Nothing here calls
the CUDA library.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
import oracle
from helpers import csc_cols, dense_inverse_ref


def pivoted_dense(p):
    """Atilde = P A Q as a dense array (rperm / cperm: new -> old)."""
    a = p.dense()
    return a[p.meta["rperm"]][:, p.meta["cperm"]]


def brute_structures(at):
    """C_L(k), C_U(k) by dense boolean elimination of Atilde (diagonal present)."""
    n = at.shape[0]
    F = at != 0
    np.fill_diagonal(F, True)
    cl, cu = [], []
    for k in range(n):
        rows = np.nonzero(F[k + 1:, k])[0] + k + 1
        cols = np.nonzero(F[k, k + 1:])[0] + k + 1
        cl.append(rows)
        cu.append(cols)
        F[np.ix_(rows, cols)] = True
    return cl, cu


CASES = [
    ("random", lambda: gen.general_random(45, 0.06, 401)),
    ("random_c", lambda: gen.general_random(40, 0.07, 402, complex_values=True)),
    ("oneway", lambda: gen.upwind_oneway_2d(8, 403, max_sn=16)),
    ("oneway_c", lambda: gen.upwind_oneway_2d(7, 404, max_sn=16, complex_values=True)),
    ("dense_rows", lambda: gen.general_random(30, 0.4, 405)),
    ("no_row_pivot", lambda: gen.general_random(35, 0.08, 406, row_scramble=False)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_structures_match_brute_force(name, make, oracle_lib):
    p = make()
    s = oracle.ganalyze(p)
    cl, cu = brute_structures(pivoted_dense(p))
    for k in range(p.n):
        assert np.array_equal(s.col_l(k), cl[k]), k
        assert np.array_equal(s.row_u(k), cu[k]), k
    if name != "dense_rows":
        assert s.nnzl != s.nnzu or any(not np.array_equal(s.col_l(k), s.row_u(k))
                                       for k in range(p.n))


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_selected_inverse_matches_double_double(name, make, oracle_lib):
    p = make()
    sel = oracle.general_selected_inverse(p)
    at = pivoted_dense(p)
    ref = (oracle.dense_inverse_dd_complex(at) if np.iscomplexobj(at)
           else np.sum(oracle.dense_inverse_dd(at), axis=0))
    rows, cols = sel.sym.inverse_pattern()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(sel.values() - ref[rows, cols])) <= 1e-13 * scale
    # the computed set is the pattern of (L+U)^T: it holds every (j, i) with Atilde_ij != 0
    ii, jj = np.nonzero(at)
    have = set(zip(rows.tolist(), cols.tolist()))
    assert all((j, i) in have for i, j in zip(ii.tolist(), jj.tolist()))


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_extraction_theorem2(name, make, oracle_lib):
    """out[p] = (A^{-1})_{x,y} for every entry A_{y,x} (Eq. sel_entries)."""
    p = make()
    sel = oracle.general_selected_inverse(p)
    out = oracle.gextract(sel, p.colptr, p.rowind)
    inv = dense_inverse_ref(p)
    x = csc_cols(p.colptr)
    assert np.max(np.abs(out - inv[x, p.rowind])) <= 1e-13 * np.max(np.abs(inv))


@pytest.mark.parametrize("triangle", ["upper", "lower"])
def test_triangular_selects_only_the_diagonal(triangle, oracle_lib):
    """Section 1: for a triangular matrix only the diagonal is selected and
    (A^{-1})_ii = 1 / A_ii; every other computed entry is an exact zero of
    the inverse's other triangle."""
    p = gen.general_random(30, 0.2, 407, triangle=triangle, row_scramble=False)
    at = pivoted_dense(p)
    sel = oracle.general_selected_inverse(p)
    assert np.array_equal(sel.bd, 1.0 / np.diag(at))
    assert np.all(sel.bl == 0) and np.all(sel.bu == 0)
    s = sel.sym
    if triangle == "upper":
        assert s.nnzl == 0
    else:
        assert s.nnzu == 0


@pytest.mark.parametrize("make", [
    lambda: gen.conv_diff_2d(9, 408, max_sn=16),
    lambda: gen.random_struct_sym(60, 0.06, 409, complex_values=True, permute=True),
    lambda: gen.upwind_3d(5, 410, max_sn=16),
])
def test_symmetric_pattern_equals_structurally_symmetric_oracle(make, oracle_lib):
    """P = Q^T on a structurally symmetric pattern: the general oracle gives,
    bit for bit, the structurally symmetric oracle's values (strict
    supernodes, so both use the exact fill)."""
    p = make()
    g = oracle.general_selected_inverse(p)
    s = oracle.selected_inverse(p, relax_pct=0)
    assert np.array_equal(g.sym.lptr, s.sym.sptr) and np.array_equal(g.sym.lidx, s.sym.sidx)
    assert np.array_equal(g.sym.uptr, s.sym.sptr) and np.array_equal(g.sym.uidx, s.sym.sidx)
    # general: BU holds B_{i,k} (i > k), BL holds B_{k,j}; symmetric oracle:
    # its lower array holds B_{i,k}, its upper array B_{k,j}
    assert np.array_equal(g.bu, s.low) and np.array_equal(g.bl, s.up)
    assert np.array_equal(g.bd, s.diag)


def _transpose_problem(p):
    """A^T with the row and column orderings swapped (Atilde' = Atilde^T)."""
    import scipy.sparse as sp
    a = sp.csc_matrix((p.values, p.rowind, p.colptr), shape=(p.n, p.n)).T.tocsc()
    a.sort_indices()
    return gen.Problem(p.name + "_T", p.n, a.indptr.astype(np.int64), a.indices.astype(np.int64),
                       a.data.copy(), p.meta["rperm"], p.max_supernode, p.dims,
                       meta={"rperm": p.meta["cperm"], "cperm": p.meta["rperm"]})


@pytest.mark.parametrize("name,make", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_transpose_invariance(name, make, oracle_lib):
    """selinv(A^T) = selinv(A)^T on the selected set."""
    p = make()
    q = _transpose_problem(p)
    a = oracle.general_selected_inverse(p)
    b = oracle.general_selected_inverse(q)
    ra, ca = a.sym.inverse_pattern()
    rb, cb = b.sym.inverse_pattern()
    va = dict(zip(zip(ra.tolist(), ca.tolist()), a.values()))
    vb = dict(zip(zip(cb.tolist(), rb.tolist()), b.values()))
    assert set(va) == set(vb)
    scale = max(abs(v) for v in va.values())
    assert max(abs(va[k] - vb[k]) for k in va) <= 1e-14 * scale


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_row_and_column_identities(name, make, oracle_lib):
    """sum_j A_ij (A^{-1})_ji = 1 and sum_i (A^{-1})_ji A_ij = 1 for every
    row i and column j: both use only selected entries (the extraction
    returns (A^{-1})_{x,y} for each entry A_{y,x})."""
    p = make()
    out = oracle.gextract(oracle.general_selected_inverse(p), p.colptr, p.rowind)
    x = csc_cols(p.colptr)
    prod = p.values * out
    row = np.zeros(p.n, dtype=prod.dtype)
    col = np.zeros(p.n, dtype=prod.dtype)
    np.add.at(row, p.rowind, prod)
    np.add.at(col, x, prod)
    scale = np.zeros(p.n)
    np.add.at(scale, p.rowind, np.abs(prod))
    assert np.max(np.abs(row - 1) / scale) <= 1e-13
    cs = np.zeros(p.n)
    np.add.at(cs, x, np.abs(prod))
    assert np.max(np.abs(col - 1) / cs) <= 1e-13


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mutation, oracle_lib):
    p = gen.upwind_oneway_2d(8, 411, max_sn=16)
    at = pivoted_dense(p)
    ref = np.sum(oracle.dense_inverse_dd(at), axis=0)
    try:
        sel = oracle.general_selected_inverse(p, mutation=mutation)
    except oracle.OracleError:
        return  # a read outside the pattern of (L+U)^T: caught
    rows, cols = sel.sym.inverse_pattern()
    assert np.max(np.abs(sel.values() - ref[rows, cols])) > 1e-6 * np.max(np.abs(ref))
