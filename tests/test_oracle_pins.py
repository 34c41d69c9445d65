"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA library.  Each test pins the oracle to something
other than itself: closed forms, brute force on tiny inputs, a
double-double dense inverse, LAPACK (numpy.linalg) as an independent
library routine, and identities the selected inverse must satisfy.  The last
tests plant mistakes in the oracle (its ``mutation`` switch) and check that
the pins catch every one of them.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle
from helpers import csc_cols, dense_inverse_ref, normwise_error, selected_error

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def brute_symbolic(problem):
    """Dense boolean symbolic elimination of P A P^T: struct(j) and parent(j)."""
    n = problem.n
    perm = problem.perm
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    F = np.zeros((n, n), dtype=bool)
    cols = csc_cols(problem.colptr)
    F[iperm[problem.rowind], iperm[cols]] = True
    np.fill_diagonal(F, True)
    for k in range(n):
        rows = np.nonzero(F[k + 1:, k])[0] + k + 1
        colsu = np.nonzero(F[k, k + 1:])[0] + k + 1
        F[np.ix_(rows, colsu)] = True
    structs = [np.nonzero(F[j + 1:, j])[0] + j + 1 for j in range(n)]
    parent = np.array([s[0] if s.size else -1 for s in structs], dtype=np.int64)
    return structs, parent


def sel_coo(sel):
    rows, cols = sel.sym.lu_pattern()
    return rows, cols, sel.values_lu_order()


def sel_vs_dense(sel, ainv_dense):
    """Selected entries (permuted indices) against a dense inverse in original order."""
    rows, cols, vals = sel_coo(sel)
    p = sel.sym.perm
    ref = ainv_dense[p[rows], p[cols]]
    return selected_error(vals, ref, rows, cols, sel.sym.n), normwise_error(vals, ref)


SMALL = [
    ("tridiag", lambda c: gen.tridiagonal(40, 11, complex_values=c)),
    ("arrow", lambda c: gen.arrow(30, 12, complex_values=c)),
    ("dense", lambda c: gen.dense(24, 13, complex_values=c, max_sn=8)),
    ("random_sparse", lambda c: gen.random_struct_sym(80, 0.04, 14, complex_values=c)),
    ("random_denser", lambda c: gen.random_struct_sym(60, 0.15, 15, complex_values=c)),
    ("conv_diff_2d", lambda c: gen.conv_diff_2d(9, 16, imag_diag=0.1 if c else 0.0, max_sn=16)),
    ("upwind_3d", lambda c: gen.upwind_3d(5, 17, max_sn=16)),
    ("stencil27", lambda c: gen.stencil27_complex(4, 18, max_sn=16)),
    ("dg_blocks", lambda c: gen.dg_blocks(2, 6, 19, max_sn=12)),
]


# ---------------------------------------------------------------------------
# double-double dense inverse
# ---------------------------------------------------------------------------
def test_dd_inverse_tridiagonal_closed_form():
    """(tridiag(-1, 2, -1))^{-1}_{ij} = min(i,j) (n+1-max(i,j)) / (n+1), 1-based."""
    n = 13
    a = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    hi, lo = oracle.dense_inverse_dd(a)
    for i in range(n):
        for j in range(n):
            exact = Fraction(min(i + 1, j + 1) * (n + 1 - max(i + 1, j + 1)), n + 1)
            got = Fraction(hi[i, j]) + Fraction(lo[i, j])
            assert abs(got - exact) <= Fraction(1, 10**28)


def test_dd_inverse_against_lapack():
    rng = np.random.default_rng(3)
    a = rng.uniform(-1, 1, (60, 60)) + 30 * np.eye(60)
    hi, lo = oracle.dense_inverse_dd(a)
    assert normwise_error(hi + lo, np.linalg.inv(a)) < 1e-14
    # the residual of the double-double result is far below double rounding
    res = a @ hi - np.eye(60) + a @ lo
    assert np.abs(res).max() < 1e-14


def test_dd_inverse_complex_embedding():
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, 1, (25, 25)) + 1j * rng.uniform(-1, 1, (25, 25)) + 15 * np.eye(25)
    inv = oracle.dense_inverse_dd_complex(a)
    assert normwise_error(inv, np.linalg.inv(a)) < 1e-14


def test_dd_inverse_singular():
    a = np.ones((4, 4))
    with pytest.raises(oracle.OracleError):
        oracle.dense_inverse_dd(a)


# ---------------------------------------------------------------------------
# symbolic analysis
# ---------------------------------------------------------------------------
def test_analyze_tridiagonal_closed_form():
    n = 12
    s = oracle.analyze(gen.tridiagonal(n, 1), relax_pct=0)
    assert np.array_equal(s.parent, np.r_[np.arange(1, n), -1])
    assert np.array_equal(np.diff(s.sptr), np.r_[np.ones(n - 1, dtype=np.int64), 0])
    # strict rule: only the last two columns form a supernode of width 2
    assert np.array_equal(s.supptr, np.r_[np.arange(n - 1), n])
    assert np.array_equal(s.sup_depth, np.arange(n - 1)[::-1])


def test_analyze_dense_closed_form():
    n, w = 10, 4
    s = oracle.analyze(gen.dense(n, 1, max_sn=w), relax_pct=0)
    assert np.array_equal(s.parent, np.r_[np.arange(1, n), -1])
    assert np.array_equal(np.diff(s.sptr), np.arange(n)[::-1])
    assert np.array_equal(s.supptr, [0, 4, 8, 10])
    assert np.array_equal(s.sup_parent, [1, 2, -1])


def test_analyze_diagonal_and_arrow():
    n = 7
    idx = np.arange(n, dtype=np.int64)
    diag = gen.Problem("diag", n, np.arange(n + 1, dtype=np.int64), idx, np.ones(n), idx, 4)
    s = oracle.analyze(diag, relax_pct=50)
    assert np.all(s.parent == -1) and s.nsup == n and np.all(s.sup_depth == 0)
    s = oracle.analyze(gen.arrow(n, 2), relax_pct=0)
    assert np.array_equal(s.parent, np.r_[np.full(n - 1, n - 1), -1])
    assert np.array_equal(s.supptr, np.r_[np.arange(n - 1), n])


@pytest.mark.parametrize("seed", range(6))
def test_analyze_against_brute_force(seed):
    p = gen.random_struct_sym(45, 0.06 + 0.02 * seed, 100 + seed)
    s = oracle.analyze(p, relax_pct=0)
    structs, parent = brute_symbolic(p)
    assert np.array_equal(s.parent, parent)
    for j in range(p.n):
        assert np.array_equal(s.sidx[s.sptr[j]:s.sptr[j + 1]], structs[j])


def _paper_rule_supernodes(structs, parent, max_sn):
    """The paper's strict definition: j+1 joins j iff parent(j) = j+1 and
    struct(j) = {j+1} U struct(j+1), cut every max_sn columns."""
    n = len(structs)
    first = [0]
    for j in range(n - 1):
        same = parent[j] == j + 1 and np.array_equal(structs[j], np.r_[j + 1, structs[j + 1]])
        if not (same and (j + 1 - first[-1]) < max_sn):
            first.append(j + 1)
    return np.array(first + [n])


@pytest.mark.parametrize("maker", [
    lambda: gen.conv_diff_2d(12, 5, max_sn=16),
    lambda: gen.upwind_3d(6, 6, max_sn=32),
    lambda: gen.random_struct_sym(70, 0.05, 7, max_sn=5),
    lambda: gen.dense(20, 8, max_sn=6),
])
def test_strict_supernodes_follow_paper_definition(maker):
    p = maker()
    s = oracle.analyze(p, relax_pct=0)
    structs, parent = brute_symbolic(p)
    assert np.array_equal(s.supptr, _paper_rule_supernodes(structs, parent, p.max_supernode))


@pytest.mark.parametrize("relax", [10, 20, 60])
def test_relaxed_supernode_invariants(relax):
    p = gen.upwind_3d(7, 9, max_sn=40)
    exact = oracle.analyze(p, relax_pct=0)
    s = oracle.analyze(p, relax_pct=relax)
    cnt = np.diff(exact.sptr)
    assert np.array_equal(s.parent, exact.parent)
    for k in range(s.nsup):
        f, l = int(s.supptr[k]), int(s.supptr[k + 1]) - 1
        assert l - f + 1 <= p.max_supernode
        # every column's parent lies inside the block (except the last column)
        assert all(f <= exact.parent[i] <= l for i in range(f, l))
        R = exact.sidx[exact.sptr[l]:exact.sptr[l + 1]]
        total = sum((l - i) + R.size for i in range(f, l + 1))
        zeros = total - cnt[f:l + 1].sum()
        assert 100 * zeros <= relax * total
        # the relaxed per-column structure is (i, l] U R
        for i in range(f, l + 1):
            assert np.array_equal(s.sidx[s.sptr[i]:s.sptr[i + 1]], np.r_[np.arange(i + 1, l + 1), R])
        # greedy maximality: the next column could not have joined
        if l + 1 < p.n:
            l2 = l + 1
            ok = (l2 - f + 1) <= p.max_supernode and all(
                f <= exact.parent[i] <= l2 for i in range(f, l2))
            if ok:
                R2 = cnt[l2]
                total2 = sum((l2 - i) + R2 for i in range(f, l2 + 1))
                zeros2 = total2 - cnt[f:l2 + 1].sum()
                ok = 100 * zeros2 <= relax * total2
            assert not ok
    # supernodal tree: parent of K holds the parent of K's last column
    for k in range(s.nsup):
        l = int(s.supptr[k + 1]) - 1
        pk = s.sup_parent[k]
        if exact.parent[l] < 0:
            assert pk == -1 and s.sup_depth[k] == 0
        else:
            assert s.supptr[pk] <= exact.parent[l] < s.supptr[pk + 1]
            assert s.sup_depth[k] == s.sup_depth[pk] + 1


def test_fig1_golden_structure():
    fields = {}
    with open(os.path.join(HERE, "golden", "fig1_pattern.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(":", 1)
            fields[k.strip()] = v.split()
    n = int(fields["n"][0])
    entries = {(i, i) for i in range(n)}
    for r in fields["L_col0_rows"]:
        entries |= {(int(r), 0), (0, int(r))}
    for c in fields["U_row0_cols"]:
        entries |= {(0, int(c)), (int(c), 0)}
    rows = np.array([e[0] for e in sorted(entries, key=lambda e: (e[1], e[0]))])
    cols = np.array([e[1] for e in sorted(entries, key=lambda e: (e[1], e[0]))])
    colptr = np.r_[0, np.cumsum(np.bincount(cols, minlength=n))]
    p = gen.Problem("fig1", n, colptr, rows, np.ones(rows.size), np.arange(n), 1)
    s = oracle.analyze(p, relax_pct=0)
    for j in (0, 2, 3):
        want = [int(x) for x in fields[f"sym_struct_col{j}"]]
        assert list(s.sidx[s.sptr[j]:s.sptr[j + 1]]) == want
    # the fills and the A^{-1} entries read at step 0 lie on the pattern of L+U
    onpat = set(zip(*s.lu_pattern()))
    for key in ("fill_rows_cols", "ainv_read"):
        for e in fields[key]:
            i, j = (int(t) for t in e.split(","))
            assert (i, j) in onpat


def test_non_symmetric_pattern_rejected():
    n = 3
    colptr = np.array([0, 2, 3, 4])
    rowind = np.array([0, 1, 1, 2])  # A_10 != 0 but A_01 == 0
    p = gen.Problem("ns", n, colptr, rowind, np.ones(4), np.arange(n), 2)
    with pytest.raises(oracle.OracleError) as e:
        oracle.analyze(p)
    assert e.value.code == -2


# ---------------------------------------------------------------------------
# LU
# ---------------------------------------------------------------------------
def dense_factors(fac):
    s = fac.sym
    n = s.n
    L = np.eye(n, dtype=fac.low.dtype)
    U = np.diag(fac.diag)
    cols = csc_cols(s.sptr)
    L[s.sidx, cols] = fac.low
    U[cols, s.sidx] = fac.up
    return L, U


@pytest.mark.parametrize("name,maker", SMALL)
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("relax", [0, 30])
def test_lu_reconstructs_permuted_matrix(name, maker, cplx, relax):
    p = maker(cplx)
    s = oracle.analyze(p, relax_pct=relax)
    fac = oracle.lu(s, p.colptr, p.rowind, p.values)
    L, U = dense_factors(fac)
    a = p.dense()[np.ix_(p.perm, p.perm)]
    assert np.abs(L @ U - a).max() <= 1e-14 * np.abs(a).max()
    assert np.allclose(np.triu(L, 1), 0) and np.allclose(np.tril(U, -1), 0)


def test_lu_2x2_closed_form():
    """Section 2: L_21 = A_21 / U_11, U_12 = A_12, S_22 = A_22 - L_21 U_12."""
    a11, a12, a21, a22 = 3.0, -1.25, 0.5, 2.0
    p = gen.Problem("2x2", 2, np.array([0, 2, 4]), np.array([0, 1, 0, 1]),
                    np.array([a11, a21, a12, a22]), np.array([0, 1]), 2)
    s = oracle.analyze(p, relax_pct=0)
    fac = oracle.lu(s, p.colptr, p.rowind, p.values)
    assert fac.low[0] == a21 / a11 and fac.up[0] == a12
    assert fac.diag[0] == a11 and fac.diag[1] == a22 - (a21 / a11) * a12
    sel = oracle.selinv(fac)
    S = a22 - (a21 / a11) * a12
    # Eq. Ainv2by2 with scalars
    assert np.isclose(sel.diag[1], 1 / S, rtol=1e-15)
    assert np.isclose(sel.low[0], -(1 / S) * (a21 / a11), rtol=1e-15)
    assert np.isclose(sel.up[0], -(1 / a11) * a12 * (1 / S), rtol=1e-15)
    assert np.isclose(sel.diag[0], 1 / a11 + (1 / a11) * a12 * (1 / S) * (a21 / a11), rtol=1e-15)


def test_lu_zero_pivot_reported():
    p = gen.tridiagonal(6, 3)
    v = p.values.copy()
    v[0] = 0.0  # A_00
    s = oracle.analyze(p, relax_pct=0)
    with pytest.raises(oracle.OracleError) as e:
        oracle.lu(s, p.colptr, p.rowind, v)
    assert e.value.code == -3 and "column 0" in str(e.value)


# ---------------------------------------------------------------------------
# selected inversion
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,maker", SMALL)
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("relax", [0, 20, 100])
def test_selinv_matches_dd_dense_inverse(name, maker, cplx, relax):
    p = maker(cplx)
    sel = oracle.selected_inverse(p, relax_pct=relax)
    err, nerr = sel_vs_dense(sel, dense_inverse_ref(p))
    assert err < 1e-13 and nerr < 1e-13, (err, nerr)


def test_selinv_block_2x2_formula():
    """Eq. Ainv2by2 with a block split after the first supernode."""
    p = gen.upwind_3d(4, 21, max_sn=8)
    s = oracle.analyze(p, relax_pct=0)
    sel = oracle.selinv(oracle.lu(s, p.colptr, p.rowind, p.values))
    a = p.dense()[np.ix_(p.perm, p.perm)]
    m = int(s.supptr[1])
    A11, A12, A21, A22 = a[:m, :m], a[:m, m:], a[m:, :m], a[m:, m:]
    # block LU with L11 unit lower, U11 upper (A11 = L11 U11)
    L11 = np.eye(m)
    U11 = A11.copy()
    for k in range(m):
        L11[k + 1:, k] = U11[k + 1:, k] / U11[k, k]
        U11[k + 1:, :] -= np.outer(L11[k + 1:, k], U11[k, :])
    U11 = np.triu(U11)
    L21 = A21 @ np.linalg.inv(U11)
    U12 = np.linalg.inv(L11) @ A12
    S = A22 - L21 @ U12
    Sinv = np.linalg.inv(S)
    iU, iL = np.linalg.inv(U11), np.linalg.inv(L11)
    blk = np.block([[iU @ iL + iU @ U12 @ Sinv @ L21 @ iL, -iU @ U12 @ Sinv],
                    [-Sinv @ L21 @ iL, Sinv]])
    rows, cols, vals = sel_coo(sel)
    assert normwise_error(vals, blk[rows, cols]) < 1e-13


@pytest.mark.parametrize("maker", [
    lambda: gen.make_config(1),
    lambda: gen.upwind_3d(9, 22, max_sn=64),
    lambda: gen.stencil27_complex(5, 23, max_sn=64),
])
def test_selinv_row_and_column_identities(maker):
    """sum_j A_ij (A^{-1})_ji = 1 and sum_j (A^{-1})_ij A_ji = 1 for every i,
    using only selected entries (generalises Tr[A A^{-1}] = N, Section 1)."""
    p = maker()
    sel = oracle.selected_inverse(p)
    B = oracle.extract(sel, p.colptr, p.rowind)          # B[p] = (A^{-1})_{row, col}
    cols = csc_cols(p.colptr)
    # position of the transposed entry (col, row) in CSC order
    key = cols * p.n + p.rowind
    tkey = p.rowind * p.n + cols
    order = np.argsort(key)
    tpos = order[np.searchsorted(key[order], tkey)]
    Bt = B[tpos]                                          # (A^{-1})_{col, row}
    rowsum = np.zeros(p.n, dtype=B.dtype)
    np.add.at(rowsum, p.rowind, p.values * Bt)            # sum_j A_ij B_ji
    colsum = np.zeros(p.n, dtype=B.dtype)
    np.add.at(colsum, cols, B * p.values[tpos])           # sum_i B_ji A_ij
    scale = np.zeros(p.n)
    np.add.at(scale, p.rowind, np.abs(p.values) * np.abs(Bt))
    assert np.all(np.abs(rowsum - 1) <= 1e-12 * np.maximum(scale, 1))
    assert np.all(np.abs(colsum - 1) <= 1e-12 * np.maximum(scale, 1))
    assert abs(rowsum.sum() - p.n) < 1e-9 * p.n


def test_selinv_transpose():
    """selinv(A^T) = selinv(A)^T on the pattern."""
    p = gen.upwind_3d(6, 24, max_sn=32)
    a = p.dense()
    cols = csc_cols(p.colptr)
    pt = gen.Problem("t", p.n, p.colptr, p.rowind, a.T[p.rowind, cols], p.perm, p.max_supernode)
    B = oracle.extract(oracle.selected_inverse(p), p.colptr, p.rowind)
    Bt = oracle.extract(oracle.selected_inverse(pt), p.colptr, p.rowind)
    ref = np.zeros_like(a)
    ref[p.rowind, cols] = B
    assert normwise_error(Bt, ref.T[p.rowind, cols]) < 1e-13


def test_selinv_symmetric_input_gives_symmetric_result():
    p = gen.random_struct_sym(70, 0.08, 25, symmetric_values=True, max_sn=8)
    a = p.dense()
    assert np.array_equal(a, a.T)
    B = oracle.extract(oracle.selected_inverse(p), p.colptr, p.rowind)
    cols = csc_cols(p.colptr)
    m = np.zeros_like(a)
    m[p.rowind, cols] = B
    assert np.abs(m - m.T).max() < 1e-14 * np.abs(m).max()


def test_selinv_permutation_invariance():
    """Theorem 2: the result in the original ordering does not depend on P."""
    p = gen.conv_diff_2d(10, 26, max_sn=16)
    q = gen.Problem("rp", p.n, p.colptr, p.rowind, p.values,
                    np.random.default_rng(0).permutation(p.n), 16)
    B1 = oracle.extract(oracle.selected_inverse(p), p.colptr, p.rowind)
    B2 = oracle.extract(oracle.selected_inverse(q), p.colptr, p.rowind)
    assert normwise_error(B2, B1) < 1e-13


def test_selinv_alternative_diagonal_formula():
    """Section 2: B_KK also equals (U_KK L_KK)^{-1} - B_{K,C} Lhat_{C,K}
    (the formula noted beside Algorithm 1 step 4); column form with L_kk = 1:
    B_kk = 1/U_kk - sum_{j in C} B_kj L_jk."""
    p = gen.stencil27_complex(4, 27, max_sn=16)
    s = oracle.analyze(p)
    fac = oracle.lu(s, p.colptr, p.rowind, p.values)
    sel = oracle.selinv(fac)
    for k in range(p.n):
        b, e = s.sptr[k], s.sptr[k + 1]
        alt = 1 / fac.diag[k] - np.sum(sel.up[b:e] * fac.low[b:e])
        assert abs(alt - sel.diag[k]) <= 1e-13 * max(1.0, abs(sel.diag[k]))


def test_selinv_tridiagonal_toeplitz_closed_form():
    n = 20
    i = np.arange(n - 1)
    colptr = np.r_[0, 1 + np.minimum(np.arange(n), 1) + np.minimum(n - 1 - np.arange(n), 1)]
    colptr = np.cumsum(np.r_[0, np.diff(colptr)])
    rows, vals = [], []
    for j in range(n):
        for r in (j - 1, j, j + 1):
            if 0 <= r < n:
                rows.append(r)
                vals.append(2.0 if r == j else -1.0)
    colptr = np.r_[0, np.cumsum([min(j + 2, n) - max(j - 1, 0) for j in range(n)])]
    p = gen.Problem("toeplitz", n, colptr, np.array(rows), np.array(vals), np.arange(n), 4)
    B = oracle.extract(oracle.selected_inverse(p, relax_pct=0), p.colptr, p.rowind)
    cols = csc_cols(p.colptr)
    exact = np.array([min(r + 1, c + 1) * (n + 1 - max(r + 1, c + 1)) / (n + 1)
                      for r, c in zip(p.rowind, cols)])
    assert np.abs(B - exact).max() < 1e-13 * exact.max()
    del i


# ---------------------------------------------------------------------------
# planted mistakes: every mutation must fail at least one pin
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mutation", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistakes(mutation):
    p = gen.upwind_3d(5, 28, max_sn=16)
    sel = oracle.selected_inverse(p, mutation=mutation)
    err, _ = sel_vs_dense(sel, dense_inverse_ref(p))
    assert err > 1e-6
