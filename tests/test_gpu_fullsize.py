"""Full-size runs of the larger workloads: the 60^3 complex 27-point operator,
the pole-expansion batch (40 complex shifts of a 32^3 operator and 64 uneven
2D grids in one sweep) and the 16^3 x 64 DG operator (3.2e9 stored entries,
beyond 32-bit offsets).  The scalar oracle cannot finish them, so they are
checked by properties that hold at any size:

* row and column identities: sum_j A_ij (A^{-1})_ji = 1 and
  sum_j (A^{-1})_ij A_ji = 1 for every i, using only entries on pattern(A)
  (a generalisation of Tr[A A^{-1}] = N to every row and column);
* a few columns of A^{-1} from GMRES solves with SciPy (independent of the
  CUDA path) where the operator is well enough conditioned;
* the split-precision sweep against the FP64 sweep of the same handle.
"""
from __future__ import annotations

import numpy as np
import pytest

import gen
from helpers import csc_cols

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_04539_gb300 import build
    build.build()
    return _t


def transpose_positions(p):
    """For entry q = (i, j) of A's CSC pattern, the position of (j, i)."""
    c = csc_cols(p.colptr)
    key = c * p.n + p.rowind
    order = np.argsort(key)
    return order[np.searchsorted(key[order], p.rowind * p.n + c)]


def _sums(idx, w, n):
    if np.iscomplexobj(w):
        return np.bincount(idx, w.real, n) + 1j * np.bincount(idx, w.imag, n)
    return np.bincount(idx, w, n)


def identity_errors(p, vals, B, tpos):
    """max_i |sum_j A_ij B_ji - 1| and the same over columns, each relative to
    sum_j |A_ij B_ji| (B on pattern(A), CSC order like A)."""
    c = csc_cols(p.colptr)
    prod = vals * B[tpos]                  # A_ij B_ji at entry (i, j)
    row = _sums(p.rowind, prod, p.n)
    rowabs = np.bincount(p.rowind, np.abs(prod), p.n)
    prod2 = B * vals[tpos]                 # B_ij A_ji at entry (i, j)
    col = _sums(c, prod2, p.n)
    colabs = np.bincount(c, np.abs(prod2), p.n)
    return (np.abs(row - 1) / rowabs).max(), (np.abs(col - 1) / colabs).max()


def run_both(torch, h, values, nbatch=1):
    """FP64 and split sweeps of one handle; pattern-of-A outputs per instance."""
    import paper_1708_04539_gb300 as ps
    h.factor(torch.from_numpy(np.ascontiguousarray(values)).cuda())
    out = {}
    for prec in (ps.PREC_FP64, ps.PREC_OZAKI_FP16):
        h.selinv(precision=prec)
        out[prec] = [h.get_selected(batch=b) for b in range(nbatch)]
    h.sync()
    h.close()
    return out[ps.PREC_FP64], out[ps.PREC_OZAKI_FP16]


def run_problem(torch, p):
    import paper_1708_04539_gb300 as ps
    return run_both(torch, ps.SelInv.from_problem(p), p.values, p.nbatch)


def check_instance(p, b, B64, Bsp, tpos, tol64=1e-11, tolsp=1e-9):
    vals = p.values if p.values.ndim == 1 else p.values[b]
    r64, c64 = identity_errors(p, vals, B64, tpos)
    assert r64 < tol64 and c64 < tol64, (b, r64, c64)
    rsp, csp = identity_errors(p, vals, Bsp, tpos)
    assert rsp < tolsp and csp < tolsp, (b, rsp, csp)
    assert np.abs(Bsp - B64).max() <= tolsp * np.abs(B64).max()


def test_config3_complex27_full_size(torch):
    import scipy.sparse as sp
    from scipy.sparse.linalg import gmres, LinearOperator
    p = gen.make_config(3)
    B64, Bsp = run_problem(torch, p)
    tpos = transpose_positions(p)
    check_instance(p, 0, B64[0], Bsp[0], tpos)
    # columns of A^{-1} by Jacobi-preconditioned GMRES (diagonally dominant)
    A = sp.csc_matrix((p.values, p.rowind, p.colptr), shape=(p.n, p.n))
    dinv = 1.0 / A.diagonal()
    M = LinearOperator(A.shape, matvec=lambda x: dinv * x, dtype=A.dtype)
    rng = np.random.default_rng(11)
    for j in rng.choice(p.n, 3, replace=False):
        e = np.zeros(p.n, dtype=A.dtype)
        e[j] = 1
        try:
            x, info = gmres(A, e, M=M, rtol=1e-12, atol=0.0, restart=200, maxiter=50)
        except TypeError:  # SciPy before 1.12 names it tol
            x, info = gmres(A, e, M=M, tol=1e-12, atol=0.0, restart=200, maxiter=50)
        assert info == 0
        lo, hi = p.colptr[j], p.colptr[j + 1]
        got = B64[0][lo:hi]                     # (A^{-1})_{i j} for i in pattern column j
        ref = x[p.rowind[lo:hi]]
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(x).max()


def test_config4_pole_batch_full_size(torch):
    import paper_1708_04539_gb300 as ps
    fam, *grids = gen.make_config(4)
    B64, Bsp = run_problem(torch, fam)
    tpos = transpose_positions(fam)
    for b in range(fam.nbatch):
        check_instance(fam, b, B64[b], Bsp[b], tpos)
    group = ps.InstanceGroup([(q.n, q.colptr, q.rowind, q.perm) for q in grids])
    G64, Gsp = run_both(torch, group.handle, group.values([q.values for q in grids]))
    parts64, partssp = group.split(G64[0]), group.split(Gsp[0])
    for q, part64, partsp in zip(grids, parts64, partssp):
        check_instance(q, 0, part64, partsp, transpose_positions(q))


def test_config5_dg_full_size(torch):
    """3.2e9 stored entries per array: offsets beyond 32 bits on every path."""
    p = gen.make_config(5)
    B64, Bsp = run_problem(torch, p)
    tpos = transpose_positions(p)
    check_instance(p, 0, B64[0], Bsp[0], tpos)
