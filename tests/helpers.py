"""Shared test helpers: error metrics and pattern bookkeeping (no method arithmetic)."""
from __future__ import annotations

import numpy as np


def selected_error(x, r, rows, cols, n=None):
    """Error of ``x`` against reference ``r`` on a set of selected entries.

    For each selected (i, j): |x_ij - r_ij| / rho_ij with
    rho_ij = max(max_k |r_ik|, max_k |r_kj|) over the selected entries of row i
    and column j (an elementwise relative error is not attainable for the
    tiny, decaying off-diagonal entries of an inverse).  Complex: modulus.
    Returns the maximum over all entries.
    """
    x = np.asarray(x)
    r = np.asarray(r)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if r.size == 0:
        return 0.0
    if n is None:
        n = int(max(rows.max(), cols.max())) + 1
    a = np.abs(r)
    rowmax = np.zeros(n)
    colmax = np.zeros(n)
    np.maximum.at(rowmax, rows, a)
    np.maximum.at(colmax, cols, a)
    rho = np.maximum(rowmax[rows], colmax[cols])
    rho = np.where(rho > 0, rho, 1.0)
    return float(np.max(np.abs(x - r) / rho))


def normwise_error(x, r):
    r = np.asarray(r)
    m = np.max(np.abs(r)) if r.size else 1.0
    return float(np.max(np.abs(np.asarray(x) - r)) / (m if m > 0 else 1.0)) if r.size else 0.0


def csc_cols(colptr):
    return np.repeat(np.arange(len(colptr) - 1, dtype=np.int64), np.diff(colptr))


def dense_inverse_ref(problem, b=0):
    """Double-double inverse of a small problem (oracle routine), as complex or real."""
    import oracle
    a = problem.dense(b)
    if np.iscomplexobj(a):
        return oracle.dense_inverse_dd_complex(a)
    hi, lo = oracle.dense_inverse_dd(a)
    return hi + lo
