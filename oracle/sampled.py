"""Sampled columns and rows of A^{-1} for workloads too large for the scalar
oracle (TEST INFRASTRUCTURE ONLY).

Column j of A^{-1} solves A x = e_j; row i solves A^T y = e_i.  The solves go
through SciPy's sparse LU (SuperLU) as a library primitive, on the original
(unpermuted) matrix, so they share nothing with either the scalar oracle or
the CUDA path.  Every selected entry in a sampled row or column can be
checked against them.
"""
from __future__ import annotations

import numpy as np


class SampledInverse:
    def __init__(self, problem, b: int = 0):
        import scipy.sparse as sp
        from scipy.sparse.linalg import splu
        vals = problem.values if problem.values.ndim == 1 else problem.values[b]
        a = sp.csc_matrix((vals, problem.rowind, problem.colptr), shape=(problem.n, problem.n))
        self.n = problem.n
        self.dtype = vals.dtype
        # factor the symmetrically reordered matrix (the input ordering keeps
        # SuperLU's fill small); partial pivoting stays on
        self._perm = np.asarray(problem.perm, dtype=np.int64)
        ap = a[self._perm][:, self._perm].tocsc()
        self._lu = splu(ap, permc_spec="NATURAL")

    def columns(self, cols):
        """A^{-1}[:, cols] (dense n x len(cols))."""
        cols = np.asarray(cols, dtype=np.int64)
        iperm = np.empty(self.n, dtype=np.int64)
        iperm[self._perm] = np.arange(self.n)
        # (P A P^T)^{-1} = P A^{-1} P^T: column iperm[j] of it, rows back to original
        e = np.zeros((self.n, cols.size), dtype=self.dtype)
        e[iperm[cols], np.arange(cols.size)] = 1
        x = self._lu.solve(e)
        return x[iperm]

    def rows(self, rows):
        """A^{-1}[rows, :] returned transposed (n x len(rows))."""
        rows = np.asarray(rows, dtype=np.int64)
        iperm = np.empty(self.n, dtype=np.int64)
        iperm[self._perm] = np.arange(self.n)
        e = np.zeros((self.n, rows.size), dtype=self.dtype)
        e[iperm[rows], np.arange(rows.size)] = 1
        y = self._lu.solve(e, trans="T")
        return y[iperm]
