"""Synthetic matrix families and the geometric nested-dissection ordering.

Every generator is deterministic in its ``seed``.  Random quantities use
``numpy.random.default_rng([seed, stream])`` with one stream per quantity, so
changing one quantity's recipe never shifts another's numbers.

Conventions
-----------
* CSC, 0-based, ``int64`` indices, row indices sorted within each column, the
  diagonal always present (structurally symmetric patterns only).
* ``values`` is ``[nnz]`` for one instance or ``[nbatch, nnz]`` for several
  instances that share the pattern (the complex shifts of a pole expansion).
* ``perm`` is the new -> old map of the symmetric ordering (P = Q^T):
  row/column ``perm[k]`` of A becomes row/column ``k`` of the permuted matrix.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1708045390

CONFIG_NAMES = {
    1: "2D 5-point convection-diffusion 31x31 (n=961), FP64, max supernode 64",
    2: "3D 7-point upwind convection-diffusion 40^3 (n=64000), FP64, max supernode 256",
    3: "3D 27-point non-symmetric complex stencil 60^3 (n=216000), complex128, max supernode 256",
    4: "pole-expansion batch: 40 shifts of a 32^3 7-point pattern + 64 uneven 2D grids, complex128",
    5: "DG-like block operator 16^3 elements x 64 basis functions (n=262144), FP64, max supernode 256",
}


@dataclass
class Problem:
    name: str
    n: int
    colptr: np.ndarray
    rowind: np.ndarray
    values: np.ndarray
    perm: np.ndarray
    max_supernode: int
    dims: tuple = ()
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    @property
    def nbatch(self) -> int:
        return 1 if self.values.ndim == 1 else int(self.values.shape[0])

    @property
    def is_complex(self) -> bool:
        return np.iscomplexobj(self.values)

    def dense(self, b: int = 0) -> np.ndarray:
        """Dense copy of instance ``b`` (original ordering); small n only."""
        v = self.values if self.values.ndim == 1 else self.values[b]
        a = np.zeros((self.n, self.n), dtype=v.dtype)
        cols = np.repeat(np.arange(self.n), np.diff(self.colptr))
        a[self.rowind, cols] = v
        return a


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# ---------------------------------------------------------------------------
# ordering
# ---------------------------------------------------------------------------
def nd_perm(dims, max_sn: int, dof: int = 1) -> np.ndarray:
    """Geometric nested dissection of a box grid (new -> old map).

    Stand-in for the ParMETIS ordering used in the paper's experiments.
    A box is split along its longest axis (ties: lowest axis index) at
    ``mid = lo + len // 2``; the one-plane separator at ``mid`` is ordered
    after both halves (left half, right half, separator).  Recursion stops
    when a box holds at most ``max_sn`` unknowns or every extent is <= 2;
    a leaf box and a separator plane are emitted in lexicographic order with
    x fastest.  With ``dof > 1`` every grid node carries ``dof`` consecutive
    unknowns (element-wise ordering of a DG operator).
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    strides = [1] * nd
    for d in range(1, nd):
        strides[d] = strides[d - 1] * dims[d - 1]
    out = []

    def emit(lo, hi):
        axes = [np.arange(lo[d], hi[d], dtype=np.int64) for d in range(nd)]
        # lexicographic with x fastest: iterate the last axis slowest
        grids = np.meshgrid(*axes[::-1], indexing="ij")
        idx = np.zeros(grids[0].shape, dtype=np.int64)
        for k, g in enumerate(grids):
            d = nd - 1 - k
            idx += g * strides[d]
        idx = idx.reshape(-1)
        if dof > 1:
            idx = (idx[:, None] * dof + np.arange(dof, dtype=np.int64)[None, :]).reshape(-1)
        out.append(idx)

    def rec(lo, hi):
        ext = [hi[d] - lo[d] for d in range(nd)]
        if min(ext) <= 0:
            return
        if math.prod(ext) * dof <= max_sn or max(ext) <= 2:
            emit(lo, hi)
            return
        d = int(np.argmax(ext))  # first maximum = lowest axis index on ties
        mid = lo[d] + ext[d] // 2
        lhi = list(hi); lhi[d] = mid
        rlo = list(lo); rlo[d] = mid + 1
        slo = list(lo); slo[d] = mid
        shi = list(hi); shi[d] = mid + 1
        rec(list(lo), lhi)
        rec(rlo, list(hi))
        emit(slo, shi)

    rec([0] * nd, list(dims))
    perm = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    n = math.prod(dims) * dof
    assert perm.size == n and np.array_equal(np.sort(perm), np.arange(n))
    return perm


# ---------------------------------------------------------------------------
# assembly helpers
# ---------------------------------------------------------------------------
def _coords(dims):
    n = math.prod(dims)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx
    for d in dims:
        coords.append(rem % d)
        rem = rem // d
    return idx, coords


def _neighbour(dims, coords, offset):
    """(mask, j) with j the index of node + offset where it stays inside."""
    mask = np.ones(coords[0].shape, dtype=bool)
    j = np.zeros(coords[0].shape, dtype=np.int64)
    stride = 1
    for d, (m, o) in enumerate(zip(dims, offset)):
        c = coords[d] + o
        mask &= (c >= 0) & (c < m)
        j += np.clip(c, 0, m - 1) * stride
        stride *= m
    return mask, j


def _to_csc(n, rows, cols, vals):
    """COO (no duplicates) -> sorted CSC.  ``vals`` may be [nnz] or [nb, nnz]."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    order = np.lexsort((rows, cols))
    rows = rows[order]
    cols = cols[order]
    key = cols * n + rows
    if key.size > 1 and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate entries in COO input")
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(cols, minlength=n), out=colptr[1:])
    vals = np.asarray(vals)
    vals = vals[..., order]
    return colptr, rows, np.ascontiguousarray(vals)


# ---------------------------------------------------------------------------
# families
# ---------------------------------------------------------------------------
def conv_diff_2d(m: int, seed: int, sigma: float = 0.1, imag_diag: float = 0.0,
                 max_sn: int = 64, name: str | None = None) -> Problem:
    """2D 5-point convection-diffusion on an m x m grid.

    For node i and axis d, beta_{i,d} ~ U(0, 0.5); a_{i,i+e_d} = -1 + beta,
    a_{i,i-e_d} = -1 - beta (Dirichlet: neighbours outside are dropped);
    a_ii = 4 + sigma (+ i * imag_diag).  Strictly diagonally dominant by
    rows and non-symmetric.
    """
    dims = (m, m)
    idx, coords = _coords(dims)
    n = idx.size
    beta = _rng(seed, 1).uniform(0.0, 0.5, size=(n, 2))
    rows, cols, vals = [idx], [idx], [np.full(n, 4.0 + sigma)]
    for d in range(2):
        for sgn in (+1, -1):
            off = [0, 0]
            off[d] = sgn
            mask, j = _neighbour(dims, coords, off)
            rows.append(idx[mask])
            cols.append(j[mask])
            vals.append(-1.0 + sgn * beta[mask, d])
    v = np.concatenate(vals)
    if imag_diag:
        v = v.astype(np.complex128)
        v[:n] += 1j * imag_diag
    colptr, rowind, v = _to_csc(n, np.concatenate(rows), np.concatenate(cols), v)
    return Problem(name or f"conv_diff_2d_{m}", n, colptr, rowind, v,
                   nd_perm(dims, max_sn), max_sn, dims)


def _upwind_3d_values(dims, seed, shift):
    idx, coords = _coords(dims)
    n = idx.size
    v = _rng(seed, 2).uniform(-1.0, 1.0, size=(n, 3))
    diag = 6.0 + np.abs(v).sum(axis=1) + shift
    rows, cols, vals = [idx], [idx], [diag]
    for d in range(3):
        for sgn in (+1, -1):
            off = [0, 0, 0]
            off[d] = sgn
            mask, j = _neighbour(dims, coords, off)
            val = np.full(n, -1.0)
            # upwind convection: v_d > 0 couples to the -e_d neighbour,
            # v_d <= 0 to the +e_d neighbour (the diagonal gets |v_d|).
            if sgn < 0:
                val = val - np.where(v[:, d] > 0, v[:, d], 0.0)
            else:
                val = val + np.where(v[:, d] > 0, 0.0, v[:, d])
            rows.append(idx[mask])
            cols.append(j[mask])
            vals.append(val[mask])
    return n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def upwind_3d(m: int, seed: int, shift: float = 0.1, max_sn: int = 256,
              name: str | None = None) -> Problem:
    """3D 7-point upwind convection-diffusion on an m^3 grid (real).

    Velocity v_i ~ U(-1,1)^3 per node; diffusion -1 to every neighbour;
    upwind convection adds -v_d to a_{i,i-e_d} when v_d > 0, else +v_d to
    a_{i,i+e_d}; a_ii = 6 + sum_d |v_d| + shift.
    """
    dims = (m, m, m)
    n, r, c, v = _upwind_3d_values(dims, seed, shift)
    colptr, rowind, v = _to_csc(n, r, c, v)
    return Problem(name or f"upwind_3d_{m}", n, colptr, rowind, v,
                   nd_perm(dims, max_sn), max_sn, dims)


def sym_diffusion_3d(m: int, seed: int, shift: float = 0.1, max_sn: int = 256,
                     name: str | None = None) -> Problem:
    """3D 7-point diffusion with symmetric random coefficients (real, A = A^T).

    Each grid edge (i, i + e_d) gets a_{i,i+e_d} = a_{i+e_d,i} = -(1 + u), u ~ U(0,1)
    drawn per edge; a_ii = sum of |off-diagonals| + shift.
    """
    dims = (m, m, m)
    idx, coords = _coords(dims)
    n = idx.size
    rng = _rng(seed, 3)
    rows, cols, vals = [], [], []
    offsum = np.zeros(n)
    for d in range(3):
        off = [0, 0, 0]
        off[d] = 1
        mask, j = _neighbour(dims, coords, off)
        i = idx[mask]
        jj = j[mask]
        w = -(1.0 + rng.uniform(0.0, 1.0, size=i.size))
        rows += [i, jj]
        cols += [jj, i]
        vals += [w, w]
        np.add.at(offsum, i, np.abs(w))
        np.add.at(offsum, jj, np.abs(w))
    rows.append(idx)
    cols.append(idx)
    vals.append(offsum + shift)
    colptr, rowind, v = _to_csc(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    return Problem(name or f"sym_diffusion_3d_{m}", n, colptr, rowind, v,
                   nd_perm(dims, max_sn), max_sn, dims)


def stencil27_complex(m: int, seed: int, z: complex = 0.5 + 0.1j, eps: float = 0.2,
                      max_sn: int = 256, name: str | None = None) -> Problem:
    """3D 27-point complex operator A = H - z S + eps N on an m^3 grid.

    H real symmetric with U(-1,1) off-diagonals, S diagonal ~ U(1,2), N real
    non-symmetric U(-1,1) on the same pattern with N_ii = 0, and
    H_ii = sum_j (|H_ij| + eps |N_ij|) + 1 + Re(z) S_ii.
    """
    dims = (m, m, m)
    idx, coords = _coords(dims)
    n = idx.size
    offs = [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)
            if (a, b, c) != (0, 0, 0)]
    half = [o for o in offs if o > (0, 0, 0)]
    rng_h, rng_n = _rng(seed, 3), _rng(seed, 4)
    S = _rng(seed, 5).uniform(1.0, 2.0, size=n)
    rows, cols, hv, nv = [], [], [], []
    for o in half:
        mask, j = _neighbour(dims, coords, o)
        i = idx[mask]
        j = j[mask]
        h = rng_h.uniform(-1.0, 1.0, size=i.size)
        n1 = rng_n.uniform(-1.0, 1.0, size=i.size)
        n2 = rng_n.uniform(-1.0, 1.0, size=i.size)
        rows += [i, j]
        cols += [j, i]
        hv += [h, h]
        nv += [n1, n2]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    hv = np.concatenate(hv)
    nv = np.concatenate(nv)
    off = hv + eps * nv
    rowsum = np.bincount(rows, weights=np.abs(hv) + eps * np.abs(nv), minlength=n)
    hdiag = rowsum + 1.0 + z.real * S
    diag = hdiag - z * S
    v = np.concatenate([diag, off.astype(np.complex128)])
    colptr, rowind, v = _to_csc(n, np.concatenate([idx, rows]), np.concatenate([idx, cols]), v)
    return Problem(name or f"stencil27_{m}", n, colptr, rowind, v,
                   nd_perm(dims, max_sn), max_sn, dims, meta={"z": z, "eps": eps})


def shifted_family(m: int, seed: int, nshift: int = 40, radius: float = 2.0,
                   centre: complex = 1.0 + 0.0j, base_shift: float = 3.1,
                   max_sn: int = 256, name: str | None = None) -> Problem:
    """One 3D 7-point pattern with ``nshift`` complex shifts A_l = A0 - z_l I.

    A0 is the upwind 3D operator with diagonal shift ``base_shift``; the
    shifts z_l = centre + radius * exp(i theta_l), theta_l = 2 pi (l+1/2)/nshift,
    lie on a contour as in a pole expansion.
    """
    dims = (m, m, m)
    n, r, c, v = _upwind_3d_values(dims, seed, base_shift)
    colptr, rowind, v0 = _to_csc(n, r, c, v)
    theta = 2.0 * np.pi * (np.arange(nshift) + 0.5) / nshift
    zs = centre + radius * np.exp(1j * theta)
    cols = np.repeat(np.arange(n), np.diff(colptr))
    isdiag = rowind == cols
    vals = np.repeat(v0[None, :].astype(np.complex128), nshift, axis=0)
    vals[:, isdiag] -= zs[:, None]
    return Problem(name or f"shifted_{m}x{nshift}", n, colptr, rowind, vals,
                   nd_perm(dims, max_sn), max_sn, dims, meta={"z": zs})


def dg_blocks(me: int, nb: int, seed: int, max_sn: int = 256,
              name: str | None = None) -> Problem:
    """Block-sparse DG-like operator: me^3 elements, nb unknowns per element.

    Element blocks dense nb x nb ~ U(-1,1); face blocks to the 6 neighbours
    dense nb x nb ~ U(-1,1) * (1 + 0.5 w), w = +1 for the downwind neighbour
    and -1 for the upwind one along a per-axis flow direction drawn from the
    seed; a_ii = (row abs-sum of the off-diagonal entries) + 1.
    """
    dims = (me, me, me)
    eidx, coords = _coords(dims)
    ne = eidx.size
    n = ne * nb
    flow = np.where(_rng(seed, 6).uniform(size=3) < 0.5, -1, 1)
    rng_b = _rng(seed, 7)
    bi = np.repeat(np.arange(nb, dtype=np.int64), nb)   # row within block
    bj = np.tile(np.arange(nb, dtype=np.int64), nb)     # column within block
    rows, cols, vals = [], [], []
    blocks = [(0, 0, 0)] + [tuple(s if k == d else 0 for k in range(3))
                            for d in range(3) for s in (1, -1)]
    for o in blocks:
        mask, ej = _neighbour(dims, coords, o)
        ei = eidx[mask]
        ej = ej[mask]
        val = rng_b.uniform(-1.0, 1.0, size=(ei.size, nb * nb))
        if o != (0, 0, 0):
            d = int(np.nonzero(o)[0][0])
            w = 1.0 if o[d] == flow[d] else -1.0
            val *= 1.0 + 0.5 * w
        rows.append((ei[:, None] * nb + bi[None, :]).reshape(-1))
        cols.append((ej[:, None] * nb + bj[None, :]).reshape(-1))
        vals.append(val.reshape(-1))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    isdiag = rows == cols
    vals[isdiag] = 0.0
    rowsum = np.bincount(rows, weights=np.abs(vals), minlength=n)
    vals[isdiag] = rowsum[rows[isdiag]] + 1.0
    colptr, rowind, v = _to_csc(n, rows, cols, vals)
    return Problem(name or f"dg_{me}x{nb}", n, colptr, rowind, v,
                   nd_perm(dims, max_sn, dof=nb), max_sn, dims, meta={"nb": nb, "flow": flow})


# ---------------------------------------------------------------------------
# small test families
# ---------------------------------------------------------------------------
def _finish_small(n, rows, cols, seed, complex_values, name, max_sn, perm=None,
                  symmetric_values=False):
    rng = _rng(seed, 8)
    off = rows != cols
    r, c = rows[off], cols[off]
    vals = rng.uniform(-1.0, 1.0, size=r.size)
    if complex_values:
        vals = vals + 1j * rng.uniform(-1.0, 1.0, size=r.size)
    if symmetric_values:
        # mirror the value of (min, max) onto (max, min)
        key = np.minimum(r, c) * n + np.maximum(r, c)
        uniq, inv = np.unique(key, return_inverse=True)
        base = rng.uniform(-1.0, 1.0, size=uniq.size)
        if complex_values:
            base = base + 1j * rng.uniform(-1.0, 1.0, size=uniq.size)
        vals = base[inv]
    rowsum = np.bincount(r, weights=np.abs(vals), minlength=n)
    diag = rowsum + 1.0 + rng.uniform(0.0, 1.0, size=n)
    if complex_values:
        diag = diag + 1j * rng.uniform(-0.5, 0.5, size=n)
    idx = np.arange(n, dtype=np.int64)
    colptr, rowind, v = _to_csc(n, np.concatenate([idx, r]), np.concatenate([idx, c]),
                                np.concatenate([diag, vals]))
    if perm is None:
        perm = np.arange(n, dtype=np.int64)
    return Problem(name, n, colptr, rowind, v, np.asarray(perm, dtype=np.int64), max_sn, (n,))


def random_struct_sym(n: int, density: float, seed: int, complex_values: bool = False,
                      max_sn: int = 16, symmetric_values: bool = False,
                      permute: bool = True) -> Problem:
    """Random structurally symmetric pattern, diagonally dominant values."""
    rng = _rng(seed, 9)
    m = int(round(density * n * (n - 1) / 2))
    i = rng.integers(0, n, size=4 * m + 8)
    j = rng.integers(0, n, size=4 * m + 8)
    keep = i < j
    key = np.unique(i[keep] * n + j[keep])[:m]
    i, j = key // n, key % n
    rows = np.concatenate([np.arange(n), i, j])
    cols = np.concatenate([np.arange(n), j, i])
    perm = rng.permutation(n) if permute else None
    return _finish_small(n, rows, cols, seed, complex_values,
                         f"random_{n}_{density}", max_sn, perm, symmetric_values)


def tridiagonal(n: int, seed: int, complex_values: bool = False, max_sn: int = 16) -> Problem:
    i = np.arange(n - 1)
    rows = np.concatenate([np.arange(n), i, i + 1])
    cols = np.concatenate([np.arange(n), i + 1, i])
    return _finish_small(n, rows, cols, seed, complex_values, f"tridiag_{n}", max_sn)


def arrow(n: int, seed: int, complex_values: bool = False, max_sn: int = 16) -> Problem:
    """Arrow matrix with the dense row/column last (no fill)."""
    i = np.arange(n - 1)
    rows = np.concatenate([np.arange(n), i, np.full(n - 1, n - 1)])
    cols = np.concatenate([np.arange(n), np.full(n - 1, n - 1), i])
    return _finish_small(n, rows, cols, seed, complex_values, f"arrow_{n}", max_sn)


def dense(n: int, seed: int, complex_values: bool = False, max_sn: int = 16) -> Problem:
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return _finish_small(n, ii.reshape(-1), jj.reshape(-1), seed, complex_values,
                         f"dense_{n}", max_sn)


# ---------------------------------------------------------------------------
# general (not structurally symmetric) patterns with static pivoting
# ---------------------------------------------------------------------------
def _scramble(n, rows, cols, vals, seed, name, max_sn, dims, cperm, row_scramble):
    """A = P^T Atilde Q^T from a pivoted matrix Atilde given in COO (new
    indices): rperm / cperm (new -> old, in meta) recover Atilde = P A Q.
    The rows of A are a random permutation of Atilde's when row_scramble
    (the row permutation a static pivoting would have to find), else they
    follow the columns (P = Q^T)."""
    rng = _rng(seed, 11)
    cperm = np.asarray(cperm, dtype=np.int64)
    rperm = rng.permutation(n).astype(np.int64) if row_scramble else cperm.copy()
    colptr, rowind, v = _to_csc(n, rperm[rows], cperm[cols], vals)
    return Problem(name, n, colptr, rowind, v, cperm, max_sn, dims,
                   meta={"rperm": rperm, "cperm": cperm, "general": True})


def general_random(n: int, density: float, seed: int, complex_values: bool = False,
                   max_sn: int = 16, triangle: str = "", row_scramble: bool = True) -> Problem:
    """Random pattern that is NOT structurally symmetric: each off-diagonal
    (i, j) of the pivoted matrix Atilde is present with probability
    `density`, independently of (j, i) (triangle "upper" / "lower": only
    that triangle).  Atilde is strictly diagonally dominant by rows and
    columns (no-pivot LU is safe); A is Atilde with scrambled rows and
    columns (see _scramble)."""
    rng = _rng(seed, 12)
    m = int(round(density * n * (n - 1)))
    i = rng.integers(0, n, size=2 * m + 8)
    j = rng.integers(0, n, size=2 * m + 8)
    keep = i != j
    if triangle == "upper":
        keep &= i < j
    elif triangle == "lower":
        keep &= i > j
    key = np.unique(i[keep] * n + j[keep])
    key = rng.permutation(key)[:m]
    r, c = key // n, key % n
    vals = rng.uniform(-1.0, 1.0, size=r.size)
    if complex_values:
        vals = vals + 1j * rng.uniform(-1.0, 1.0, size=r.size)
    a = np.abs(vals)
    diag = (np.bincount(r, weights=a, minlength=n) + np.bincount(c, weights=a, minlength=n)
            + 1.0 + rng.uniform(0.0, 1.0, size=n))
    if complex_values:
        diag = diag + 1j * rng.uniform(-0.5, 0.5, size=n)
    idx = np.arange(n, dtype=np.int64)
    return _scramble(n, np.concatenate([idx, r]), np.concatenate([idx, c]),
                     np.concatenate([diag, vals]), seed, f"general_{n}_{density}{triangle}",
                     max_sn, (n,), rng.permutation(n), row_scramble)


def upwind_oneway_2d(m: int, seed: int, max_sn: int = 64, complex_values: bool = False,
                     row_scramble: bool = True) -> Problem:
    """2D convection on an m x m grid with one-sided (upwind) couplings:
    node i couples to its -x and -y neighbours always and to its +x / +y
    neighbour with probability 1/2 each, so the pattern is not structurally
    symmetric.  Values U(-1, 0) off the diagonal, a_ii = 1 + sum of the
    absolute values of row i and column i.  Columns in the grid's nested
    dissection order; rows scrambled (static pivoting restores them)."""
    dims = (m, m)
    idx, coords = _coords(dims)
    n = idx.size
    rng = _rng(seed, 13)
    rows, cols = [], []
    for d in range(2):
        for sgn, prob in ((-1, 1.0), (+1, 0.5)):
            off = [0, 0]
            off[d] = sgn
            mask, j = _neighbour(dims, coords, off)
            mask &= rng.uniform(0.0, 1.0, size=n) < prob
            rows.append(idx[mask])
            cols.append(j[mask])
    r, c = np.concatenate(rows), np.concatenate(cols)
    vals = -rng.uniform(0.0, 1.0, size=r.size)
    if complex_values:
        vals = vals + 1j * rng.uniform(-0.5, 0.5, size=r.size)
    a = np.abs(vals)
    diag = 1.0 + np.bincount(r, weights=a, minlength=n) + np.bincount(c, weights=a, minlength=n)
    perm = nd_perm(dims, max_sn)
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    # Atilde in the nested-dissection order: new index iperm[old]
    return _scramble(n, iperm[np.concatenate([idx, r])], iperm[np.concatenate([idx, c])],
                     np.concatenate([diag.astype(vals.dtype), vals]), seed,
                     f"upwind_oneway_2d_{m}", max_sn, dims, perm, row_scramble)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def make_config(k: int, size: int | None = None, instances: int | None = None):
    """Workload ``k`` (1..5), optionally at a reduced grid ``size``.

    Returns a Problem, except config 4 which returns a list: the shifted 3D
    family first, then the uneven 2D grids.
    """
    seed = SEED_BASE + k
    if k == 1:
        return conv_diff_2d(size or 31, seed, sigma=0.1, max_sn=64, name="cfg1")
    if k == 2:
        return upwind_3d(size or 40, seed, shift=0.1, max_sn=256, name="cfg2")
    if k == 3:
        return stencil27_complex(size or 60, seed, max_sn=256, name="cfg3")
    if k == 4:
        nshift = instances or 40
        fam = shifted_family(size or 32, seed, nshift=nshift, max_sn=256, name="cfg4_shifts")
        ngrid = 64 if instances is None else instances
        lo, hi = (20, 100) if size is None else (max(4, size // 2), max(5, size))
        grids = []
        for g in range(ngrid):
            mg = lo + ((hi - lo) * g) // max(1, ngrid - 1)
            grids.append(conv_diff_2d(mg, seed + g, sigma=0.1, imag_diag=0.1, max_sn=256,
                                      name=f"cfg4_grid{g}"))
        return [fam] + grids
    if k == 5:
        return dg_blocks(size or 16, 64, seed, max_sn=256, name="cfg5")
    raise ValueError(f"unknown config {k}")
