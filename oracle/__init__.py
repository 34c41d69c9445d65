"""CPU oracle for the selected inversion path (TEST INFRASTRUCTURE ONLY).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.

The compiled part (``oracle.c``) is the scalar, column-by-column statement of
the method (Section 2, Theorem 1 and Theorem 2); ``sampled.py`` computes
individual columns of A^{-1} by sparse triangular solves for workloads too
large for the scalar oracle.  ``build()`` compiles ``liboracle.so`` with the
system C compiler.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -2: "pattern not structurally symmetric",
          -3: "zero pivot", -4: "out of memory", -5: "singular"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C11, no FMA contraction)."""
    src = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_general.c")]
    deps = src + [os.path.join(_HERE, "oracle.h"), os.path.join(_HERE, "oracle_num.inc"),
                  os.path.join(_HERE, "oracle_gnum.inc")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(d) <= t for d in deps):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp] + src + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        lib.oracle_analyze.argtypes = [I, P, P, P, I, I, ctypes.POINTER(P)]
        lib.oracle_analyze.restype = ctypes.c_int
        lib.oracle_sym_free.argtypes = [P]
        lib.oracle_sym_free.restype = None
        for name in ("oracle_sym_n", "oracle_sym_nnzl", "oracle_sym_nsup"):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = I
        for name in ("oracle_sym_parent", "oracle_sym_sptr", "oracle_sym_sidx",
                     "oracle_sym_supptr", "oracle_sym_sup_parent", "oracle_sym_sup_depth"):
            getattr(lib, name).argtypes = [P]
            getattr(lib, name).restype = ctypes.POINTER(I)
        for t in ("d", "z"):
            f = getattr(lib, f"oracle_lu_{t}")
            f.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(I)]
            f.restype = ctypes.c_int
            f = getattr(lib, f"oracle_selinv_{t}")
            f.argtypes = [P, P, P, P, P, P, P, ctypes.c_int]
            f.restype = ctypes.c_int
            f = getattr(lib, f"oracle_selinv_par_{t}")
            f.argtypes = [P, P, P, P, P, P, P, ctypes.c_int]
            f.restype = ctypes.c_int
            f = getattr(lib, f"oracle_extract_{t}")
            f.argtypes = [P, P, P, P, P, P, P]
            f.restype = ctypes.c_int
        lib.oracle_dense_inverse_dd.argtypes = [I, P, P, P]
        lib.oracle_dense_inverse_dd.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _arr(p, size):
    if size == 0:
        return np.zeros(0, dtype=np.int64)
    return np.ctypeslib.as_array(p, shape=(size,)).copy()


class Symbolic:
    """Result of the oracle's symbolic analysis (all arrays int64, permuted indices)."""

    def __init__(self, n, colptr, rowind, perm, max_sn, relax_pct=0):
        lib = _load()
        self._colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self._rowind = np.ascontiguousarray(rowind, dtype=np.int64)
        self._perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib.oracle_analyze(int(n), _ptr(self._colptr), _ptr(self._rowind),
                                None if self._perm is None else _ptr(self._perm),
                                int(max_sn), int(relax_pct), ctypes.byref(h))
        if rc != 0:
            raise OracleError(rc, "analyze")
        self._h = h
        self.n = int(lib.oracle_sym_n(h))
        self.nnzl = int(lib.oracle_sym_nnzl(h))
        self.nsup = int(lib.oracle_sym_nsup(h))
        self.parent = _arr(lib.oracle_sym_parent(h), self.n)
        self.sptr = _arr(lib.oracle_sym_sptr(h), self.n + 1)
        self.sidx = _arr(lib.oracle_sym_sidx(h), self.nnzl)
        self.supptr = _arr(lib.oracle_sym_supptr(h), self.nsup + 1)
        self.sup_parent = _arr(lib.oracle_sym_sup_parent(h), self.nsup)
        self.sup_depth = _arr(lib.oracle_sym_sup_depth(h), self.nsup)
        self.perm = (np.arange(self.n, dtype=np.int64) if perm is None
                     else np.asarray(perm, dtype=np.int64).copy())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_sym_free(h)
            self._h = None

    # -- derived views ----------------------------------------------------
    def supernode_rows(self, k: int) -> np.ndarray:
        """R_K = struct(last column of supernode K)."""
        last = int(self.supptr[k + 1]) - 1
        return self.sidx[self.sptr[last]:self.sptr[last + 1]]

    def lu_pattern(self):
        """(rows, cols) of every entry of L+U in permuted indices, in the
        order diag[0..n), lower[0..nnzl), upper[0..nnzl)."""
        cols_low = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.sptr))
        rows = np.concatenate([np.arange(self.n), self.sidx, cols_low])
        cols = np.concatenate([np.arange(self.n), cols_low, self.sidx])
        return rows, cols


DEFAULT_RELAX_PCT = 20


def analyze(problem, relax_pct: int | None = None) -> Symbolic:
    if relax_pct is None:
        relax_pct = problem.meta.get("relax_pct", DEFAULT_RELAX_PCT)
    return Symbolic(problem.n, problem.colptr, problem.rowind, problem.perm,
                    problem.max_supernode, relax_pct)


class Factors:
    def __init__(self, sym, low, up, diag):
        self.sym, self.low, self.up, self.diag = sym, low, up, diag


def lu(sym: Symbolic, colptr, rowind, values) -> Factors:
    lib = _load()
    values = np.ascontiguousarray(values)
    cplx = np.iscomplexobj(values)
    dt = np.complex128 if cplx else np.float64
    values = values.astype(dt, copy=False)
    low = np.zeros(sym.nnzl, dtype=dt)
    up = np.zeros(sym.nnzl, dtype=dt)
    diag = np.zeros(sym.n, dtype=dt)
    bad = ctypes.c_int64(-1)
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int64)
    f = lib.oracle_lu_z if cplx else lib.oracle_lu_d
    rc = f(sym._h, _ptr(colptr), _ptr(rowind), _ptr(values), _ptr(low), _ptr(up), _ptr(diag),
           ctypes.byref(bad))
    if rc != 0:
        raise OracleError(rc, f"lu (column {bad.value})")
    return Factors(sym, low, up, diag)


class Selected:
    """A^{-1} on the pattern of L+U, stored like the factors (permuted indices)."""

    def __init__(self, sym, low, up, diag):
        self.sym, self.low, self.up, self.diag = sym, low, up, diag

    def values_lu_order(self):
        """Values in the order of ``Symbolic.lu_pattern()``."""
        return np.concatenate([self.diag, self.low, self.up])


def selinv(fac: Factors, mutation: int = 0) -> Selected:
    lib = _load()
    sym = fac.sym
    dt = fac.low.dtype
    bl = np.zeros(sym.nnzl, dtype=dt)
    bu = np.zeros(sym.nnzl, dtype=dt)
    bd = np.zeros(sym.n, dtype=dt)
    f = lib.oracle_selinv_z if np.iscomplexobj(fac.low) else lib.oracle_selinv_d
    rc = f(sym._h, _ptr(fac.low), _ptr(fac.up), _ptr(fac.diag), _ptr(bl), _ptr(bu), _ptr(bd),
           int(mutation))
    if rc != 0:
        raise OracleError(rc, "selinv")
    return Selected(sym, bl, bu, bd)


def selinv_parallel(fac: Factors, nthreads: int) -> Selected:
    """selinv with the independent columns of each depth of the structures'
    tree run by ``nthreads`` OpenMP threads (bit for bit selinv's result)."""
    lib = _load()
    sym = fac.sym
    dt = fac.low.dtype
    bl = np.zeros(sym.nnzl, dtype=dt)
    bu = np.zeros(sym.nnzl, dtype=dt)
    bd = np.zeros(sym.n, dtype=dt)
    f = lib.oracle_selinv_par_z if np.iscomplexobj(fac.low) else lib.oracle_selinv_par_d
    rc = f(sym._h, _ptr(fac.low), _ptr(fac.up), _ptr(fac.diag), _ptr(bl), _ptr(bu), _ptr(bd),
           int(nthreads))
    if rc != 0:
        raise OracleError(rc, "selinv_parallel")
    return Selected(sym, bl, bu, bd)


def extract(sel: Selected, colptr, rowind) -> np.ndarray:
    """Selected entries on the pattern of A in the original ordering (Theorem 2)."""
    lib = _load()
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int64)
    out = np.zeros(rowind.size, dtype=sel.low.dtype)
    f = lib.oracle_extract_z if np.iscomplexobj(sel.low) else lib.oracle_extract_d
    rc = f(sel.sym._h, _ptr(colptr), _ptr(rowind), _ptr(sel.low), _ptr(sel.up), _ptr(sel.diag),
           _ptr(out))
    if rc != 0:
        raise OracleError(rc, "extract")
    return out


def dense_inverse_dd(a: np.ndarray):
    """(hi, lo) of the double-double Gauss-Jordan inverse of a real matrix."""
    lib = _load()
    a = np.asfortranarray(a, dtype=np.float64)
    n = a.shape[0]
    hi = np.zeros((n, n), dtype=np.float64, order="F")
    lo = np.zeros((n, n), dtype=np.float64, order="F")
    rc = lib.oracle_dense_inverse_dd(n, _ptr(a), _ptr(hi), _ptr(lo))
    if rc != 0:
        raise OracleError(rc, "dense inverse")
    return hi, lo


def dense_inverse_dd_complex(a: np.ndarray) -> np.ndarray:
    """Complex inverse through the real embedding [[X, -Y], [Y, X]] of X + iY."""
    n = a.shape[0]
    x, y = a.real, a.imag
    big = np.block([[x, -y], [y, x]])
    hi, lo = dense_inverse_dd(big)
    inv = hi + lo
    return inv[:n, :n] + 1j * inv[n:, :n]


def selected_inverse(problem, b: int = 0, mutation: int = 0, relax_pct: int | None = None):
    """Convenience: analyze + lu + selinv for instance b of a Problem."""
    sym = analyze(problem, relax_pct)
    vals = problem.values if problem.values.ndim == 1 else problem.values[b]
    fac = lu(sym, problem.colptr, problem.rowind, vals)
    return selinv(fac, mutation=mutation)


# ---------------------------------------------------------------------------
# general patterns and static pivoting (oracle_general.c)
# ---------------------------------------------------------------------------
def _gload():
    lib = _load()
    if getattr(lib, "_general_bound", False):
        return lib
    P = ctypes.c_void_p
    I = ctypes.c_int64
    lib.oracle_ganalyze.argtypes = [I, P, P, P, P, ctypes.POINTER(P)]
    lib.oracle_ganalyze.restype = ctypes.c_int
    lib.oracle_gsym_free.argtypes = [P]
    lib.oracle_gsym_free.restype = None
    for name in ("oracle_gsym_n", "oracle_gsym_nnzl", "oracle_gsym_nnzu"):
        getattr(lib, name).argtypes = [P]
        getattr(lib, name).restype = I
    for name in ("oracle_gsym_lptr", "oracle_gsym_lidx", "oracle_gsym_uptr", "oracle_gsym_uidx"):
        getattr(lib, name).argtypes = [P]
        getattr(lib, name).restype = ctypes.POINTER(I)
    for t in ("d", "z"):
        f = getattr(lib, f"oracle_glu_{t}")
        f.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(I)]
        f.restype = ctypes.c_int
        f = getattr(lib, f"oracle_gselinv_{t}")
        f.argtypes = [P, P, P, P, P, P, P, ctypes.c_int]
        f.restype = ctypes.c_int
        f = getattr(lib, f"oracle_gextract_{t}")
        f.argtypes = [P, P, P, P, P, P, P]
        f.restype = ctypes.c_int
    lib._general_bound = True
    return lib


class GSymbolic:
    """Structures C_L(k) (columns of L) and C_U(k) (rows of U) of
    Atilde = P A Q, permuted indices (oracle_ganalyze)."""

    def __init__(self, n, colptr, rowind, rperm=None, cperm=None):
        lib = _gload()
        self._colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self._rowind = np.ascontiguousarray(rowind, dtype=np.int64)
        rp = None if rperm is None else np.ascontiguousarray(rperm, dtype=np.int64)
        cp = None if cperm is None else np.ascontiguousarray(cperm, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib.oracle_ganalyze(int(n), _ptr(self._colptr), _ptr(self._rowind),
                                 None if rp is None else _ptr(rp),
                                 None if cp is None else _ptr(cp), ctypes.byref(h))
        if rc != 0:
            raise OracleError(rc, "ganalyze")
        self._h = h
        self.n = int(lib.oracle_gsym_n(h))
        self.nnzl = int(lib.oracle_gsym_nnzl(h))
        self.nnzu = int(lib.oracle_gsym_nnzu(h))
        self.lptr = _arr(lib.oracle_gsym_lptr(h), self.n + 1)
        self.lidx = _arr(lib.oracle_gsym_lidx(h), self.nnzl)
        self.uptr = _arr(lib.oracle_gsym_uptr(h), self.n + 1)
        self.uidx = _arr(lib.oracle_gsym_uidx(h), self.nnzu)
        self.rperm = np.arange(self.n) if rp is None else rp.copy()
        self.cperm = np.arange(self.n) if cp is None else cp.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_gsym_free(h)
            self._h = None

    def col_l(self, k):
        return self.lidx[self.lptr[k]:self.lptr[k + 1]]

    def row_u(self, k):
        return self.uidx[self.uptr[k]:self.uptr[k + 1]]

    def inverse_pattern(self):
        """(rows, cols) of the computed entries B_{i,j} of Atilde^{-1} (the
        pattern of (L+U)^T) in the order diag, BL, BU."""
        kl = np.repeat(np.arange(self.n), np.diff(self.lptr))
        ku = np.repeat(np.arange(self.n), np.diff(self.uptr))
        rows = np.concatenate([np.arange(self.n), kl, self.uidx])
        cols = np.concatenate([np.arange(self.n), self.lidx, ku])
        return rows, cols


def ganalyze(problem) -> GSymbolic:
    """General analysis of a Problem with optional ``rperm``/``cperm`` in its
    meta (default: its symmetric ``perm`` for both)."""
    rp = problem.meta.get("rperm", problem.perm)
    cp = problem.meta.get("cperm", problem.perm)
    return GSymbolic(problem.n, problem.colptr, problem.rowind, rp, cp)


class GFactors:
    def __init__(self, sym, low, up, diag):
        self.sym, self.low, self.up, self.diag = sym, low, up, diag


class GSelected:
    def __init__(self, sym, bl, bu, bd):
        self.sym, self.bl, self.bu, self.bd = sym, bl, bu, bd

    def values(self):
        """Values in the order of GSymbolic.inverse_pattern()."""
        return np.concatenate([self.bd, self.bl, self.bu])


def glu(sym: GSymbolic, colptr, rowind, values) -> GFactors:
    lib = _gload()
    values = np.ascontiguousarray(values)
    cplx = np.iscomplexobj(values)
    dt = np.complex128 if cplx else np.float64
    values = values.astype(dt, copy=False)
    low = np.zeros(sym.nnzl, dtype=dt)
    up = np.zeros(sym.nnzu, dtype=dt)
    diag = np.zeros(sym.n, dtype=dt)
    bad = ctypes.c_int64(-1)
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int64)
    f = lib.oracle_glu_z if cplx else lib.oracle_glu_d
    rc = f(sym._h, _ptr(colptr), _ptr(rowind), _ptr(values), _ptr(low), _ptr(up), _ptr(diag),
           ctypes.byref(bad))
    if rc != 0:
        raise OracleError(rc, f"glu (column {bad.value})")
    return GFactors(sym, low, up, diag)


def gselinv(fac: GFactors, mutation: int = 0) -> GSelected:
    lib = _gload()
    sym = fac.sym
    dt = fac.diag.dtype
    bl = np.zeros(sym.nnzl, dtype=dt)
    bu = np.zeros(sym.nnzu, dtype=dt)
    bd = np.zeros(sym.n, dtype=dt)
    f = lib.oracle_gselinv_z if np.iscomplexobj(fac.diag) else lib.oracle_gselinv_d
    rc = f(sym._h, _ptr(fac.low), _ptr(fac.up), _ptr(fac.diag), _ptr(bl), _ptr(bu), _ptr(bd),
           int(mutation))
    if rc != 0:
        raise OracleError(rc, "gselinv")
    return GSelected(sym, bl, bu, bd)


def gextract(sel: GSelected, colptr, rowind) -> np.ndarray:
    """out[p] = (A^{-1})_{x,y} for entry p of A at row y = rowind[p], column x."""
    lib = _gload()
    colptr = np.ascontiguousarray(colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(rowind, dtype=np.int64)
    out = np.zeros(rowind.size, dtype=sel.bd.dtype)
    f = lib.oracle_gextract_z if np.iscomplexobj(sel.bd) else lib.oracle_gextract_d
    rc = f(sel.sym._h, _ptr(colptr), _ptr(rowind), _ptr(sel.bl), _ptr(sel.bu), _ptr(sel.bd),
           _ptr(out))
    if rc != 0:
        raise OracleError(rc, "gextract")
    return out


def general_selected_inverse(problem, b: int = 0, mutation: int = 0) -> GSelected:
    """ganalyze + glu + gselinv for instance b of a Problem."""
    sym = ganalyze(problem)
    vals = problem.values if problem.values.ndim == 1 else problem.values[b]
    return gselinv(glu(sym, problem.colptr, problem.rowind, vals), mutation=mutation)
