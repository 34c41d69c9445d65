"""ctypes binding of libpselinv.so: the same entry points as include/pselinv.h.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA); only
their data pointers are passed.  Streams are torch.cuda.Stream objects,
raw cudaStream_t integers, or None (the current torch stream if torch has
CUDA, else the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libpselinv.so")

F64, C128 = 1, 2
PREC_FP64, PREC_OZAKI_FP16 = 0, 1
SCHED_LEVEL, SCHED_PER_SUPERNODE = 0, 1
LAYOUT_PATTERN_A, LAYOUT_SUPERNODAL, LAYOUT_FACTORS = 0, 1, 2

ERRORS = {0: "ok", -1: "invalid argument", -2: "not structurally symmetric", -3: "zero pivot",
          -4: "out of memory", -5: "CUDA error", -6: "timeout", -7: "index check failed",
          -8: "unsupported"}

_EXPORTS = [
    "pselinv_default_opts", "pselinv_analyze", "pselinv_factor", "pselinv_selinv",
    "pselinv_get_selected", "pselinv_get_structure", "pselinv_profile", "pselinv_plan_stats",
    "pselinv_sync", "pselinv_last_info", "pselinv_error_string", "pselinv_free",
    "pselinv_block_inverse_noalloc", "pselinv_tune", "pselinv_tune_records",
    "pselinv_plan_get", "pselinv_plan_set", "pselinv_wait_selftest", "pselinv_measure_fp64_peak",
    "pselinv_set_schedule", "pselinv_set_factor_precision", "pselinv_group",
    "pselinv_analyze_general",
    "pselinv_partition", "pselinv_set_subset", "pselinv_export_block", "pselinv_import_block",
    "pselinv_weighted_sum", "pselinv_trace",
    "pselinv_model_create", "pselinv_model_train", "pselinv_model_gradients",
    "pselinv_model_predict", "pselinv_model_get_params", "pselinv_model_set_params",
    "pselinv_model_encode", "pselinv_model_free",
]

TUNE_RESET, TUNE_EXHAUSTIVE, TUNE_MODEL = 0, 1, 2

STEP_KINDS = {0: "gemm", 1: "tri_inv", 2: "diag_lu", 3: "gather", 4: "scatter_sub", 5: "copy",
              6: "memset", 7: "scatter_values", 8: "slice", 9: "ozaki_gemm", 10: "recombine",
              11: "small_level", 12: "gather_slice", 13: "output_maxima"}


class LibraryMissing(RuntimeError):
    pass


class PselinvError(RuntimeError):
    def __init__(self, code, what, info=-1):
        msg = f"{what}: {ERRORS.get(code, code)} ({code})"
        if info >= 0:
            msg += f", info {info}"
        super().__init__(msg)
        self.code = code
        self.info = info


class Opts(ctypes.Structure):
    _fields_ = [("max_supernode", ctypes.c_int32), ("relax_pct", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("check_level", ctypes.c_int32),
                ("host_only", ctypes.c_int32), ("split_normalise", ctypes.c_int32),
                ("symmetric", ctypes.c_int32), ("nd_leaf", ctypes.c_int32),
                ("factor_precision", ctypes.c_int32), ("factor_split_mflops", ctypes.c_int32),
                ("ozaki_a_tmem", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


_P64 = ctypes.POINTER(ctypes.c_int64)


class TuneRecord(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("level", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("param", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("feat", ctypes.c_float * 8), ("ms", ctypes.c_double)]


class StepStat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("level", ctypes.c_int32), ("tasks", ctypes.c_int64),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("ms", ctypes.c_double),
                ("param", ctypes.c_int32), ("side", ctypes.c_int32), ("start_ms", ctypes.c_double)]


class Structure(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nsuper", ctypes.c_int64), ("nlevels", ctypes.c_int64),
                ("storage_size", ctypes.c_int64), ("nnz_a", ctypes.c_int64),
                ("perm", _P64), ("etree", _P64), ("sn_first", _P64), ("sn_width", _P64),
                ("sn_parent", _P64), ("sn_depth", _P64), ("sn_offset", _P64),
                ("rows_ptr", _P64), ("rows", _P64), ("level_ptr", _P64), ("level_sn", _P64),
                ("value_map", _P64), ("flops_selinv", ctypes.c_double),
                ("flops_selinv_exact", ctypes.c_double), ("flops_factor", ctypes.c_double),
                ("general", ctypes.c_int64), ("rperm", _P64), ("urows_ptr", _P64),
                ("urows", _P64), ("out_map", _P64)]


_lib = None


def lib_path() -> str:
    return _LIB


def load_library():
    """Load libpselinv.so (raises LibraryMissing if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB):
        raise LibraryMissing(f"{_LIB} is missing: build it with "
                             "`python -m paper_1708_04539_gb300.build`")
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.pselinv_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.pselinv_default_opts.restype = None
    lib.pselinv_plan_save.argtypes = [P, ctypes.c_int, ctypes.c_char_p]
    lib.pselinv_plan_save.restype = ctypes.c_int
    lib.pselinv_plan_load.argtypes = [P, ctypes.c_int, ctypes.c_char_p]
    lib.pselinv_plan_load.restype = ctypes.c_int
    lib.pselinv_order_nd.argtypes = [I64, P, P, I64, P]
    lib.pselinv_order_nd.restype = ctypes.c_int
    lib.pselinv_analyze.argtypes = [I64, P, P, P, ctypes.POINTER(Opts), ctypes.POINTER(P)]
    lib.pselinv_analyze.restype = ctypes.c_int
    lib.pselinv_factor.argtypes = [P, ctypes.c_int, I64, P, P]
    lib.pselinv_factor.restype = ctypes.c_int
    lib.pselinv_selinv.argtypes = [P, ctypes.c_int, P]
    lib.pselinv_selinv.restype = ctypes.c_int
    lib.pselinv_get_selected.argtypes = [P, ctypes.c_int, I64, P, P]
    lib.pselinv_get_selected.restype = ctypes.c_int
    lib.pselinv_get_structure.argtypes = [P, ctypes.POINTER(Structure)]
    lib.pselinv_get_structure.restype = ctypes.c_int
    lib.pselinv_profile.argtypes = [P, ctypes.c_int, P, ctypes.POINTER(StepStat), I64,
                                    ctypes.POINTER(I64)]
    lib.pselinv_profile.restype = ctypes.c_int
    lib.pselinv_plan_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.pselinv_plan_stats.restype = ctypes.c_int
    lib.pselinv_sync.argtypes = [P, P]
    lib.pselinv_sync.restype = ctypes.c_int
    lib.pselinv_last_info.argtypes = [P]
    lib.pselinv_last_info.restype = I64
    lib.pselinv_error_string.argtypes = [ctypes.c_int]
    lib.pselinv_error_string.restype = ctypes.c_char_p
    lib.pselinv_free.argtypes = [P]
    lib.pselinv_free.restype = None
    lib.pselinv_block_inverse_noalloc.argtypes = [ctypes.c_int, I64, P, I64, P, I64, P]
    lib.pselinv_block_inverse_noalloc.restype = ctypes.c_int
    lib.pselinv_wait_selftest.argtypes = [P, I64]
    lib.pselinv_wait_selftest.restype = ctypes.c_int
    lib.pselinv_measure_fp64_peak.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]
    lib.pselinv_measure_fp64_peak.restype = ctypes.c_int
    lib.pselinv_analyze_general.argtypes = [I64, P, P, P, P, ctypes.POINTER(Opts),
                                            ctypes.POINTER(P)]
    lib.pselinv_analyze_general.restype = ctypes.c_int
    lib.pselinv_group.argtypes = [P, I64, ctypes.POINTER(Opts), ctypes.POINTER(P)]
    lib.pselinv_group.restype = ctypes.c_int
    lib.pselinv_partition.argtypes = [P, ctypes.c_int32, P]
    lib.pselinv_partition.restype = ctypes.c_int
    lib.pselinv_set_subset.argtypes = [P, P, ctypes.c_int32]
    lib.pselinv_set_subset.restype = ctypes.c_int
    lib.pselinv_export_block.argtypes = [P, I64, I64, P, P]
    lib.pselinv_export_block.restype = ctypes.c_int
    lib.pselinv_import_block.argtypes = [P, I64, I64, P, P]
    lib.pselinv_import_block.restype = ctypes.c_int
    lib.pselinv_set_schedule.argtypes = [P, ctypes.c_int]
    lib.pselinv_set_schedule.restype = ctypes.c_int
    lib.pselinv_set_factor_precision.argtypes = [P, ctypes.c_int, ctypes.c_int32]
    lib.pselinv_set_factor_precision.restype = ctypes.c_int
    RP = ctypes.POINTER(TuneRecord)
    lib.pselinv_tune.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.pselinv_tune.restype = ctypes.c_int
    lib.pselinv_tune_records.argtypes = [P, RP, I64, ctypes.POINTER(I64)]
    lib.pselinv_tune_records.restype = ctypes.c_int
    lib.pselinv_plan_get.argtypes = [P, ctypes.c_int, P, I64, ctypes.POINTER(I64)]
    lib.pselinv_plan_get.restype = ctypes.c_int
    lib.pselinv_plan_set.argtypes = [P, ctypes.c_int, P, I64]
    lib.pselinv_plan_set.restype = ctypes.c_int
    lib.pselinv_weighted_sum.argtypes = [P, P, P, P]
    lib.pselinv_weighted_sum.restype = ctypes.c_int
    lib.pselinv_trace.argtypes = [P, P, P, P, P]
    lib.pselinv_trace.restype = ctypes.c_int
    lib.pselinv_model_create.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(P)]
    lib.pselinv_model_create.restype = ctypes.c_int
    lib.pselinv_model_train.argtypes = [P, RP, I64, ctypes.c_int32, ctypes.c_float, P,
                                        ctypes.POINTER(ctypes.c_float)]
    lib.pselinv_model_train.restype = ctypes.c_int
    lib.pselinv_model_gradients.argtypes = [P, RP, I64, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float), P]
    lib.pselinv_model_gradients.restype = ctypes.c_int
    lib.pselinv_model_predict.argtypes = [P, RP, I64, ctypes.POINTER(ctypes.c_double), P]
    lib.pselinv_model_predict.restype = ctypes.c_int
    lib.pselinv_model_get_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), I64,
                                             ctypes.POINTER(I64)]
    lib.pselinv_model_get_params.restype = ctypes.c_int
    lib.pselinv_model_set_params.argtypes = [P, ctypes.POINTER(ctypes.c_float), I64]
    lib.pselinv_model_set_params.restype = ctypes.c_int
    lib.pselinv_model_encode.argtypes = [RP, I64, ctypes.POINTER(ctypes.c_float)]
    lib.pselinv_model_encode.restype = ctypes.c_int
    lib.pselinv_model_free.argtypes = [P]
    lib.pselinv_model_free.restype = None
    _lib = lib
    return lib


def exported_symbols():
    return list(_EXPORTS)


def _ptr(x):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported array type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _is_complex(x) -> bool:
    if isinstance(x, np.ndarray):
        return np.iscomplexobj(x)
    return bool(getattr(x, "is_complex", lambda: False)())


class SelInv:
    """One analysed pattern (a handle of the C library)."""

    @staticmethod
    def _opts(lib, max_supernode=256, relax_pct=20, schedule=SCHED_LEVEL, use_graph=True,
              check_level=0, precision=PREC_FP64, slices=0, host_only=False,
              split_normalise=False, symmetric=False, nd_leaf=0, factor_precision=PREC_FP64,
              factor_split_mflops=0, ozaki_a_tmem=False):
        opts = Opts()
        lib.pselinv_default_opts(ctypes.byref(opts))
        opts.max_supernode = int(max_supernode)
        opts.relax_pct = int(relax_pct)
        opts.schedule = int(schedule)
        opts.use_graph = 1 if use_graph else 0
        opts.check_level = int(check_level)
        opts.precision = int(precision)
        opts.slices = int(slices)
        opts.host_only = 1 if host_only else 0
        opts.split_normalise = 1 if split_normalise else 0
        opts.symmetric = 1 if symmetric else 0
        opts.nd_leaf = int(nd_leaf)  # perm None: 0 natural order, > 0 nested dissection
        opts.factor_precision = int(factor_precision)
        opts.factor_split_mflops = int(factor_split_mflops)
        opts.ozaki_a_tmem = 1 if ozaki_a_tmem else 0
        return opts

    def __init__(self, n, colptr, rowind, perm=None, **kw):
        lib = load_library()
        self._lib = lib
        opts = self._opts(lib, **kw)
        self._colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self._rowind = np.ascontiguousarray(rowind, dtype=np.int64)
        p = None if perm is None else np.ascontiguousarray(perm, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib.pselinv_analyze(int(n), _ptr(self._colptr), _ptr(self._rowind), _ptr(p),
                                 ctypes.byref(opts), ctypes.byref(h))
        if rc != 0:
            raise PselinvError(rc, "pselinv_analyze")
        self._h = h
        self.n = int(n)
        self.nnz = int(self._colptr[-1])
        self.dtype = None
        self.nbatch = 0

    @classmethod
    def general(cls, n, colptr, rowind, rperm=None, cperm=None, **kw):
        """Handle of a general pattern with static pivoting, Atilde = P A Q
        (pselinv_analyze_general; rperm / cperm new -> old)."""
        lib = load_library()
        self = cls.__new__(cls)
        self._lib = lib
        opts = cls._opts(lib, **kw)
        self._colptr = np.ascontiguousarray(colptr, dtype=np.int64)
        self._rowind = np.ascontiguousarray(rowind, dtype=np.int64)
        rp = None if rperm is None else np.ascontiguousarray(rperm, dtype=np.int64)
        cp = None if cperm is None else np.ascontiguousarray(cperm, dtype=np.int64)
        h = ctypes.c_void_p()
        rc = lib.pselinv_analyze_general(int(n), _ptr(self._colptr), _ptr(self._rowind), _ptr(rp),
                                         _ptr(cp), ctypes.byref(opts), ctypes.byref(h))
        if rc != 0:
            raise PselinvError(rc, "pselinv_analyze_general")
        self._h = h
        self.n = int(n)
        self.nnz = int(self._colptr[-1])
        self.dtype = None
        self.nbatch = 0
        return self

    @classmethod
    def from_general_problem(cls, problem, **kw):
        """General handle of a Problem whose meta carries rperm / cperm."""
        kw.setdefault("max_supernode", problem.max_supernode)
        return cls.general(problem.n, problem.colptr, problem.rowind,
                           problem.meta.get("rperm", problem.perm),
                           problem.meta.get("cperm", problem.perm), **kw)

    @classmethod
    def group(cls, members, **kw):
        """One handle for the direct sum of the members' patterns, in member
        order (pselinv_group); keyword options as for the constructor (none:
        the first member's options)."""
        lib = load_library()
        arr = (ctypes.c_void_p * len(members))(*[m._h.value for m in members])
        opts = cls._opts(lib, **kw) if kw else None
        h = ctypes.c_void_p()
        rc = lib.pselinv_group(arr, len(members), ctypes.byref(opts) if opts is not None else None,
                               ctypes.byref(h))
        if rc != 0:
            raise PselinvError(rc, "pselinv_group")
        self = cls.__new__(cls)
        self._lib = lib
        self._h = h
        self._colptr = np.concatenate([[0]] + [m._colptr[1:] + off for m, off in zip(
            members, np.cumsum([0] + [m.nnz for m in members[:-1]]))]).astype(np.int64)
        self._rowind = np.concatenate([m._rowind + off for m, off in zip(
            members, np.cumsum([0] + [m.n for m in members[:-1]]))]).astype(np.int64)
        self.n = int(sum(m.n for m in members))
        self.nnz = int(sum(m.nnz for m in members))
        self.dtype = None
        self.nbatch = 0
        return self

    @classmethod
    def from_problem(cls, problem, **kw):
        kw.setdefault("max_supernode", problem.max_supernode)
        return cls(problem.n, problem.colptr, problem.rowind, problem.perm, **kw)

    # -- C ABI wrappers ------------------------------------------------------
    def _check(self, rc, what):
        if rc != 0:
            raise PselinvError(rc, what, int(self._lib.pselinv_last_info(self._h)))

    def factor(self, values, stream=None):
        """values: [nnz] or [nbatch, nnz] float64/complex128 (numpy or torch)."""
        shape = tuple(values.shape)
        nbatch = 1 if len(shape) == 1 else shape[0]
        if shape[-1] != self.nnz:
            raise ValueError("values do not match the pattern")
        dt = C128 if _is_complex(values) else F64
        rc = self._lib.pselinv_factor(self._h, dt, nbatch, _ptr(values), _stream(stream))
        self._check(rc, "pselinv_factor")
        self.dtype, self.nbatch = dt, nbatch

    def selinv(self, precision=-1, stream=None):
        self._check(self._lib.pselinv_selinv(self._h, int(precision), _stream(stream)),
                    "pselinv_selinv")

    def get_selected(self, out=None, batch=0, layout=LAYOUT_PATTERN_A, stream=None):
        """Selected entries of instance ``batch``; ``out`` may be host or device."""
        if out is None:
            size = self.nnz if layout == LAYOUT_PATTERN_A else self.structure()["storage_size"]
            if self.nbatch == 0:
                raise PselinvError(-1, "get_selected before factor")
            out = np.zeros(size, dtype=np.complex128 if self.dtype == C128 else np.float64)
        self._check(self._lib.pselinv_get_selected(self._h, int(layout), int(batch), _ptr(out),
                                                   _stream(stream)), "pselinv_get_selected")
        return out

    def profile(self, which=0, stream=None):
        """Launch-by-launch timing of the selinv (0) or factor (1) plan, or the
        timeline of the selinv plan on its own streams (2)."""
        cap = 1 << 16
        buf = (StepStat * cap)()
        cnt = ctypes.c_int64(0)
        self._check(self._lib.pselinv_profile(self._h, int(which), _stream(stream), buf, cap,
                                              ctypes.byref(cnt)), "pselinv_profile")
        return [{"kind": STEP_KINDS.get(buf[i].kind, buf[i].kind), "level": buf[i].level,
                 "tasks": buf[i].tasks, "flops": buf[i].flops, "bytes": buf[i].bytes,
                 "ms": buf[i].ms, "param": buf[i].param, "side": buf[i].side,
                 "start_ms": buf[i].start_ms}
                for i in range(min(cnt.value, cap))]

    def plan_stats(self):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        self._check(self._lib.pselinv_plan_stats(self._h, ctypes.byref(a), ctypes.byref(b)),
                    "pselinv_plan_stats")
        return {"launches_selinv": a.value, "launches_factor": b.value}

    def partition(self, nranks):
        """Rank of every supernode of a partitioned sweep (-1: the top)."""
        ns = int(self.structure()["nsuper"])
        owner = np.empty(max(ns, 1), dtype=np.int32)
        self._check(self._lib.pselinv_partition(self._h, int(nranks), _ptr(owner)),
                    "pselinv_partition")
        return owner[:ns]

    def set_subset(self, owner=None, rank=0):
        """Later sweeps cover the supernodes with owner == rank (None: all)."""
        o = None if owner is None else np.ascontiguousarray(owner, dtype=np.int32)
        self._check(self._lib.pselinv_set_subset(self._h, _ptr(o), int(rank)), "pselinv_set_subset")

    def export_block(self, K, buf, batch=0, stream=None):
        """buf (CUDA tensor, c_K^2 scalars) = Ainv(R_K, R_K)."""
        self._check(self._lib.pselinv_export_block(self._h, int(K), int(batch), _ptr(buf),
                                                   _stream(stream)), "pselinv_export_block")
        return buf

    def import_block(self, K, buf, batch=0, stream=None):
        """Write Ainv(R_K, R_K) from buf (CUDA tensor) into the storage."""
        self._check(self._lib.pselinv_import_block(self._h, int(K), int(batch), _ptr(buf),
                                                   _stream(stream)), "pselinv_import_block")

    def set_schedule(self, schedule):
        """Schedule of later selinv/tune calls (SCHED_LEVEL or SCHED_PER_SUPERNODE)."""
        self._check(self._lib.pselinv_set_schedule(self._h, int(schedule)), "pselinv_set_schedule")

    def set_factor_precision(self, precision, split_mflops=0):
        """Precision of the Schur products of later factor calls (PREC_FP64 or
        PREC_OZAKI_FP16; split_mflops < 0: every level split)."""
        self._check(self._lib.pselinv_set_factor_precision(self._h, int(precision),
                                                           int(split_mflops)),
                    "pselinv_set_factor_precision")

    def tune(self, precision=PREC_FP64, mode=TUNE_EXHAUSTIVE, model=None, stream=None):
        """Autotune the launch shapes of the selected-inversion plan."""
        mh = None if model is None else model._h
        self._check(self._lib.pselinv_tune(self._h, int(precision), int(mode), mh, _stream(stream)),
                    "pselinv_tune")

    def tune_records(self):
        cnt = ctypes.c_int64(0)
        self._check(self._lib.pselinv_tune_records(self._h, None, 0, ctypes.byref(cnt)),
                    "pselinv_tune_records")
        buf = (TuneRecord * max(1, cnt.value))()
        self._check(self._lib.pselinv_tune_records(self._h, buf, cnt.value, ctypes.byref(cnt)),
                    "pselinv_tune_records")
        return [buf[i] for i in range(cnt.value)]

    def plan_get(self, precision=PREC_FP64):
        """Tuned launch shapes as a list of (level, slot, value) triples."""
        cnt = ctypes.c_int64(0)
        self._check(self._lib.pselinv_plan_get(self._h, int(precision), None, 0, ctypes.byref(cnt)),
                    "pselinv_plan_get")
        buf = (ctypes.c_int32 * max(3, 3 * cnt.value))()
        self._check(self._lib.pselinv_plan_get(self._h, int(precision), buf, cnt.value,
                                               ctypes.byref(cnt)), "pselinv_plan_get")
        return [(buf[3 * i], buf[3 * i + 1], buf[3 * i + 2]) for i in range(cnt.value)]

    def plan_set(self, triples, precision=PREC_FP64):
        """Replace the tuned launch shapes (triples from plan_get)."""
        flat = [int(v) for t in triples for v in t]
        buf = (ctypes.c_int32 * max(3, len(flat)))(*flat)
        self._check(self._lib.pselinv_plan_set(self._h, int(precision), buf, len(flat) // 3),
                    "pselinv_plan_set")

    def plan_save(self, path, precision=PREC_FP64):
        """Write the tuned values of `precision` to a cache file."""
        self._check(self._lib.pselinv_plan_save(self._h, int(precision), os.fsencode(path)),
                    "pselinv_plan_save")

    def plan_load(self, path, precision=PREC_FP64):
        """Load tuned values saved for this structure and precision."""
        self._check(self._lib.pselinv_plan_load(self._h, int(precision), os.fsencode(path)),
                    "pselinv_plan_load")

    def _weights(self, weights):
        cplx = self.dtype == C128
        w = np.ascontiguousarray(weights, dtype=np.complex128 if cplx else np.float64)
        if w.size != self.nbatch:
            raise ValueError(f"{w.size} weights for {self.nbatch} instances")
        return w

    def weighted_sum(self, weights, out=None, stream=None):
        """sum_l w_l A_l^{-1} on pattern(A), CSC order (a pole-expansion sum)."""
        w = self._weights(weights)
        if out is None:
            out = np.zeros(self.nnz, dtype=w.dtype)
        self._check(self._lib.pselinv_weighted_sum(self._h, _ptr(w), _ptr(out), _stream(stream)),
                    "pselinv_weighted_sum")
        return out

    def trace(self, weights, B, stream=None):
        """sum_l w_l Tr[B A_l^{-1}] for B given on pattern(A) in CSC order."""
        w = self._weights(weights)
        if isinstance(B, np.ndarray):
            B = np.ascontiguousarray(B, dtype=w.dtype)
        res = np.zeros(1, dtype=w.dtype)
        self._check(self._lib.pselinv_trace(self._h, _ptr(w), _ptr(B), _ptr(res), _stream(stream)),
                    "pselinv_trace")
        return res[0]

    def sync(self, stream=None):
        self._check(self._lib.pselinv_sync(self._h, _stream(stream)), "pselinv_sync")

    def structure(self) -> dict:
        s = Structure()
        self._check(self._lib.pselinv_get_structure(self._h, ctypes.byref(s)),
                    "pselinv_get_structure")

        def arr(p, size):
            if size == 0:
                return np.zeros(0, dtype=np.int64)
            return np.ctypeslib.as_array(p, shape=(size,)).copy()

        ns = s.nsuper
        out = {
            "n": s.n, "nsuper": ns, "nlevels": s.nlevels, "storage_size": s.storage_size,
            "nnz_a": s.nnz_a,
            "perm": arr(s.perm, s.n), "etree": arr(s.etree, s.n),
            "sn_first": arr(s.sn_first, ns), "sn_width": arr(s.sn_width, ns),
            "sn_parent": arr(s.sn_parent, ns), "sn_depth": arr(s.sn_depth, ns),
            "sn_offset": arr(s.sn_offset, ns), "rows_ptr": arr(s.rows_ptr, ns + 1),
            "level_ptr": arr(s.level_ptr, s.nlevels + 1), "level_sn": arr(s.level_sn, ns),
            "value_map": arr(s.value_map, s.nnz_a),
            "flops_selinv": s.flops_selinv, "flops_selinv_exact": s.flops_selinv_exact,
            "flops_factor": s.flops_factor,
        }
        out["rows"] = arr(s.rows, int(out["rows_ptr"][-1]) if ns else 0)
        out["general"] = bool(s.general)
        out["rperm"] = arr(s.rperm, s.n)
        out["urows_ptr"] = arr(s.urows_ptr, ns + 1)
        out["urows"] = arr(s.urows, int(out["urows_ptr"][-1]) if ns else 0)
        out["out_map"] = arr(s.out_map, s.nnz_a)
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.pselinv_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class CostModel:
    """The learned launch-shape cost model (an MLP on the device)."""

    def __init__(self, hidden=32, seed=1):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.pselinv_model_create(int(hidden), int(seed), ctypes.byref(h))
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_create")
        self._h = h

    @staticmethod
    def _recs(records):
        arr = (TuneRecord * len(records))()
        for i, r in enumerate(records):
            arr[i] = r
        return arr

    def train(self, records, epochs=2000, lr=3e-3, stream=None):
        loss = ctypes.c_float(0)
        rc = self._lib.pselinv_model_train(self._h, self._recs(records), len(records), int(epochs),
                                           float(lr), _stream(stream), ctypes.byref(loss))
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_train")
        return loss.value

    def gradients(self, records, stream=None):
        n = self.num_params()
        g = (ctypes.c_float * n)()
        loss = ctypes.c_float(0)
        rc = self._lib.pselinv_model_gradients(self._h, self._recs(records), len(records), g,
                                               ctypes.byref(loss), _stream(stream))
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_gradients")
        return np.array(g[:], dtype=np.float32), loss.value

    def predict(self, records, stream=None):
        out = (ctypes.c_double * len(records))()
        rc = self._lib.pselinv_model_predict(self._h, self._recs(records), len(records), out,
                                             _stream(stream))
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_predict")
        return np.array(out[:])

    def num_params(self):
        cnt = ctypes.c_int64(0)
        self._lib.pselinv_model_get_params(self._h, None, 0, ctypes.byref(cnt))
        return cnt.value

    def params(self):
        n = self.num_params()
        buf = (ctypes.c_float * n)()
        cnt = ctypes.c_int64(0)
        rc = self._lib.pselinv_model_get_params(self._h, buf, n, ctypes.byref(cnt))
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_get_params")
        return np.array(buf[:], dtype=np.float32)

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        rc = self._lib.pselinv_model_set_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                p.size)
        if rc != 0:
            raise PselinvError(rc, "pselinv_model_set_params")

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.pselinv_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode_records(records):
    """Network inputs (n x 16, float32) of tuning records (host computation)."""
    lib = load_library()
    arr = CostModel._recs(records)
    x = np.zeros((len(records), 16), dtype=np.float32)
    rc = lib.pselinv_model_encode(arr, len(records), x.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    if rc != 0:
        raise PselinvError(rc, "pselinv_model_encode")
    return x


def make_record(**kw):
    r = TuneRecord()
    for k, v in kw.items():
        if k == "feat":
            for i, f in enumerate(v):
                r.feat[i] = f
        else:
            setattr(r, k, v)
    return r


NOALLOC_MAX_S = 256


def _noalloc_args(lu_block, out, s):
    """Check the operands of block_inverse_noalloc before any pointer reaches
    the GPU; returns (s, dtype code).  Both must be contiguous CUDA tensors
    of one device and one dtype (float64 or complex128) holding at least
    s * s scalars each (column-major storage, leading dimension s)."""
    for name, t in (("lu_block", lu_block), ("out", out)):
        if not (hasattr(t, "is_cuda") and hasattr(t, "data_ptr")):
            raise TypeError(f"{name} must be a CUDA torch tensor, not {type(t).__name__}")
        if not t.is_cuda:
            raise ValueError(f"{name} must be on a CUDA device (got {t.device})")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    import torch
    if lu_block.dtype not in (torch.float64, torch.complex128):
        raise ValueError(f"lu_block must be float64 or complex128, not {lu_block.dtype}")
    if out.dtype != lu_block.dtype:
        raise ValueError(f"out has dtype {out.dtype}, lu_block {lu_block.dtype}")
    if out.device != lu_block.device:
        raise ValueError(f"out is on {out.device}, lu_block on {lu_block.device}")
    if s is None:
        if lu_block.dim() == 2 and lu_block.shape[0] == lu_block.shape[1]:
            s = int(lu_block.shape[0])
        elif lu_block.dim() == 1:
            r = int(np.sqrt(lu_block.numel()) + 0.5)
            if r * r != lu_block.numel():
                raise ValueError(f"a flat lu_block of {lu_block.numel()} scalars is not square; "
                                 "pass s")
            s = r
        else:
            raise ValueError(f"cannot infer s from shape {tuple(lu_block.shape)}; pass s")
    s = int(s)
    if not 1 <= s <= NOALLOC_MAX_S:
        raise ValueError(f"s = {s} outside 1..{NOALLOC_MAX_S}")
    for name, t in (("lu_block", lu_block), ("out", out)):
        if t.numel() < s * s:
            raise ValueError(f"{name} holds {t.numel()} scalars, fewer than s * s = {s * s}")
    return s, (C128 if lu_block.dtype == torch.complex128 else F64)


def block_inverse_noalloc(lu_block, out, s=None, stream=None):
    """(L U)^{-1} of an LU-factored s x s block (column-major device arrays)
    through the allocation-free entry point; see pselinv_block_inverse_noalloc.

    ``lu_block`` and ``out`` are contiguous CUDA tensors of the same device
    and dtype (float64 or complex128) with at least s * s scalars; ``s``
    defaults to the side of a square 2-D tensor or of a flat buffer whose
    length is a perfect square.  The call runs with the tensors' device
    current (the library requires that of its pointers)."""
    s, dt = _noalloc_args(lu_block, out, s)
    lib = load_library()
    import torch
    with torch.cuda.device(lu_block.device):
        rc = lib.pselinv_block_inverse_noalloc(dt, s, _ptr(lu_block), s, _ptr(out), s,
                                               _stream(stream))
    if rc != 0:
        raise PselinvError(rc, "pselinv_block_inverse_noalloc")
    return out


class InstanceGroup:
    """Several independent matrices of different patterns in one handle.

    The direct sum A_1 (+) A_2 (+) ... is block diagonal, its elimination tree
    is the forest of the instances' trees, and the depth levels of the sweep
    then hold supernodes of every instance: one factorisation and one
    selected inversion (one set of level launches) serve the whole group.
    The selected inverse of a block-diagonal matrix is the block diagonal of
    the selected inverses, so each instance's result is a slice of the
    group's.
    """

    def __init__(self, patterns, **kw):
        """patterns: list of (n, colptr, rowind, perm or None); the grouped
        handle is built by pselinv_group from host-only member analyses."""
        self.n = [int(p[0]) for p in patterns]
        self.nnz = [int(np.asarray(p[1])[-1]) for p in patterns]
        self.row_off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.nz_off = np.concatenate([[0], np.cumsum(self.nnz)]).astype(np.int64)
        mkw = {k: v for k, v in kw.items() if k in ("max_supernode", "relax_pct")}
        members = [SelInv(n, cp, ri, pm, host_only=True, **mkw) for (n, cp, ri, pm) in patterns]
        self.handle = SelInv.group(members, **kw)
        for m in members:
            m.close()
        self.colptr = self.handle._colptr
        self.rowind = self.handle._rowind

    def values(self, per_instance):
        """Concatenate the instances' CSC values (host arrays)."""
        return np.concatenate([np.asarray(v) for v in per_instance])

    def split(self, out):
        """Per-instance views of a pattern-of-A result of the group."""
        return [out[self.nz_off[i]:self.nz_off[i + 1]] for i in range(len(self.n))]


def order_nd(n, colptr, rowind, leaf=4):
    """Nested-dissection ordering (new -> old) of a structurally symmetric
    CSC pattern, computed on the host by ``pselinv_order_nd`` (small leaves
    dissect further and store less fill: 464k entries of L over the test
    graphs with leaf 4 against 572k with leaf 64)."""
    lib = load_library()
    cp = np.ascontiguousarray(colptr, dtype=np.int64)
    ri = np.ascontiguousarray(rowind, dtype=np.int64)
    perm = np.empty(int(n), dtype=np.int64)
    rc = lib.pselinv_order_nd(int(n), _ptr(cp), _ptr(ri), int(leaf), _ptr(perm))
    if rc != 0:
        raise PselinvError(rc, "pselinv_order_nd")
    return perm


def measure_fp64_peak(stream=None):
    """(TFLOP/s, ms) of the library's FP64 fused multiply-add loop on every SM
    of the current device (the FP64 roofline's denominator)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load_library().pselinv_measure_fp64_peak(_stream(stream), ctypes.byref(tf),
                                                  ctypes.byref(ms))
    if rc != 0:
        raise PselinvError(rc, "pselinv_measure_fp64_peak")
    return tf.value, ms.value


def wait_selftest(budget_us=20000, stream=None):
    """Status of the bounded-wait check (PSELINV_ERR_TIMEOUT = -6 expected)."""
    return int(load_library().pselinv_wait_selftest(_stream(stream), int(budget_us)))


def inverse_coordinates(st: dict):
    """(rows, cols) in permuted indices of the entry of Atilde^{-1} that every
    slot of the supernodal storage holds after pselinv_selinv.  Structurally
    symmetric handles: as supernodal_coordinates.  General handles (the
    pattern of (L+U)^T): diagonal block Ainv_KK, L panel (Ainv_{K,R_L})^T,
    U^T panel Ainv_{R_U,K}."""
    if not st.get("general", False):
        return supernodal_coordinates(st)
    total = int(st["storage_size"])
    rows = np.empty(total, dtype=np.int64)
    cols = np.empty(total, dtype=np.int64)
    for K in range(int(st["nsuper"])):
        f, s = int(st["sn_first"][K]), int(st["sn_width"][K])
        RL = st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]]
        RU = st["urows"][st["urows_ptr"][K]:st["urows_ptr"][K + 1]]
        o = int(st["sn_offset"][K])
        loc = np.arange(f, f + s)
        rows[o:o + s * s] = np.tile(loc, s)
        cols[o:o + s * s] = np.repeat(loc, s)
        o += s * s
        rows[o:o + RL.size * s] = np.repeat(loc, RL.size)
        cols[o:o + RL.size * s] = np.tile(RL, s)
        o += RL.size * s
        rows[o:o + RU.size * s] = np.tile(RU, s)
        cols[o:o + RU.size * s] = np.repeat(loc, RU.size)
    return rows, cols


def supernodal_coordinates(st: dict):
    """(rows, cols) in permuted indices of every slot of the supernodal storage
    of one instance (diagonal block, L panel, U^T panel per supernode)."""
    total = int(st["storage_size"])
    rows = np.empty(total, dtype=np.int64)
    cols = np.empty(total, dtype=np.int64)
    for K in range(int(st["nsuper"])):
        f, s = int(st["sn_first"][K]), int(st["sn_width"][K])
        R = st["rows"][st["rows_ptr"][K]:st["rows_ptr"][K + 1]]
        c = R.size
        o = int(st["sn_offset"][K])
        loc = np.arange(f, f + s)
        rows[o:o + s * s] = np.tile(loc, s)
        cols[o:o + s * s] = np.repeat(loc, s)
        o += s * s
        rows[o:o + c * s] = np.tile(R, s)
        cols[o:o + c * s] = np.repeat(loc, c)
        o += c * s
        rows[o:o + c * s] = np.repeat(loc, c)
        cols[o:o + c * s] = np.tile(R, s)
    return rows, cols
