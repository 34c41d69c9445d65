/*
 * pselinv -- supernodal selected inversion of a structurally symmetric,
 * non-symmetric sparse matrix on one NVIDIA GB300 (sm_103a).
 *
 * Method: Jacquelin, Lin, Yang, "PSelInv -- A distributed memory parallel
 * algorithm for selected inversion: the non-symmetric case" (Section 2,
 * Algorithm 1; Theorems 1 and 2).  Given A (n x n, CSC) and a symmetric
 * fill-reducing ordering P (P A P^T = Atilde), the library factors
 * Atilde = L U without pivoting (L unit lower, U upper; Eq. LU) and returns
 * every entry of A^{-1} on the pattern of L + U, by sweeping the
 * supernodal elimination tree from the roots to the leaves:
 *
 *   Lhat_{C,K} = L_{C,K} (L_{K,K})^{-1},  Uhat_{K,C} = (U_{K,K})^{-1} U_{K,C}  (Alg. 1 step 2)
 *   Ainv_{C,K} = -Ainv_{C,C} Lhat_{C,K}                                  (Alg. 1 step 3)
 *   Ainv_{K,K} = (U_{K,K})^{-1} (L_{K,K})^{-1} - Uhat_{K,C} Ainv_{C,K}   (Alg. 1 step 4)
 *   Ainv_{K,C} = -Uhat_{K,C} Ainv_{C,C}                                  (Alg. 1 step 5)
 *
 * written here in the non-transposed form (the paper stores A^{-T} in
 * place; transposing its steps 3-5 gives the lines above).  C is the row
 * structure R_K of supernode K (C_L = C_U for a structurally symmetric
 * pattern, Section 1).
 *
 * Conventions for every entry point
 *  - All functions return PSELINV_OK (0) or a negative PSELINV_ERR_* code;
 *    none exits or aborts.  pselinv_error_string() describes a code.
 *  - Index arrays are 0-based int64.  `perm` is new -> old: row/column
 *    perm[k] of A becomes row/column k of Atilde.
 *  - Input buffers are copied; the library never keeps a caller pointer.
 *    The handle owns all device memory it allocates (freed by pselinv_free).
 *    Output buffers belong to the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is ordered on that stream.
 *  - Value buffers may be host or device pointers (detected with
 *    cudaPointerGetAttributes); host buffers are copied through the stream.
 *  - Complex values (PSELINV_C128) are interleaved (re, im) doubles.
 */
#ifndef PSELINV_H
#define PSELINV_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pselinv_status {
  PSELINV_OK = 0,
  PSELINV_ERR_ARG = -1,            /* bad argument or call order */
  PSELINV_ERR_NOT_STRUCT_SYM = -2, /* pattern(A) != pattern(A^T) */
  PSELINV_ERR_ZERO_PIVOT = -3,     /* zero pivot; column in pselinv_last_info */
  PSELINV_ERR_OOM = -4,            /* host or device allocation failed */
  PSELINV_ERR_CUDA = -5,           /* a CUDA call failed */
  PSELINV_ERR_TIMEOUT = -6,        /* a bounded device wait gave up */
  PSELINV_ERR_CHECK = -7,          /* a checked index map read was out of range */
  PSELINV_ERR_UNSUPPORTED = -8     /* option not available for this dtype */
};

enum pselinv_dtype { PSELINV_F64 = 1, PSELINV_C128 = 2 };

enum pselinv_precision {
  PSELINV_PREC_FP64 = 0,      /* every product in FP64 */
  PSELINV_PREC_OZAKI_FP16 = 1 /* Ainv_CC products as sliced FP16 tensor-core GEMMs */
};

enum pselinv_schedule {
  PSELINV_SCHED_LEVEL = 0,         /* one batched launch per elimination-tree level */
  PSELINV_SCHED_PER_SUPERNODE = 1  /* separate launches for every supernode */
};

enum pselinv_layout {
  PSELINV_LAYOUT_PATTERN_A = 0,  /* nnz(A) values, CSC order of the input, original indices */
  PSELINV_LAYOUT_SUPERNODAL = 1, /* the whole supernodal storage of Ainv (see pselinv_structure) */
  PSELINV_LAYOUT_FACTORS = 2     /* the supernodal storage of the LU factors (same layout) */
};

typedef struct pselinv_opts {
  int32_t max_supernode; /* widest supernode (columns), 1..256; default 256 */
  int32_t relax_pct;     /* max share (%) of explicit zeros a relaxed supernode adds; default 20 */
  int32_t precision;     /* pselinv_precision used by pselinv_selinv when it is passed -1 */
  int32_t slices;        /* FP16 slices per operand for PREC_OZAKI_FP16; 0 = default */
  int32_t schedule;      /* pselinv_schedule; default PSELINV_SCHED_LEVEL */
  int32_t use_graph;     /* 1: record the selinv sweep once in a CUDA graph and replay it */
  int32_t check_level;   /* 1: bounds-check every index-map read on the device */
  int32_t host_only;     /* 1: pselinv_analyze makes no CUDA call (structure inspection only;
                            the handle then refuses pselinv_factor) */
  int32_t split_normalise; /* PREC_OZAKI_FP16 only.  0 (default): the normalisation (Lhat,
                            Uhat^T, Algorithm 1 step 2) and D_K = U_KK^{-1} L_KK^{-1} stay in
                            FP64 like the triangular inverses and the final Ainv_KK
                            combination; 1: in split levels they are sliced products too
                            (faster, one more rounding stage) */
  int32_t symmetric;     /* 1: the values satisfy A = A^T (real symmetric or complex
                            symmetric, not Hermitian).  Then Uhat = Lhat^T and
                            Ainv(K, C) = Ainv(C, K)^T: the sweep skips the normalisation
                            of U, step 5's product (a copy) and the column slicing of G
                            (the symmetric variant of Algorithm 1).  Not checked: values
                            that are not symmetric give a wrong result.  Default 0. */
  int32_t nd_leaf;       /* perm == NULL in pselinv_analyze: 0 (default) the natural order;
                            > 0 the nested-dissection ordering of pselinv_order_nd with
                            leaves of at most nd_leaf vertices (see the structure's perm) */
  int32_t factor_precision; /* PSELINV_PREC_FP64 (default) or PSELINV_PREC_OZAKI_FP16: the
                            panel solves L_{C,K} = A_{C,K} U_KK^{-1}, U_{K,C}^T =
                            A_{K,C}^T L_KK^{-T} and the Schur-complement products
                            L_{C,K} U_{K,C} of pselinv_factor as sliced FP16 tensor-core
                            products (exact FP32 accumulation, FP64 result) on the levels
                            whose Schur products reach factor_split_mflops; the diagonal
                            LU, the triangular inverses and the scatter into the
                            ancestors stay FP64 */
  int32_t factor_split_mflops; /* factor_precision = OZAKI_FP16: smallest Schur-product work
                            (MFLOP) of a level that goes split; 0 = default (200); < 0:
                            every level */
  int32_t ozaki_a_tmem;  /* sliced products: 0 (default) the MMAs read the A slices straight
                            from shared memory (each A tile once per slice pair); 1 from
                            tensor memory, copied there once per K half (tcgen05.cp; the
                            64-bit totals then live in shared memory).  The same exact
                            integer sums either way; 1 measured slower on GB300. */
  int32_t reserved[2];
} pselinv_opts;

typedef struct pselinv_ctx* pselinv_t;

/* Borrowed views of the symbolic structure (valid until pselinv_free).
 * Supernode K covers permuted columns [sn_first[K], sn_first[K] + sn_width[K]),
 * its row structure R_K = rows[rows_ptr[K] .. rows_ptr[K+1]) (sorted, > last
 * column), c_K = rows_ptr[K+1] - rows_ptr[K].  Its storage (one instance)
 * starts at element sn_offset[K]:
 *   diagonal block  s x s column-major (L_KK below, U_KK on/above the diagonal;
 *                   after selinv: Ainv_KK)
 *   L panel         c x s column-major at sn_offset[K] + s*s
 *                   (row p = R_K[p]; after selinv: Ainv_{R_K, K})
 *   U^T panel       c x s column-major at sn_offset[K] + s*s + c*s
 *                   (entry (p, t) = U_{first+t, R_K[p]}; after selinv:
 *                   (Ainv_{K, R_K})^T)
 * storage_size is the number of scalars of one instance. */
typedef struct pselinv_structure {
  int64_t n;
  int64_t nsuper;
  int64_t nlevels;             /* depth levels of the supernodal tree */
  int64_t storage_size;
  int64_t nnz_a;
  const int64_t* perm;         /* [n] new -> old */
  const int64_t* etree;        /* [n] column elimination tree of the exact fill, -1 = root */
  const int64_t* sn_first;     /* [nsuper] */
  const int64_t* sn_width;     /* [nsuper] */
  const int64_t* sn_parent;    /* [nsuper] -1 = root */
  const int64_t* sn_depth;     /* [nsuper] 0 = root */
  const int64_t* sn_offset;    /* [nsuper] */
  const int64_t* rows_ptr;     /* [nsuper + 1] */
  const int64_t* rows;         /* [rows_ptr[nsuper]] */
  const int64_t* level_ptr;    /* [nlevels + 1] supernodes of depth d: level_sn[level_ptr[d]..) */
  const int64_t* level_sn;     /* [nsuper] */
  const int64_t* value_map;    /* [nnz_a] storage slot of each entry of A (CSC order) */
  double flops_selinv;         /* sum_K 4 c^2 s + 4 c s^2 + 4/3 s^3 on this structure (real) */
  double flops_selinv_exact;   /* the same sum on the strict (relax 0) supernodes */
  double flops_factor;         /* sum_K 2 c^2 s + 2 c s^2 + 2/3 s^3 (real) */
  /* General patterns (handles of pselinv_analyze_general; for the others
   * general = 0, rperm = perm, urows = rows and out_map = value_map):
   * rows_ptr / rows hold R_L(K) (= C_L, the L panel's c_L rows) and
   * urows_ptr / urows R_U(K) (= C_U, the columns of U right of K, the c_U
   * rows of the U^T panel, which follows the L panel: at sn_offset[K] +
   * s*s + c_L*s).  After pselinv_selinv the diagonal block holds Ainv_KK,
   * the L panel (Ainv_{K,R_L})^T and the U^T panel Ainv_{R_U,K} (the
   * pattern of (L+U)^T, the paper's A^{-T} in place).  The c of the flop
   * counts is then sum_K 4 c_L c_U s + 2 (c_L + c_U) s^2 + 4/3 s^3; the
   * exact count is taken over the scalar structures.  etree[j] = first row
   * of C_L(j) (the tree of the L structures). */
  int64_t general;
  const int64_t* rperm;        /* [n] row ordering new -> old (general) */
  const int64_t* urows_ptr;    /* [nsuper + 1] */
  const int64_t* urows;        /* [urows_ptr[nsuper]] */
  const int64_t* out_map;      /* [nnz_a] storage slot of the selected entry returned for each
                                  input entry by PSELINV_LAYOUT_PATTERN_A */
} pselinv_structure;

/* Fill *opts with the defaults. */
void pselinv_default_opts(pselinv_opts* opts);

/* Symbolic analysis (host only; Section 2 supernodes, elimination tree):
 * checks pattern(A) = pattern(A^T) (a missing diagonal counts as present),
 * builds the elimination tree, the (relaxed, width-limited) supernodes, their
 * row structures, the supernodal tree and its levels, the block index maps
 * used by the device gathers/scatters, and uploads them.
 * n >= 0; colptr[n+1], rowind[nnz] host arrays, rows strictly increasing per
 * column; perm[n] host (NULL = identity, or with opts->nd_leaf > 0 the
 * nested-dissection ordering); opts NULL = defaults.
 * Needs a current CUDA device.  On success *out is a new handle. */
int pselinv_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                    const int64_t* perm, const pselinv_opts* opts, pselinv_t* out);

/* Symbolic analysis of a GENERAL pattern with static pivoting (Section 1:
 * non-symmetric matrices, Eq. sel_entries; Section 2: C_L != C_U in
 * Theorem 1 and Algorithm 1; Theorem 2 with P != Q^T).  Atilde = P A Q with
 * Atilde(i, k) = A(rperm[i], cperm[k]); rperm, cperm: host int64 new -> old
 * (NULL = identity), typically a fill-reducing column ordering and a row
 * permutation that puts large entries on the diagonal (static pivoting; the
 * library computes neither).  The pattern need not be structurally
 * symmetric; the diagonal of Atilde counts as present.  The LU factors of
 * Atilde are formed without pivoting on the structures C_L(k), C_U(k) of
 * the fill rule (eliminating k fills C_L(k) x C_U(k)), supernodes join
 * columns whose diagonal block is connected (relax_pct as for
 * pselinv_analyze), and the two supernodal row structures R_L(K), R_U(K)
 * are closed under the supernodal updates.  The depth levels of the sweep
 * follow the dependencies of Theorem 1 (K after every supernode of R_L(K)
 * and R_U(K)).  Results: pselinv_get_selected(PATTERN_A) returns, for
 * entry p of A at row y = rowind[p] of column x, the selected entry
 * (A^{-1})_{x,y} (Eq. sel_entries: the transposed position), and
 * pselinv_trace / pselinv_weighted_sum use the same entries.  Both
 * precisions are available; with PSELINV_PREC_OZAKI_FP16 the normalisation
 * stays FP64 (opts->split_normalise is ignored) and G_K = Ainv(R_U, R_L) is
 * gathered and sliced for steps 3 and 5 as for the other handles.
 * opts->symmetric must be 0; pselinv_group, pselinv_partition and the block
 * transfers return PSELINV_ERR_UNSUPPORTED for these handles.  Other errors
 * as pselinv_analyze (PSELINV_ERR_ARG for an invalid ordering or pattern). */
int pselinv_analyze_general(int64_t n, const int64_t* colptr, const int64_t* rowind,
                            const int64_t* rperm, const int64_t* cperm, const pselinv_opts* opts,
                            pselinv_t* out);

/* Fill-reducing ordering for pselinv_analyze (host only; not from the
 * paper, which orders with graph partitioners): automatic nested dissection
 * of the graph of A after George and Liu (1981), separators from the level
 * structures of pseudo-peripheral vertices, each separator ordered after
 * the two parts it separates, parts of at most `leaf` vertices (leaf >= 1)
 * in breadth-first order.  colptr/rowind: the CSC pattern as for
 * pselinv_analyze (must equal its transpose; the diagonal is ignored).
 * perm_out[n] (host, caller-owned): new -> old.  Errors: PSELINV_ERR_ARG
 * (bad pattern, leaf < 1, null pointer), PSELINV_ERR_NOT_STRUCT_SYM,
 * PSELINV_ERR_OOM. */
int pselinv_order_nd(int64_t n, const int64_t* colptr, const int64_t* rowind, int64_t leaf,
                     int64_t* perm_out);

/* One handle for several independent matrices of DIFFERENT patterns
 * (instances of uneven size; not from the paper, whose method takes one
 * matrix: the batching of Algorithm 1 over many matrices).  The group's
 * matrix is the direct sum A_1 (+) A_2 (+) ... (+) A_count of the members'
 * patterns in member order: member m's rows and columns are shifted by the
 * sizes of the members before it, and so is its ordering (the structure's
 * perm), so the group's elimination forest is the union of the members'
 * trees and every depth level of the sweep holds the supernodes of every
 * member (one launch per kernel kind and level for all of them).  The
 * selected inverse of a block-diagonal matrix is block diagonal, so each
 * member's result is its slice of the group's.
 *   members[count]: analysed handles (host_only ones too); they are only
 *     read, stay valid and are freed by the caller as usual.
 *   opts: NULL = the first member's options (with host_only off).
 * pselinv_factor of the group takes the members' CSC values concatenated in
 * member order (member m's entries at the sum of the earlier members' nnz);
 * pselinv_get_selected(PATTERN_A) returns the same concatenation, whose
 * slice m is (A_m^{-1}) on member m's pattern.  Errors as pselinv_analyze. */
int pselinv_group(const pselinv_t* members, int64_t count, const pselinv_opts* opts,
                  pselinv_t* out);

/* Supernodal LU without pivoting of nbatch instances sharing the pattern
 * (Eq. LU, Section 3's prerequisite).  values: nbatch * nnz scalars of dtype,
 * instance b at values + b*nnz, in the CSC order given to pselinv_analyze;
 * host or device.  Runs on `stream` and waits for it to report a zero pivot
 * (PSELINV_ERR_ZERO_PIVOT; pselinv_last_info gives the permuted column).
 * The panel solves and Schur products are FP64, or sliced tensor-core
 * products per opts.factor_precision (pselinv_set_factor_precision).  For a
 * handle with opts.symmetric the Schur complements L_{C,K} U_{K,C} are
 * symmetric: only their lower triangles are formed and scattered, U's panels
 * are solved from L's, and the factors are the same L and U. */
int pselinv_factor(pselinv_t h, int dtype, int64_t nbatch, const void* values, void* stream);

/* Selected inversion of every factored instance (Algorithm 1 steps 2-5):
 * precision = pselinv_precision or -1 for the handle's option.  Asynchronous
 * on `stream`. */
int pselinv_selinv(pselinv_t h, int precision, void* stream);

/* Partitioned sweep over several GPUs (not from the paper, whose parallel
 * design distributes every supernode's blocks over a process grid; here
 * whole subtrees go to a rank).  The subtrees below the top of the
 * supernodal tree are independent once the selected inverse of the top is
 * known: a supernode K below a subtree root r reads Ainv only inside the
 * subtree and at R_r x R_r (R_K minus the subtree lies in R_r), so the top
 * is computed once and each subtree root's G_r = Ainv(R_r, R_r) is sent to
 * the rank that owns it, in one exchange step.
 *   partition: owner[nsuper] (host, caller-owned) = the rank of every
 *     supernode, -1 for the top.  The heaviest subtree (by the flops of its
 *     supernodes) is split into its children until there are about eight
 *     subtrees per rank, then subtrees go to ranks heaviest first, each to
 *     the least loaded rank.  nranks = 1: no top.
 *   set_subset: later pselinv_selinv / pselinv_tune calls cover only the
 *     supernodes with owner[K] == rank (owner NULL: all again); plans are
 *     rebuilt.  Host only.
 *   export_block: buf (device, c_K x c_K column-major, caller-owned) =
 *     G_K = Ainv(R_K, R_K) of instance `batch`, gathered from the handle's
 *     selected inverse; import_block writes such a block into the handle's
 *     storage (the blocks of R_K's supernodes), as a rank does with the
 *     G_r it receives before sweeping its subtrees.  Both synchronise
 *     `stream`.
 * Structurally symmetric handles only (PSELINV_ERR_UNSUPPORTED for general
 * patterns, whose dependencies are not a tree); PSELINV_ERR_ARG for bad
 * arguments or a host `buf`. */
int pselinv_partition(pselinv_t h, int32_t nranks, int32_t* owner);
int pselinv_set_subset(pselinv_t h, const int32_t* owner, int32_t rank);
int pselinv_export_block(pselinv_t h, int64_t K, int64_t batch, void* buf, void* stream);
int pselinv_import_block(pselinv_t h, int64_t K, int64_t batch, const void* buf, void* stream);

/* Schedule of later pselinv_selinv / pselinv_tune calls (the handle's
 * opts.schedule): PSELINV_SCHED_LEVEL (one batched launch per kind and
 * depth level, the priority list of Section 3.3 as levels) or
 * PSELINV_SCHED_PER_SUPERNODE (the same products launched supernode by
 * supernode, for comparison).  The plan of each schedule is built on its
 * first use and kept.  Host only. */
int pselinv_set_schedule(pselinv_t h, int schedule);

/* Precision of the Schur-complement products of later pselinv_factor calls
 * (the handle's opts.factor_precision and opts.factor_split_mflops, see
 * pselinv_opts): PSELINV_PREC_FP64 or PSELINV_PREC_OZAKI_FP16.  The
 * factorisation plan is rebuilt on the next pselinv_factor; results already
 * computed are kept.  Host only. */
int pselinv_set_factor_precision(pselinv_t h, int precision, int32_t split_mflops);

/* Copy results of instance `batch` (Algorithm 1 step 6 and Theorem 2 for
 * PSELINV_LAYOUT_PATTERN_A: out[p] = (A^{-1})_{rowind[p], j} for entry p of
 * column j of the input; PSELINV_LAYOUT_SUPERNODAL: storage_size scalars of
 * Ainv; PSELINV_LAYOUT_FACTORS: storage_size scalars of L and U, available
 * after pselinv_factor).  out: host or device.  For a host `out` the call
 * waits for the stream. */
int pselinv_get_selected(pselinv_t h, int layout, int64_t batch, void* out, void* stream);

/* Borrowed views of the structure; valid until pselinv_free. */
int pselinv_get_structure(pselinv_t h, pselinv_structure* out);

/* Per-launch record of pselinv_profile. */
typedef struct pselinv_step_stat {
  int32_t kind;   /* pselinv_step_kind */
  int32_t level;  /* tree level of the launch, -1 for whole-tree launches */
  int64_t tasks;  /* work items (tiles, supernodes, segments) */
  double flops;   /* useful floating-point operations (real) */
  double bytes;   /* algorithmic bytes moved (operands read + results written) */
  double ms;      /* device time from CUDA events around the launch */
  int32_t param;  /* GEMM: kernel config (0 64x64, 1 32x32, 2 128x64 tiles, 3 row
                     panels); OZAKI_GEMM: K split;
                     TRI_INV: 0 wide blocks (a warp per column), 1 blocks <= 32 wide;
                     else -1 */
  int32_t side;   /* stream of the launch in a sweep: 0 main, 1 normalisation side stream,
                     2 third stream (triangular inverses of the deeper levels) */
  double start_ms; /* which = 2: time from the start of the sweep until the launch's stream
                      reached it (its wait included); else 0 */
} pselinv_step_stat;

enum pselinv_step_kind {
  PSELINV_STEP_GEMM = 0, PSELINV_STEP_TRI_INV = 1, PSELINV_STEP_DIAG_LU = 2,
  PSELINV_STEP_GATHER = 3, PSELINV_STEP_SCATTER_SUB = 4, PSELINV_STEP_COPY = 5,
  PSELINV_STEP_MEMSET = 6, PSELINV_STEP_SCATTER_VALUES = 7, PSELINV_STEP_SLICE = 8,
  PSELINV_STEP_OZAKI_GEMM = 9, PSELINV_STEP_RECOMBINE = 10,
  PSELINV_STEP_SMALL_LEVEL = 11, /* steps 3-5 of a level of narrow supernodes, one launch */
  PSELINV_STEP_GATHER_SLICE = 12, /* split levels: Ainv_CC gathered and sliced in one pass
                                     (slices in both layouts, exponents from the running
                                     maxima), with the panels' maxima or slicing; Ainv_CC is
                                     never stored in FP64 */
  PSELINV_STEP_OUTPUT_MAXIMA = 13 /* split sweeps: the running row and column maxima of
                                     |Ainv| merged with a level's finished blocks; they
                                     bound the rows and columns of every later Ainv_CC */
};

/* Run the selected-inversion plan (which = 0) or the factorisation plan
 * (which = 1) launch by launch, outside any graph and on `stream` alone,
 * with CUDA events around every launch, and report up to `cap` records in
 * out[] (*count = number of launches).  which = 2: a timeline of the
 * selected-inversion plan run on its own streams (normalisation overlapped
 * as in pselinv_selinv, no graph): ms is each launch's span on its stream
 * and start_ms when its stream reached it.  The results are the same as
 * pselinv_selinv / pselinv_factor produce.  Synchronises `stream`. */
int pselinv_profile(pselinv_t h, int which, void* stream, pselinv_step_stat* out, int64_t cap,
                    int64_t* count);

/* Number of kernel launches one pselinv_selinv and one pselinv_factor issue
 * with the current plans (0 if not built yet).  Runtime memsets of the plan
 * are not kernels of the library and are not counted. */
int pselinv_plan_stats(pselinv_t h, int64_t* launches_selinv, int64_t* launches_factor);

/* Allocation-free inverse of one LU-factored diagonal block (the paper has
 * no counterpart; it serves callers that cannot allocate device memory, such
 * as code running while a framework's caching allocator owns the device, or
 * code that must avoid the device-wide synchronisation of cudaMalloc and
 * cudaFree).
 *   inv_out = (L U)^{-1} = U^{-1} L^{-1}, where lu_block (s x s, column-major,
 *   leading dimension ld_in) holds L unit lower below the diagonal and U on
 *   and above it -- the layout of a diagonal block of
 *   PSELINV_LAYOUT_FACTORS.  inv_out: s x s, leading dimension ld_out.
 * Both pointers are device memory of the CURRENT device, owned by the
 * caller, and `stream` belongs to that device; a pointer that is host
 * memory or lives on another device returns PSELINV_ERR_ARG before any
 * launch (checked with cudaPointerGetAttributes).  dtype is PSELINV_F64 or
 * PSELINV_C128; 1 <= s <= PSELINV_NOALLOC_MAX_S (larger s returns
 * PSELINV_ERR_ARG).  The call allocates nothing: the two triangular inverses
 * are kept in a 2 MiB array compiled into the library, which every GPU that
 * loads the library holds until the process exits.  The first call on a
 * device looks up that array's address (with the device current) and keeps
 * it, so make that call before any stream capture, and do not use the entry
 * point on a device after cudaDeviceReset of that device.  All calls share
 * the array: calls that overlap on the GPU race and must be serialised by
 * the caller.  Work is queued on `stream`; a zero pivot in U gives
 * non-finite output and is not reported. */
#define PSELINV_NOALLOC_MAX_S 256
int pselinv_block_inverse_noalloc(int dtype, int64_t s, const void* lu_block, int64_t ld_in,
                                  void* inv_out, int64_t ld_out, void* stream);

/* One measurement of the autotuner; also the training data of the learned
 * cost model.  Not from the paper: tile shapes and K splits are the GPU
 * batching parameters of the level sweep. */
typedef struct pselinv_tune_record {
  int32_t precision; /* pselinv_precision of the plan */
  int32_t level;     /* tree level of the launch (-1 = normalisation) */
  int32_t slot;      /* 0 normalisation, 1 steps 3 and 5, 2 step 4 */
  int32_t kind;      /* PSELINV_STEP_GEMM (param = kernel config 0..3: 64x64, 32x32,
                        128x64 tiles, row panels)
                        or PSELINV_STEP_OZAKI_GEMM (param = K split 1..16) */
  int32_t param;     /* the candidate timed */
  int32_t chosen;    /* 1 for the candidate the tuner kept */
  float feat[8];     /* log2(1 + x) of: products, flops, max M, max N, max K, mean M, N, K */
  double ms;         /* device time of the launch (CUDA events) */
} pselinv_tune_record;

enum pselinv_tune_mode {
  PSELINV_TUNE_RESET = 0,      /* back to the built-in heuristic */
  PSELINV_TUNE_EXHAUSTIVE = 1, /* time every candidate of every tunable launch, keep the best */
  PSELINV_TUNE_MODEL = 2       /* pick candidates with a trained cost model (no timing) */
};

/* Autotune the selected-inversion plan of `precision` for the factored
 * instances (Algorithm 1's products are unchanged; only launch shapes
 * change).  EXHAUSTIVE runs the plan once per candidate with CUDA events
 * around every launch (the results it leaves are valid); MODEL needs
 * `model` (see pselinv_model_*).  Synchronises `stream`. */
typedef struct pselinv_model* pselinv_model_t;
int pselinv_tune(pselinv_t h, int precision, int mode, pselinv_model_t model, void* stream);

/* Learned cost model of the launch shapes (not from the paper): an MLP
 *   x (16) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> w3 . h2 + b3
 * predicting log(ms) of a launch.  Input x of a record: feat[0..7] / 32;
 * [8] kind is GEMM; [9] kind is OZAKI_GEMM; [10..12] one-hot GEMM tile config
 * 0..2 (all zero for config 3, the row panels);
 * [13] log2(K split) / 4 for OZAKI_GEMM; [14] slot / 2; [15] precision.
 * Parameters (float32, flat): W1 (H x 16, row-major), b1 (H), W2 (H x H),
 * b2 (H), w3 (H), b3 (1).  Weights live on the current device; training and
 * inference run there (one single-CTA kernel runs all epochs of full-batch
 * Adam on the mean squared error of log(ms)).
 * create: hidden in [1, 64], Glorot-uniform weights from SplitMix64(seed).
 * train: n >= 1 records (their ms are the targets), epochs >= 1, lr > 0;
 *   *final_loss (nullable) = loss of the last epoch's forward pass.
 * gradients: gradient of the loss (same layout as the parameters) without
 *   updating them; *loss_out (nullable) = the loss.
 * predict: pred_ms[i] = exp(network(record i)) (record ms ignored).
 * get/set_params: copy the flat parameters out / in (set also clears Adam).
 * encode: the network input of each record (16 floats per record, host).
 * All synchronise `stream` and return PSELINV_* codes. */
int pselinv_model_create(int32_t hidden, uint64_t seed, pselinv_model_t* out);
int pselinv_model_train(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n,
                        int32_t epochs, float lr, void* stream, float* final_loss);
int pselinv_model_gradients(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n,
                            float* grad_out, float* loss_out, void* stream);
int pselinv_model_predict(pselinv_model_t m, const pselinv_tune_record* recs, int64_t n,
                          double* pred_ms, void* stream);
int pselinv_model_get_params(pselinv_model_t m, float* out, int64_t cap, int64_t* count);
int pselinv_model_set_params(pselinv_model_t m, const float* in, int64_t count);
int pselinv_model_encode(const pselinv_tune_record* recs, int64_t n, float* x_out);
void pselinv_model_free(pselinv_model_t m);

/* The records of the last exhaustive tuning (*count = number of records;
 * up to cap are copied). */
int pselinv_tune_records(pselinv_t h, pselinv_tune_record* out, int64_t cap, int64_t* count);

/* The tuned launch shapes of the plan of `precision`, as (level, slot,
 * value) triples of int32 (not from the paper; a tuning cache, so that a
 * plan tuned once can be replayed in another process).  Slots: 0
 * normalisation GEMM kernel config (0..3: 64x64, 32x32, 128x64 tiles, row
 * panels); FP64 plan: 1 steps 3+5, 2 step 4 kernel config (0..3); split
 * plan: 1 steps 3+5, 2 step 4 K split (1, 2, 4, 8 or 16), 3 level precision
 * (0 split products, 1 FP64), 4 / 5 kernel config of the FP64 launches of
 * steps 3+5 / step 4 (an FP64 level of narrow supernodes may run as one
 * fused launch instead, PSELINV_STEP_SMALL_LEVEL).  Levels are depth levels
 * (0 = roots), up to the structure's level count.
 * get: *count = number of triples; up to cap are written to out[3 * cap].
 * set: replaces all tuned values of `precision` (count = 0 restores the
 *   built-in heuristic); the next pselinv_selinv rebuilds the plan.  An
 *   out-of-range triple returns PSELINV_ERR_ARG and changes nothing.
 *   Host-only: queues no GPU work. */
int pselinv_plan_get(pselinv_t h, int precision, int32_t* out, int64_t cap, int64_t* count);
int pselinv_plan_set(pselinv_t h, int precision, const int32_t* in, int64_t count);

/* The same tuned values as a cache file at `path` (host only): save writes
 * a header naming the precision and the structure (n, supernodes, levels)
 * and the triples; load reads it back into the handle as pselinv_plan_set
 * does.  Errors: PSELINV_ERR_ARG for a path that cannot be opened, a file
 * not in this format, a file saved for another precision or structure, or
 * a triple out of range (the handle's values are then unchanged). */
int pselinv_plan_save(pselinv_t h, int precision, const char* path);
int pselinv_plan_load(pselinv_t h, int precision, const char* path);

/* Pole-expansion consumers of a batch of selected inverses (the use of
 * selected inversion that motivates the method, Section 1: a density matrix
 * or an observable as a weighted sum over shifted matrices).  weights: host
 * array of nbatch scalars of the factored dtype (w_l; complex: interleaved).
 * Require pselinv_selinv to have run.
 *   weighted_sum: out[p] = sum_l w_l (A_l^{-1})_{rowind[p], j} for entry p of
 *     column j of the input pattern (CSC order; out: host or device, nnz
 *     scalars).
 *   trace: *out = sum_l w_l Tr[B A_l^{-1}] = sum_l w_l sum_p B[p] (A_l^{-1})_{j, rowind[p]}
 *     for B on the input pattern (B: nnz scalars in CSC order, host or
 *     device; out: one scalar, host or device).  The reduction runs in a
 *     fixed order (the result does not depend on timing).
 * Host output waits for the stream. */
int pselinv_weighted_sum(pselinv_t h, const void* weights, void* out, void* stream);
int pselinv_trace(pselinv_t h, const void* weights, const void* B, void* out, void* stream);

/* Exercise the bounded-wait failure path (not from the paper): launch a
 * kernel whose only wait (on a tensor-core completion barrier) can never
 * complete, with a budget of budget_us microseconds (1 .. 2e6).  Every wait
 * in the library is bounded the same way (2 s): it records a timeout status
 * and the kernel returns instead of hanging.  Returns PSELINV_ERR_TIMEOUT
 * when the timeout was detected and reported to the host (the expected
 * result), PSELINV_OK if it was not. */
int pselinv_wait_selftest(void* stream, int64_t budget_us);

/* FP64 peak of the current device, measured (not from the paper; the
 * denominator of the FP64 roofline that the products, normalisation and
 * factorisation kernels are reported against): one launch of a loop of
 * fused multiply-adds, eight independent chains per thread and eight CTAs
 * of 256 threads per SM, timed with CUDA events on `stream` after a shorter
 * warm-up launch.  *tflops = FP64 TFLOP/s (2 flops per FMA); *ms (nullable)
 * = the timed launch's duration.  Allocates and frees a small device
 * buffer; synchronises `stream`. */
int pselinv_measure_fp64_peak(void* stream, double* tflops, double* ms);

/* Wait for `stream` and report a device-side error recorded by earlier calls. */
int pselinv_sync(pselinv_t h, void* stream);

/* Extra information about the last error (zero-pivot column, ...), or -1. */
int64_t pselinv_last_info(pselinv_t h);

const char* pselinv_error_string(int status);

/* Release the handle and all its device memory (NULL is a no-op). */
void pselinv_free(pselinv_t h);

#ifdef __cplusplus
}
#endif
#endif
