/*
 * CPU oracle for selected inversion of a structurally symmetric sparse
 * matrix (Jacquelin, Lin, Yang: "PSelInv -- A distributed memory parallel
 * algorithm for selected inversion: the non-symmetric case").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the independent checker of the
 * CUDA library: only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code with the CUDA path.
 *
 * It is deliberately scalar and column-by-column (Section 2, Theorem 1), the
 * plainest statement of what the supernodal GPU path computes:
 *
 *   analyze  : symmetric ordering P A P^T, elimination tree parent(j) =
 *              min{i > j : L_ij != 0}, column structures
 *              struct(j) = {i > j : L_ij != 0}, supernodes (Section 2,
 *              supernode definition, width-limited), supernodal tree, depths.
 *   lu       : scalar LU without pivoting, A = L U, L unit lower (Eq. LU).
 *   selinv   : Theorem 1, Eqs. selinv_1 and selinv_2, for k = n-1 .. 0.
 *   extract  : Theorem 2 (A^{-1} = Q Atilde^{-1} P, here with P = Q^T).
 *   dd inverse: dense Gauss-Jordan inverse with partial pivoting in
 *              double-double arithmetic (Dekker / Knuth error-free
 *              transformations), used to pin the selected inverse on tiny
 *              inputs.
 *
 * Storage of anything "on the pattern of L+U" (permuted indices), for column
 * j with struct(j) = sidx[sptr[j] .. sptr[j+1]):
 *   lower[p] = X_{sidx[p], j}   (column j below the diagonal)
 *   upper[p] = X_{j, sidx[p]}   (row j right of the diagonal)
 *   diag[j]  = X_{j, j}
 * Complex values are C99 double _Complex (interleaved re, im).
 *
 * Every function returns 0 on success or a negative error code; nothing
 * exits or aborts.
 */
#ifndef PSELINV_ORACLE_H
#define PSELINV_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_ARG = -1,
  ORACLE_ERR_NOT_STRUCT_SYM = -2,
  ORACLE_ERR_ZERO_PIVOT = -3,
  ORACLE_ERR_OOM = -4,
  ORACLE_ERR_SINGULAR = -5
};

typedef struct oracle_sym oracle_sym;

/* Symbolic analysis.  colptr[n+1], rowind[nnz]: CSC pattern (0-based, rows
 * strictly increasing per column).  perm[n]: new -> old (NULL = identity).
 * max_sn >= 1 limits the supernode width; relax_pct in [0, 100] is the
 * largest share (percent) of explicit zeros a relaxed supernode may add
 * (0 = the strict definition).  With relax_pct > 0 the per-column
 * structures returned (sptr/sidx) are those of the relaxed supernodes,
 * struct'(i) = (i, l] U R_K for column i of supernode K = [f, l]; the
 * etree (parent) is always that of the exact filled pattern. */
int oracle_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                   const int64_t* perm, int64_t max_sn, int64_t relax_pct, oracle_sym** out);
void oracle_sym_free(oracle_sym* s);

int64_t oracle_sym_n(const oracle_sym* s);
int64_t oracle_sym_nnzl(const oracle_sym* s);        /* sum_j |struct(j)| */
int64_t oracle_sym_nsup(const oracle_sym* s);
const int64_t* oracle_sym_parent(const oracle_sym* s);     /* [n]   column etree, -1 = root */
const int64_t* oracle_sym_sptr(const oracle_sym* s);       /* [n+1] */
const int64_t* oracle_sym_sidx(const oracle_sym* s);       /* [nnzl] sorted rows per column */
const int64_t* oracle_sym_supptr(const oracle_sym* s);     /* [nsup+1] first column of each supernode */
const int64_t* oracle_sym_sup_parent(const oracle_sym* s); /* [nsup] -1 = root */
const int64_t* oracle_sym_sup_depth(const oracle_sym* s);  /* [nsup] 0 = root */

/* Scalar LU, no pivoting.  values: CSC values of the ORIGINAL matrix.
 * On a zero pivot returns ORACLE_ERR_ZERO_PIVOT and *bad_col = column. */
int oracle_lu_d(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                const double* values, double* Llow, double* Uup, double* Udiag,
                int64_t* bad_col);
int oracle_lu_z(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                const void* values, void* Llow, void* Uup, void* Udiag, int64_t* bad_col);

/* Selected inverse B = A^{-1} on the pattern of L+U (permuted indices) from
 * the factors of oracle_lu_*.  `mutation` must be 0 except in the tests that
 * show the pins catch planted mistakes:
 *   1 drop the last term of each sum of Eq. selinv_1
 *   2 flip the sign of the correction in Eq. selinv_2
 *   3 transpose the gathered operand in Eq. selinv_1 (B_ji for B_ij)
 *   4 skip the normalisation U_kk^{-1} of the row of U
 *   5 use the column of L in place of the row of U in the B_kj sums */
int oracle_selinv_d(const oracle_sym* s, const double* Llow, const double* Uup,
                    const double* Udiag, double* Blow, double* Bup, double* Bdiag,
                    int mutation);
int oracle_selinv_z(const oracle_sym* s, const void* Llow, const void* Uup,
                    const void* Udiag, void* Blow, void* Bup, void* Bdiag, int mutation);
/* The same, with the columns of one depth of the structures' tree (roots
 * first; they never read each other's entries) run by nthreads OpenMP
 * threads; bit for bit the result of oracle_selinv_* (no mutations). */
int oracle_selinv_par_d(const oracle_sym* s, const double* Llow, const double* Uup,
                        const double* Udiag, double* Blow, double* Bup, double* Bdiag,
                        int nthreads);
int oracle_selinv_par_z(const oracle_sym* s, const void* Llow, const void* Uup,
                        const void* Udiag, void* Blow, void* Bup, void* Bdiag, int nthreads);

/* ---------------------------------------------------------------------
 * General patterns and static pivoting (oracle_general.c): Atilde = P A Q
 * with rperm (new -> old rows) and cperm (new -> old columns), NULL =
 * identity; C_L(k) and C_U(k) need not agree.  Factors and inverse are
 * stored column k of L (rows lidx[lptr[k]..lptr[k+1]) = C_L(k)) and row k
 * of U (columns uidx[uptr[k]..uptr[k+1]) = C_U(k)):
 *   L[p] = L_{lidx[p],k}, U[p] = U_{k,uidx[p]}, D[k] = U_{k,k};
 *   BL[p] = (Atilde^{-1})_{k,lidx[p]}, BU[p] = (Atilde^{-1})_{uidx[p],k},
 *   BD[k] = (Atilde^{-1})_{k,k}   (the pattern of (L+U)^T).
 * gextract: out[p] = (A^{-1})_{x,y} for entry p of A at row y, column x
 * (Eq. sel_entries, Theorem 2).  gselinv mutations 1-4 plant mistakes
 * (see oracle_gnum.inc).
 * --------------------------------------------------------------------- */
typedef struct oracle_gsym oracle_gsym;
int oracle_ganalyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                    const int64_t* rperm, const int64_t* cperm, oracle_gsym** out);
void oracle_gsym_free(oracle_gsym* s);
int64_t oracle_gsym_n(const oracle_gsym* s);
int64_t oracle_gsym_nnzl(const oracle_gsym* s);
int64_t oracle_gsym_nnzu(const oracle_gsym* s);
const int64_t* oracle_gsym_lptr(const oracle_gsym* s);
const int64_t* oracle_gsym_lidx(const oracle_gsym* s);
const int64_t* oracle_gsym_uptr(const oracle_gsym* s);
const int64_t* oracle_gsym_uidx(const oracle_gsym* s);
int oracle_glu_d(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                 const double* values, double* L, double* U, double* D, int64_t* bad_col);
int oracle_glu_z(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                 const void* values, void* L, void* U, void* D, int64_t* bad_col);
int oracle_gselinv_d(const oracle_gsym* s, const double* L, const double* U, const double* D,
                     double* BL, double* BU, double* BD, int mutation);
int oracle_gselinv_z(const oracle_gsym* s, const void* L, const void* U, const void* D,
                     void* BL, void* BU, void* BD, int mutation);
int oracle_gextract_d(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                      const double* BL, const double* BU, const double* BD, double* out);
int oracle_gextract_z(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                      const void* BL, const void* BU, const void* BD, void* out);

/* Selected entries in the ORIGINAL ordering on the pattern of A (Theorem 2):
 * out[p] = (A^{-1})_{rowind[p], j} for p in column j. */
int oracle_extract_d(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                     const double* Blow, const double* Bup, const double* Bdiag, double* out);
int oracle_extract_z(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                     const void* Blow, const void* Bup, const void* Bdiag, void* out);

/* Dense inverse of a real n x n column-major matrix in double-double
 * arithmetic (Gauss-Jordan, partial pivoting).  inv = inv_hi + inv_lo. */
int oracle_dense_inverse_dd(int64_t n, const double* a, double* inv_hi, double* inv_lo);

#ifdef __cplusplus
}
#endif
#endif
