/*
 * CPU oracle for selected inversion of a GENERAL sparse matrix: pattern not
 * structurally symmetric, static pivoting P A Q with P != Q^T (Section 2:
 * index sets C_L and C_U of Theorem 1 may differ; Algorithm 1; Theorem 2).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Scalar, column by column:
 *
 *   ganalyze : Atilde = P A Q (rperm: new -> old rows, cperm: new -> old
 *              columns).  Structures of the LU factors without pivoting by
 *              the fill rule of Gaussian elimination: eliminating k fills
 *              every (i, m) with i in C_L(k), m in C_U(k), so
 *                C_L(k) = {i > k : Atilde_ik != 0}
 *                         U {i > k : i in C_L(j), k in C_U(j), j < k}
 *                C_U(k) = {m > k : Atilde_km != 0}
 *                         U {m > k : k in C_L(j), m in C_U(j), j < k}.
 *              The diagonal counts as present.
 *   glu      : scalar right-looking LU over that pattern, L unit lower.
 *   gselinv  : Theorem 1 for k = n-1 .. 0 with C_L = C_L(k), C_U = C_U(k):
 *                B_{i,k} = - sum_{j in C_L} B_{i,j} L_{j,k},      i in C_U
 *                B_{k,j} = - sum_{i in C_U} Uhat_{k,i} B_{i,j},   j in C_L
 *                B_{k,k} = 1 / U_{k,k} - sum_{i in C_U} Uhat_{k,i} B_{i,k}
 *              with Uhat_{k,i} = U_{k,i} / U_{k,k}; every B_{i,j} read lies
 *              on the pattern of (L+U)^T (the fill argument of the proof).
 *   gextract : Theorem 2, A^{-1} = Q Atilde^{-1} P:
 *              (A^{-1})_{x,y} = (Atilde^{-1})_{icperm[x], irperm[y]}; for
 *              every entry A_{y,x} of A the selected entry (A^{-1})_{x,y}
 *              (Eq. sel_entries) is returned.
 *
 * Storage on the pattern of L+U (permuted indices), column k of L with rows
 * lidx[lptr[k] .. lptr[k+1]) = C_L(k) and row k of U with columns
 * uidx[uptr[k] .. uptr[k+1]) = C_U(k), both sorted:
 *   factors: L[p] = L_{lidx[p], k}, U[p] = U_{k, uidx[p]}, D[k] = U_{k,k}
 *   inverse (on the pattern of (L+U)^T, the paper's A^{-T} in place):
 *            BL[p] = B_{k, lidx[p]}, BU[p] = B_{uidx[p], k}, BD[k] = B_{k,k}
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

struct oracle_gsym {
  int64_t n;
  int64_t *rperm, *cperm, *irperm, *icperm;
  int64_t *lptr, *lidx, *uptr, *uidx;
  int64_t nnzl, nnzu;
};

void oracle_gsym_free(oracle_gsym* s) {
  if (!s) return;
  free(s->rperm);
  free(s->cperm);
  free(s->irperm);
  free(s->icperm);
  free(s->lptr);
  free(s->lidx);
  free(s->uptr);
  free(s->uidx);
  free(s);
}

int64_t oracle_gsym_n(const oracle_gsym* s) { return s->n; }
int64_t oracle_gsym_nnzl(const oracle_gsym* s) { return s->nnzl; }
int64_t oracle_gsym_nnzu(const oracle_gsym* s) { return s->nnzu; }
const int64_t* oracle_gsym_lptr(const oracle_gsym* s) { return s->lptr; }
const int64_t* oracle_gsym_lidx(const oracle_gsym* s) { return s->lidx; }
const int64_t* oracle_gsym_uptr(const oracle_gsym* s) { return s->uptr; }
const int64_t* oracle_gsym_uidx(const oracle_gsym* s) { return s->uidx; }

/* growable int64 list */
typedef struct {
  int64_t* v;
  int64_t n, cap;
} ilist;
static int ilist_push(ilist* l, int64_t x) {
  if (l->n == l->cap) {
    int64_t cap = l->cap ? 2 * l->cap : 16;
    int64_t* v = (int64_t*)realloc(l->v, sizeof(int64_t) * (size_t)cap);
    if (!v) return ORACLE_ERR_OOM;
    l->v = v;
    l->cap = cap;
  }
  l->v[l->n++] = x;
  return ORACLE_OK;
}
static int cmp_i64(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : x > y;
}

static int is_perm(int64_t n, const int64_t* p, int64_t* inv) {
  for (int64_t i = 0; i < n; i++) inv[i] = -1;
  for (int64_t i = 0; i < n; i++) {
    if (p[i] < 0 || p[i] >= n || inv[p[i]] >= 0) return 0;
    inv[p[i]] = i;
  }
  return 1;
}

int oracle_ganalyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                    const int64_t* rperm, const int64_t* cperm, oracle_gsym** out) {
  if (!out || n < 0 || !colptr || (n > 0 && !rowind)) return ORACLE_ERR_ARG;
  *out = NULL;
  int rc = ORACLE_ERR_OOM;
  oracle_gsym* s = (oracle_gsym*)calloc(1, sizeof(oracle_gsym));
  if (!s) return ORACLE_ERR_OOM;
  s->n = n;
  const size_t nn = (size_t)(n + 1);
  s->rperm = (int64_t*)malloc(sizeof(int64_t) * nn);
  s->cperm = (int64_t*)malloc(sizeof(int64_t) * nn);
  s->irperm = (int64_t*)malloc(sizeof(int64_t) * nn);
  s->icperm = (int64_t*)malloc(sizeof(int64_t) * nn);
  s->lptr = (int64_t*)calloc(nn, sizeof(int64_t));
  s->uptr = (int64_t*)calloc(nn, sizeof(int64_t));
  /* per new row / column: Atilde's off-diagonal pattern, and the lists of
   * earlier steps j whose L column (ul[k]: k in C_U(j)) or U row
   * (lu_[k]: k in C_L(j)) reach k */
  ilist* arow = (ilist*)calloc(nn, sizeof(ilist));   /* Atilde(k, m), m > k */
  ilist* acol = (ilist*)calloc(nn, sizeof(ilist));   /* Atilde(i, k), i > k */
  ilist* ul = (ilist*)calloc(nn, sizeof(ilist));
  ilist* lu_ = (ilist*)calloc(nn, sizeof(ilist));
  ilist L = {0}, U = {0};
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * nn);
  if (!s->rperm || !s->cperm || !s->irperm || !s->icperm || !s->lptr || !s->uptr || !arow ||
      !acol || !ul || !lu_ || !mark)
    goto fail;
  for (int64_t i = 0; i < n; i++) {
    s->rperm[i] = rperm ? rperm[i] : i;
    s->cperm[i] = cperm ? cperm[i] : i;
  }
  rc = ORACLE_ERR_ARG;
  if (!is_perm(n, s->rperm, s->irperm) || !is_perm(n, s->cperm, s->icperm)) goto fail;
  for (int64_t c = 0; c < n; c++)
    for (int64_t p = colptr[c]; p < colptr[c + 1]; p++) {
      const int64_t r = rowind[p];
      if (r < 0 || r >= n || (p > colptr[c] && rowind[p - 1] >= r)) goto fail;
      const int64_t i = s->irperm[r], k = s->icperm[c];  /* Atilde(i, k) */
      rc = ORACLE_ERR_OOM;
      if (i > k && ilist_push(&acol[k], i)) goto fail;
      if (i < k && ilist_push(&arow[i], k)) goto fail;
      rc = ORACLE_ERR_ARG;
    }
  rc = ORACLE_ERR_OOM;
  for (int64_t i = 0; i < n; i++) mark[i] = -1;
  for (int64_t k = 0; k < n; k++) {
    /* C_L(k) */
    const int64_t l0 = L.n;
    for (int64_t t = 0; t < acol[k].n; t++)
      if (mark[acol[k].v[t]] != 2 * k) {
        mark[acol[k].v[t]] = 2 * k;
        if (ilist_push(&L, acol[k].v[t])) goto fail;
      }
    for (int64_t t = 0; t < ul[k].n; t++) {
      const int64_t j = ul[k].v[t];
      for (int64_t p = s->lptr[j]; p < s->lptr[j + 1]; p++) {
        const int64_t i = L.v[p];
        if (i > k && mark[i] != 2 * k) {
          mark[i] = 2 * k;
          if (ilist_push(&L, i)) goto fail;
        }
      }
    }
    qsort(L.v + l0, (size_t)(L.n - l0), sizeof(int64_t), cmp_i64);
    s->lptr[k + 1] = L.n;
    /* C_U(k) */
    const int64_t u0 = U.n;
    for (int64_t t = 0; t < arow[k].n; t++)
      if (mark[arow[k].v[t]] != 2 * k + 1) {
        mark[arow[k].v[t]] = 2 * k + 1;
        if (ilist_push(&U, arow[k].v[t])) goto fail;
      }
    for (int64_t t = 0; t < lu_[k].n; t++) {
      const int64_t j = lu_[k].v[t];
      for (int64_t p = s->uptr[j]; p < s->uptr[j + 1]; p++) {
        const int64_t m = U.v[p];
        if (m > k && mark[m] != 2 * k + 1) {
          mark[m] = 2 * k + 1;
          if (ilist_push(&U, m)) goto fail;
        }
      }
    }
    qsort(U.v + u0, (size_t)(U.n - u0), sizeof(int64_t), cmp_i64);
    s->uptr[k + 1] = U.n;
    /* step k reaches the L columns of C_U(k) and the U rows of C_L(k) */
    for (int64_t p = u0; p < U.n; p++)
      if (ilist_push(&ul[U.v[p]], k)) goto fail;
    for (int64_t p = l0; p < L.n; p++)
      if (ilist_push(&lu_[L.v[p]], k)) goto fail;
  }
  s->lidx = L.v;
  s->uidx = U.v;
  L.v = U.v = NULL;
  s->nnzl = s->lptr[n];
  s->nnzu = s->uptr[n];
  rc = ORACLE_OK;
fail:
  for (int64_t i = 0; i < n + 1 && arow && acol && ul && lu_; i++) {
    free(arow[i].v);
    free(acol[i].v);
    free(ul[i].v);
    free(lu_[i].v);
  }
  free(arow);
  free(acol);
  free(ul);
  free(lu_);
  free(L.v);
  free(U.v);
  free(mark);
  if (rc != ORACLE_OK) {
    oracle_gsym_free(s);
    return rc;
  }
  *out = s;
  return ORACLE_OK;
}

/* position of x in the sorted list idx[lo .. hi), or -1 */
static int64_t gfind(const int64_t* idx, int64_t lo, int64_t hi, int64_t x) {
  hi -= 1;
  while (lo <= hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (idx[mid] == x) return mid;
    if (idx[mid] < x) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

#define SCALAR double
#define SFX(name) name##_d
#include "oracle_gnum.inc"
#undef SCALAR
#undef SFX

#define SCALAR double _Complex
#define SFX(name) name##_z_impl
#include "oracle_gnum.inc"
#undef SCALAR
#undef SFX

int oracle_glu_z(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                 const void* values, void* L, void* U, void* D, int64_t* bad_col) {
  return oracle_glu_z_impl(s, colptr, rowind, (const double _Complex*)values,
                           (double _Complex*)L, (double _Complex*)U, (double _Complex*)D,
                           bad_col);
}
int oracle_gselinv_z(const oracle_gsym* s, const void* L, const void* U, const void* D,
                     void* BL, void* BU, void* BD, int mutation) {
  return oracle_gselinv_z_impl(s, (const double _Complex*)L, (const double _Complex*)U,
                               (const double _Complex*)D, (double _Complex*)BL,
                               (double _Complex*)BU, (double _Complex*)BD, mutation);
}
int oracle_gextract_z(const oracle_gsym* s, const int64_t* colptr, const int64_t* rowind,
                      const void* BL, const void* BU, const void* BD, void* out) {
  return oracle_gextract_z_impl(s, colptr, rowind, (const double _Complex*)BL,
                                (const double _Complex*)BU, (const double _Complex*)BD,
                                (double _Complex*)out);
}
