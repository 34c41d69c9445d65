/*
 * CPU oracle: symbolic analysis, double-double dense inverse, and the
 * instantiation of the scalar numeric routines for real and complex values.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct oracle_sym {
  int64_t n;
  int64_t* perm;       /* new -> old */
  int64_t* iperm;      /* old -> new */
  int64_t* parent;     /* column elimination tree */
  int64_t* sptr;       /* struct(j) as CSC */
  int64_t* sidx;
  int64_t nnzl;
  int64_t nsup;
  int64_t* supptr;
  int64_t* sup_of;
  int64_t* sup_parent;
  int64_t* sup_depth;
};

int64_t oracle_sym_n(const oracle_sym* s) { return s->n; }
int64_t oracle_sym_nnzl(const oracle_sym* s) { return s->nnzl; }
int64_t oracle_sym_nsup(const oracle_sym* s) { return s->nsup; }
const int64_t* oracle_sym_parent(const oracle_sym* s) { return s->parent; }
const int64_t* oracle_sym_sptr(const oracle_sym* s) { return s->sptr; }
const int64_t* oracle_sym_sidx(const oracle_sym* s) { return s->sidx; }
const int64_t* oracle_sym_supptr(const oracle_sym* s) { return s->supptr; }
const int64_t* oracle_sym_sup_parent(const oracle_sym* s) { return s->sup_parent; }
const int64_t* oracle_sym_sup_depth(const oracle_sym* s) { return s->sup_depth; }

void oracle_sym_free(oracle_sym* s) {
  if (!s) return;
  free(s->perm);
  free(s->iperm);
  free(s->parent);
  free(s->sptr);
  free(s->sidx);
  free(s->supptr);
  free(s->sup_of);
  free(s->sup_parent);
  free(s->sup_depth);
  free(s);
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* position of `row` in column `col` of the CSC pattern, or -1 */
static int64_t csc_find(const int64_t* colptr, const int64_t* rowind, int64_t col, int64_t row) {
  int64_t lo = colptr[col], hi = colptr[col + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (rowind[mid] == row) return mid;
    if (rowind[mid] < row) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* position of row i in struct(j) (i > j), or -1 */
int64_t oracle_find_(const oracle_sym* s, int64_t j, int64_t i) {
  int64_t lo = s->sptr[j], hi = s->sptr[j + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (s->sidx[mid] == i) return mid;
    if (s->sidx[mid] < i) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int oracle_analyze(int64_t n, const int64_t* colptr, const int64_t* rowind,
                   const int64_t* perm, int64_t max_sn, int64_t relax_pct, oracle_sym** out) {
  if (!out || n < 0 || !colptr || (n > 0 && !rowind) || max_sn < 1 || relax_pct < 0 ||
      relax_pct > 100)
    return ORACLE_ERR_ARG;
  *out = NULL;
  /* validate the CSC pattern */
  if (colptr[0] != 0) return ORACLE_ERR_ARG;
  for (int64_t j = 0; j < n; j++) {
    if (colptr[j + 1] < colptr[j]) return ORACLE_ERR_ARG;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
      if (rowind[p] < 0 || rowind[p] >= n) return ORACLE_ERR_ARG;
      if (p > colptr[j] && rowind[p] <= rowind[p - 1]) return ORACLE_ERR_ARG;
    }
  }
  /* structural symmetry: A_ij != 0  <=>  A_ji != 0 (selected-element set of
   * the structurally symmetric case, Section 1) */
  for (int64_t j = 0; j < n; j++)
    for (int64_t p = colptr[j]; p < colptr[j + 1]; p++)
      if (csc_find(colptr, rowind, rowind[p], j) < 0) return ORACLE_ERR_NOT_STRUCT_SYM;

  oracle_sym* s = (oracle_sym*)calloc(1, sizeof(oracle_sym));
  if (!s) return ORACLE_ERR_OOM;
  s->n = n;
  s->perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s->iperm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s->parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s->sptr = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
  s->sup_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* child_head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* child_next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t* buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!s->perm || !s->iperm || !s->parent || !s->sptr || !s->sup_of || !mark || !child_head ||
      !child_next || !buf) {
    free(mark); free(child_head); free(child_next); free(buf);
    oracle_sym_free(s);
    return ORACLE_ERR_OOM;
  }
  for (int64_t k = 0; k < n; k++) s->perm[k] = perm ? perm[k] : k;
  for (int64_t k = 0; k < n; k++) s->iperm[k] = -1;
  for (int64_t k = 0; k < n; k++) {
    int64_t o = s->perm[k];
    if (o < 0 || o >= n || s->iperm[o] >= 0) {
      free(mark); free(child_head); free(child_next); free(buf);
      oracle_sym_free(s);
      return ORACLE_ERR_ARG;
    }
    s->iperm[o] = k;
  }
  for (int64_t k = 0; k < n; k++) { mark[k] = -1; child_head[k] = -1; child_next[k] = -1; }

  /* struct(j) = ({i > j : (PAP^T)_ij != 0} U  U_{c: parent(c)=j} struct(c)) \ {j},
   * computed column by column in increasing j; parent(j) = min struct(j). */
  int64_t cap = 16 + 4 * (colptr[n] > 0 ? colptr[n] : 1);
  s->sidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  if (!s->sidx) {
    free(mark); free(child_head); free(child_next); free(buf);
    oracle_sym_free(s);
    return ORACLE_ERR_OOM;
  }
  int64_t nnzl = 0;
  for (int64_t j = 0; j < n; j++) {
    int64_t cnt = 0;
    int64_t oj = s->perm[j];
    mark[j] = j;
    for (int64_t p = colptr[oj]; p < colptr[oj + 1]; p++) {
      int64_t i = s->iperm[rowind[p]];
      if (i > j && mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
    }
    for (int64_t c = child_head[j]; c >= 0; c = child_next[c]) {
      for (int64_t q = s->sptr[c]; q < s->sptr[c + 1]; q++) {
        int64_t i = s->sidx[q];
        if (i != j && mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
      }
    }
    qsort(buf, (size_t)cnt, sizeof(int64_t), cmp_i64);
    if (nnzl + cnt > cap) {
      while (nnzl + cnt > cap) cap *= 2;
      int64_t* t = (int64_t*)realloc(s->sidx, sizeof(int64_t) * (size_t)cap);
      if (!t) {
        free(mark); free(child_head); free(child_next); free(buf);
        oracle_sym_free(s);
        return ORACLE_ERR_OOM;
      }
      s->sidx = t;
    }
    memcpy(s->sidx + nnzl, buf, sizeof(int64_t) * (size_t)cnt);
    nnzl += cnt;
    s->sptr[j + 1] = nnzl;
    s->parent[j] = cnt > 0 ? buf[0] : -1;
    if (cnt > 0) {
      int64_t p = buf[0];
      child_next[j] = child_head[p];
      child_head[p] = j;
    }
  }
  s->nnzl = nnzl;

  /* Supernodes (Section 2, supernode definition with the width limit and
   * the relaxation the paper allows): the column range [f, j] is extended by
   * column j+1 iff
   *   (a) the width stays <= max_sn,
   *   (b) every column i in [f, j] has its parent in [f, j+1], so that
   *       struct(i) \ [f, j+1] is contained in struct(j+1) (the block's row
   *       structure below it is R = struct(j+1)), and
   *   (c) storing the block densely (diagonal block plus |R| rows) adds at
   *       most relax_pct percent explicit zeros to its lower part:
   *       100 * zeros <= relax_pct * total, with
   *       total = sum_{i=f}^{j+1} (j+1-i + |R|), zeros = total - sum_i |struct(i)|.
   * With relax_pct = 0 this is the strict definition: consecutive columns
   * with parent(j) = j+1 and struct(j) = {j+1} U struct(j+1). */
  int64_t nsup = 0;
  {
    int64_t f = 0;
    buf[nsup++] = 0;
    if (n > 0) s->sup_of[0] = 0;
    for (int64_t j = 0; j + 1 < n; j++) {
      const int64_t l = j + 1;
      int joins = (l - f + 1) <= max_sn;
      for (int64_t i = f; i <= j && joins; i++)
        if (s->parent[i] < f || s->parent[i] > l) joins = 0;
      if (joins) {
        const int64_t R = s->sptr[l + 1] - s->sptr[l];
        int64_t total = 0, nz = 0;
        for (int64_t i = f; i <= l; i++) {
          total += (l - i) + R;
          nz += s->sptr[i + 1] - s->sptr[i];
        }
        if (100 * (total - nz) > relax_pct * total) joins = 0;
      }
      if (!joins) { f = l; buf[nsup++] = l; } /* buf reused: first column of each supernode */
      s->sup_of[l] = nsup - 1;
    }
    if (n == 0) nsup = 0;
  }
  s->nsup = nsup;
  s->supptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsup + 1));
  s->sup_parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsup + 1));
  s->sup_depth = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsup + 1));
  if (!s->supptr || !s->sup_parent || !s->sup_depth) {
    free(mark); free(child_head); free(child_next); free(buf);
    oracle_sym_free(s);
    return ORACLE_ERR_OOM;
  }
  for (int64_t k = 0; k < nsup; k++) s->supptr[k] = buf[k];
  s->supptr[nsup] = n;
  /* Per-column structures of the (possibly relaxed) supernodes: column i of
   * K = [f, l] stores rows (i, l] U R_K with R_K = struct(l); explicit zeros
   * count as nonzeros from here on.  For relax_pct = 0 this reproduces the
   * exact structures. */
  {
    int64_t nnz2 = 0;
    for (int64_t k = 0; k < nsup; k++) {
      const int64_t f = s->supptr[k], l = s->supptr[k + 1] - 1;
      const int64_t R = s->sptr[l + 1] - s->sptr[l];
      for (int64_t i = f; i <= l; i++) nnz2 += (l - i) + R;
    }
    int64_t* sptr2 = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    int64_t* sidx2 = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz2 + 1));
    if (!sptr2 || !sidx2) {
      free(sptr2); free(sidx2);
      free(mark); free(child_head); free(child_next); free(buf);
      oracle_sym_free(s);
      return ORACLE_ERR_OOM;
    }
    int64_t q = 0;
    for (int64_t k = 0; k < nsup; k++) {
      const int64_t f = s->supptr[k], l = s->supptr[k + 1] - 1;
      for (int64_t i = f; i <= l; i++) {
        for (int64_t r = i + 1; r <= l; r++) sidx2[q++] = r;
        for (int64_t p = s->sptr[l]; p < s->sptr[l + 1]; p++) sidx2[q++] = s->sidx[p];
        sptr2[i + 1] = q;
      }
    }
    free(s->sptr);
    free(s->sidx);
    s->sptr = sptr2;
    s->sidx = sidx2;
    s->nnzl = nnz2;
  }
  /* supernodal tree: the parent of K is the supernode holding the parent of
   * K's last column; parents have larger indices, so depths (root = 0) are
   * filled from the last supernode down. */
  for (int64_t k = 0; k < nsup; k++) {
    int64_t last = s->supptr[k + 1] - 1;
    s->sup_parent[k] = s->parent[last] >= 0 ? s->sup_of[s->parent[last]] : -1;
  }
  for (int64_t k = nsup - 1; k >= 0; k--)
    s->sup_depth[k] = s->sup_parent[k] < 0 ? 0 : s->sup_depth[s->sup_parent[k]] + 1;

  free(mark); free(child_head); free(child_next); free(buf);
  *out = s;
  return ORACLE_OK;
}

/* ---------------------------------------------------------------------
 * double-double arithmetic (error-free transformations: Knuth's TwoSum,
 * Dekker's Fast2Sum, TwoProduct through a correctly rounded fma)
 * --------------------------------------------------------------------- */
typedef struct { double hi, lo; } dd;

static dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}
static dd fast_two_sum(double a, double b) {
  double s = a + b;
  double e = b - (s - a);
  dd r = {s, e};
  return r;
}
static dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static dd dd_mul(dd x, dd y) {
  double p = x.hi * y.hi;
  double e = fma(x.hi, y.hi, -p);
  e += x.hi * y.lo + x.lo * y.hi;
  return fast_two_sum(p, e);
}
static dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_add(x, dd_neg(dd_mul((dd){q1, 0.0}, y)));
  double q2 = r.hi / y.hi;
  r = dd_add(r, dd_neg(dd_mul((dd){q2, 0.0}, y)));
  double q3 = r.hi / y.hi;
  dd q = fast_two_sum(q1, q2);
  return dd_add(q, (dd){q3, 0.0});
}

int oracle_dense_inverse_dd(int64_t n, const double* a, double* inv_hi, double* inv_lo) {
  if (n < 0 || (n > 0 && (!a || !inv_hi || !inv_lo))) return ORACLE_ERR_ARG;
  /* augmented [A | I] in double-double, column-major n x 2n */
  dd* m = (dd*)malloc(sizeof(dd) * (size_t)(2 * n * n + 1));
  if (!m) return ORACLE_ERR_OOM;
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) {
      m[i + j * n] = (dd){a[i + j * n], 0.0};
      m[i + (n + j) * n] = (dd){i == j ? 1.0 : 0.0, 0.0};
    }
  for (int64_t k = 0; k < n; k++) {
    int64_t piv = k;
    for (int64_t i = k + 1; i < n; i++)
      if (fabs(m[i + k * n].hi) > fabs(m[piv + k * n].hi)) piv = i;
    if (m[piv + k * n].hi == 0.0) { free(m); return ORACLE_ERR_SINGULAR; }
    if (piv != k)
      for (int64_t j = 0; j < 2 * n; j++) {
        dd t = m[k + j * n]; m[k + j * n] = m[piv + j * n]; m[piv + j * n] = t;
      }
    dd p = m[k + k * n];
    for (int64_t j = 0; j < 2 * n; j++) m[k + j * n] = dd_div(m[k + j * n], p);
    for (int64_t i = 0; i < n; i++) {
      if (i == k) continue;
      dd f = m[i + k * n];
      if (f.hi == 0.0 && f.lo == 0.0) continue;
      for (int64_t j = 0; j < 2 * n; j++)
        m[i + j * n] = dd_add(m[i + j * n], dd_neg(dd_mul(f, m[k + j * n])));
    }
  }
  for (int64_t j = 0; j < n; j++)
    for (int64_t i = 0; i < n; i++) {
      inv_hi[i + j * n] = m[i + (n + j) * n].hi;
      inv_lo[i + j * n] = m[i + (n + j) * n].lo;
    }
  free(m);
  return ORACLE_OK;
}

/* ---------------------------------------------------------------------
 * numeric routines, instantiated for real and complex scalars
 * --------------------------------------------------------------------- */
#define SCALAR double
#define SFX(name) name##_d
#define SABS(x) fabs(x)
#include "oracle_num.inc"
#undef SCALAR
#undef SFX
#undef SABS

#define SCALAR double _Complex
#define SFX(name) name##_z_impl
#define SABS(x) cabs(x)
#include "oracle_num.inc"
#undef SCALAR
#undef SFX
#undef SABS

int oracle_lu_z(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                const void* values, void* Llow, void* Uup, void* Udiag, int64_t* bad_col) {
  return oracle_lu_z_impl(s, colptr, rowind, (const double _Complex*)values,
                          (double _Complex*)Llow, (double _Complex*)Uup,
                          (double _Complex*)Udiag, bad_col);
}
int oracle_selinv_z(const oracle_sym* s, const void* Llow, const void* Uup, const void* Udiag,
                    void* Blow, void* Bup, void* Bdiag, int mutation) {
  return oracle_selinv_z_impl(s, (const double _Complex*)Llow, (const double _Complex*)Uup,
                              (const double _Complex*)Udiag, (double _Complex*)Blow,
                              (double _Complex*)Bup, (double _Complex*)Bdiag, mutation);
}
int oracle_selinv_par_z(const oracle_sym* s, const void* Llow, const void* Uup, const void* Udiag,
                        void* Blow, void* Bup, void* Bdiag, int nthreads) {
  return oracle_selinv_par_z_impl(s, (const double _Complex*)Llow, (const double _Complex*)Uup,
                                  (const double _Complex*)Udiag, (double _Complex*)Blow,
                                  (double _Complex*)Bup, (double _Complex*)Bdiag, nthreads);
}
int oracle_extract_z(const oracle_sym* s, const int64_t* colptr, const int64_t* rowind,
                     const void* Blow, const void* Bup, const void* Bdiag, void* out) {
  return oracle_extract_z_impl(s, colptr, rowind, (const double _Complex*)Blow,
                               (const double _Complex*)Bup, (const double _Complex*)Bdiag,
                               (double _Complex*)out);
}
