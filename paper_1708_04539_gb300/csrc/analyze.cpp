// Host symbolic analysis (no CUDA): elimination tree, column counts,
// relaxed width-limited supernodes, supernodal row structures R_K, levels,
// block index maps and the value map.
//
// Algorithms: the elimination tree by Liu's ancestor walk with path
// compression; column counts by traversing each row subtree of the tree;
// supernodal row structures by merging the children's R_J with the
// supernode's own adjacency.  (The scalar reference builds the same objects
// column by column from their definitions.)
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace pselinv {

namespace {

// Supernode partition (Section 2's supernode definition, width limited,
// with the relaxation the paper allows).  [f, l-1] is extended by column l
// iff the width stays <= max_sn, every column of [f, l-1] has its parent in
// [f, l], and storing the block densely (diagonal block plus |struct(l)|
// rows) keeps 100 * zeros <= relax_pct * total over its strictly lower part.
// Returns the first column of every supernode plus n.
std::vector<int64_t> partition(int64_t n, const std::vector<int64_t>& etree,
                               const std::vector<int64_t>& cnt, int64_t max_sn,
                               int64_t relax_pct) {
  std::vector<int64_t> first;
  if (n == 0) {
    first.push_back(0);
    return first;
  }
  first.push_back(0);
  int64_t f = 0;
  int64_t maxpar = etree[0];  // max parent over [f, l-1]; -1 marks a root inside
  bool has_root = etree[0] < 0;
  int64_t nzsum = cnt[0];
  for (int64_t l = 1; l < n; l++) {
    const int64_t w = l - f + 1;
    bool join = w <= max_sn && !has_root && maxpar <= l;
    if (join) {
      const int64_t total = w * (w - 1) / 2 + w * cnt[l];
      const int64_t zeros = total - (nzsum + cnt[l]);
      join = 100 * zeros <= relax_pct * total;
    }
    if (join) {
      nzsum += cnt[l];
    } else {
      first.push_back(l);
      f = l;
      nzsum = cnt[l];
      maxpar = -1;
      has_root = false;
    }
    if (etree[l] < 0) has_root = true;
    maxpar = std::max(maxpar, etree[l]);
  }
  first.push_back(n);
  return first;
}

}  // namespace

int analyze_host(int64_t n, const int64_t* colptr, const int64_t* rowind, const int64_t* perm,
                 int64_t max_sn, int64_t relax_pct, HostSym& S) {
  try {
    if (n < 0 || !colptr || (n > 0 && !rowind) || max_sn < 1 || relax_pct < 0 || relax_pct > 100)
      return PSELINV_ERR_ARG;
    if (colptr[0] != 0) return PSELINV_ERR_ARG;
    for (int64_t j = 0; j < n; j++) {
      if (colptr[j + 1] < colptr[j]) return PSELINV_ERR_ARG;
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
        if (rowind[p] < 0 || rowind[p] >= n) return PSELINV_ERR_ARG;
        if (p > colptr[j] && rowind[p] <= rowind[p - 1]) return PSELINV_ERR_ARG;
      }
    }
    const int64_t nnz = colptr[n];
    S.n = n;
    S.nnz = nnz;
    S.max_sn = max_sn;
    S.relax_pct = relax_pct;

    // structural symmetry: the transpose (by counting sort) equals the input
    {
      std::vector<int64_t> tptr(n + 1, 0), tidx(nnz), fill(n);
      for (int64_t p = 0; p < nnz; p++) tptr[rowind[p] + 1]++;
      for (int64_t j = 0; j < n; j++) tptr[j + 1] += tptr[j];
      for (int64_t j = 0; j < n; j++) fill[j] = tptr[j];
      for (int64_t j = 0; j < n; j++)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) tidx[fill[rowind[p]]++] = j;
      if (!std::equal(tptr.begin(), tptr.end(), colptr)) return PSELINV_ERR_NOT_STRUCT_SYM;
      if (!std::equal(tidx.begin(), tidx.end(), rowind)) return PSELINV_ERR_NOT_STRUCT_SYM;
    }

    S.perm.resize(n);
    S.iperm.assign(n, -1);
    for (int64_t k = 0; k < n; k++) {
      const int64_t o = perm ? perm[k] : k;
      if (o < 0 || o >= n || S.iperm[o] >= 0) return PSELINV_ERR_ARG;
      S.perm[k] = o;
      S.iperm[o] = k;
    }

    // adjacency of P A P^T without the diagonal, per new column
    std::vector<int64_t> aptr(n + 1, 0), aidx;
    for (int64_t oj = 0; oj < n; oj++)
      for (int64_t p = colptr[oj]; p < colptr[oj + 1]; p++)
        if (rowind[p] != oj) aptr[S.iperm[oj] + 1]++;
    for (int64_t j = 0; j < n; j++) aptr[j + 1] += aptr[j];
    aidx.resize(aptr[n]);
    {
      std::vector<int64_t> pos(aptr.begin(), aptr.end() - 1);
      for (int64_t oj = 0; oj < n; oj++)
        for (int64_t p = colptr[oj]; p < colptr[oj + 1]; p++)
          if (rowind[p] != oj) aidx[pos[S.iperm[oj]]++] = S.iperm[rowind[p]];
    }

    // elimination tree (Liu): for column j, every i < j adjacent to j is
    // a descendant of j; walk from i to its current root with path
    // compression and hang that root under j.
    S.etree.assign(n, -1);
    {
      std::vector<int64_t> anc(n, -1);
      for (int64_t j = 0; j < n; j++) {
        for (int64_t p = aptr[j]; p < aptr[j + 1]; p++) {
          int64_t r = aidx[p];
          if (r >= j) continue;
          while (anc[r] != -1 && anc[r] != j) {
            const int64_t t = anc[r];
            anc[r] = j;
            r = t;
          }
          if (anc[r] == -1) {
            anc[r] = j;
            S.etree[r] = j;
          }
        }
      }
    }

    // column counts |struct(x)|: row i of L is the union of the tree paths
    // from every k < i adjacent to i up to i (the row subtree).
    S.colcount.assign(n, 0);
    {
      std::vector<int64_t> mark(n, -1);
      for (int64_t i = 0; i < n; i++) {
        mark[i] = i;
        for (int64_t p = aptr[i]; p < aptr[i + 1]; p++) {
          int64_t x = aidx[p];
          if (x >= i) continue;
          while (x >= 0 && mark[x] != i) {
            mark[x] = i;
            S.colcount[x]++;
            x = S.etree[x];
          }
        }
      }
    }

    // supernodes
    const std::vector<int64_t> first = partition(n, S.etree, S.colcount, max_sn, relax_pct);
    const int64_t ns = (int64_t)first.size() - 1;
    S.ns = ns;
    S.sn_first.assign(first.begin(), first.end() - 1);
    S.sn_width.resize(ns);
    S.sup_of.resize(n);
    for (int64_t k = 0; k < ns; k++) {
      S.sn_width[k] = first[k + 1] - first[k];
      for (int64_t j = first[k]; j < first[k + 1]; j++) S.sup_of[j] = k;
    }

    // R_K = (adjacency of K's columns U R_J of the child supernodes J)
    //       restricted to rows after K's last column
    S.rows_ptr.assign(ns + 1, 0);
    S.rows.clear();
    S.sn_parent.assign(ns, -1);
    {
      std::vector<std::vector<int64_t>> children(ns);
      std::vector<int64_t> mark(n, -1), buf;
      for (int64_t k = 0; k < ns; k++) {
        const int64_t f = first[k], l = first[k + 1] - 1;
        buf.clear();
        for (int64_t j = f; j <= l; j++)
          for (int64_t p = aptr[j]; p < aptr[j + 1]; p++) {
            const int64_t r = aidx[p];
            if (r > l && mark[r] != k) {
              mark[r] = k;
              buf.push_back(r);
            }
          }
        for (int64_t J : children[k])
          for (int64_t p = S.rows_ptr[J]; p < S.rows_ptr[J + 1]; p++) {
            const int64_t r = S.rows[p];
            if (r > l && mark[r] != k) {
              mark[r] = k;
              buf.push_back(r);
            }
          }
        std::sort(buf.begin(), buf.end());
        if ((int64_t)buf.size() != S.colcount[l]) return PSELINV_ERR_ARG;  // inconsistent structure
        S.rows.insert(S.rows.end(), buf.begin(), buf.end());
        S.rows_ptr[k + 1] = (int64_t)S.rows.size();
        if (!buf.empty()) {
          S.sn_parent[k] = S.sup_of[buf[0]];
          children[S.sn_parent[k]].push_back(k);
        }
      }
    }

    // depth (roots 0) and height (leaves 0); parents have larger indices
    S.sn_depth.assign(ns, 0);
    S.sn_height.assign(ns, 0);
    for (int64_t k = ns - 1; k >= 0; k--)
      S.sn_depth[k] = S.sn_parent[k] < 0 ? 0 : S.sn_depth[S.sn_parent[k]] + 1;
    for (int64_t k = 0; k < ns; k++)
      if (S.sn_parent[k] >= 0)
        S.sn_height[S.sn_parent[k]] = std::max(S.sn_height[S.sn_parent[k]], S.sn_height[k] + 1);
    auto bucket = [&](const std::vector<int64_t>& key, std::vector<int64_t>& ptr,
                      std::vector<int64_t>& items) {
      int64_t nl = 0;
      for (int64_t k = 0; k < ns; k++) nl = std::max(nl, key[k] + 1);
      ptr.assign(nl + 1, 0);
      for (int64_t k = 0; k < ns; k++) ptr[key[k] + 1]++;
      for (int64_t d = 0; d < nl; d++) ptr[d + 1] += ptr[d];
      items.resize(ns);
      std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
      for (int64_t k = 0; k < ns; k++) items[pos[key[k]]++] = k;
    };
    bucket(S.sn_depth, S.level_ptr, S.level_sn);
    bucket(S.sn_height, S.hlevel_ptr, S.hlevel_sn);

    // storage: per supernode [diag s*s | L panel c*s | U^T panel c*s]
    S.sn_offset.resize(ns);
    int64_t off = 0;
    S.flops_selinv = S.flops_factor = 0;
    for (int64_t k = 0; k < ns; k++) {
      const double s = (double)S.sn_width[k], c = (double)(S.rows_ptr[k + 1] - S.rows_ptr[k]);
      S.sn_offset[k] = off;
      off += S.sn_width[k] * S.sn_width[k] + 2 * (S.rows_ptr[k + 1] - S.rows_ptr[k]) * S.sn_width[k];
      S.flops_selinv += 4 * c * c * s + 4 * c * s * s + 4.0 / 3.0 * s * s * s;
      S.flops_factor += 2 * c * c * s + 2 * c * s * s + 2.0 / 3.0 * s * s * s;
    }
    S.storage = off;
    {
      const std::vector<int64_t> strict = partition(n, S.etree, S.colcount, max_sn, 0);
      S.flops_selinv_exact = 0;
      for (size_t k = 0; k + 1 < strict.size(); k++) {
        const double s = (double)(strict[k + 1] - strict[k]);
        const double c = (double)S.colcount[strict[k + 1] - 1];
        S.flops_selinv_exact += 4 * c * c * s + 4 * c * s * s + 4.0 / 3.0 * s * s * s;
      }
    }

    // blocks of R_K and the relative index maps
    S.sn_blk.assign(ns + 1, 0);
    S.blk_sn.clear();
    S.blk_pb.clear();
    S.blk_pe.clear();
    S.blk_rel.clear();
    S.rows_blk.assign(S.rows.size(), 0);
    S.relidx.clear();
    for (int64_t k = 0; k < ns; k++) {
      const int64_t rb = S.rows_ptr[k], c = S.rows_ptr[k + 1] - rb;
      S.sn_blk[k] = (int32_t)S.blk_sn.size();
      int64_t p = 0;
      while (p < c) {
        const int64_t J = S.sup_of[S.rows[rb + p]];
        int64_t pe = p;
        while (pe < c && S.sup_of[S.rows[rb + pe]] == J) pe++;
        const int32_t b = (int32_t)S.blk_sn.size();
        S.blk_sn.push_back((int32_t)J);
        S.blk_pb.push_back((int32_t)p);
        S.blk_pe.push_back((int32_t)pe);
        S.blk_rel.push_back((int64_t)S.relidx.size());
        for (int64_t q = p; q < pe; q++) {
          S.rows_blk[rb + q] = b;
          S.relidx.push_back((int32_t)(S.rows[rb + q] - first[J]));
        }
        // rows after the block: positions in R_J (merge of two sorted lists)
        int64_t t = S.rows_ptr[J];
        const int64_t te = S.rows_ptr[J + 1];
        for (int64_t q = pe; q < c; q++) {
          const int64_t r = S.rows[rb + q];
          while (t < te && S.rows[t] < r) t++;
          if (t == te || S.rows[t] != r) return PSELINV_ERR_ARG;  // violates the fill argument
          S.relidx.push_back((int32_t)(t - S.rows_ptr[J]));
        }
        p = pe;
      }
    }
    S.sn_blk[ns] = (int32_t)S.blk_sn.size();

    // storage slot of every input entry
    S.value_map.resize(nnz);
    auto find_row = [&](int64_t K, int64_t r) -> int64_t {
      const int64_t* b = S.rows.data() + S.rows_ptr[K];
      const int64_t* e = S.rows.data() + S.rows_ptr[K + 1];
      const int64_t* it = std::lower_bound(b, e, r);
      return (it != e && *it == r) ? (int64_t)(it - b) : -1;
    };
    for (int64_t oj = 0; oj < n; oj++)
      for (int64_t p = colptr[oj]; p < colptr[oj + 1]; p++) {
        const int64_t i = S.iperm[rowind[p]], j = S.iperm[oj];
        const int64_t I = S.sup_of[i], J = S.sup_of[j];
        int64_t slot;
        if (I == J) {
          slot = S.sn_offset[J] + (i - first[J]) + (j - first[J]) * S.sn_width[J];
        } else if (I > J) {
          const int64_t pos = find_row(J, i);
          if (pos < 0) return PSELINV_ERR_ARG;
          const int64_t cJ = S.rows_ptr[J + 1] - S.rows_ptr[J];
          slot = S.sn_offset[J] + S.sn_width[J] * S.sn_width[J] + pos + (j - first[J]) * cJ;
        } else {
          const int64_t pos = find_row(I, j);
          if (pos < 0) return PSELINV_ERR_ARG;
          const int64_t cI = S.rows_ptr[I + 1] - S.rows_ptr[I];
          slot = S.sn_offset[I] + S.sn_width[I] * S.sn_width[I] + cI * S.sn_width[I] + pos +
                 (i - first[I]) * cI;
        }
        S.value_map[p] = slot;
      }
    return PSELINV_OK;
  } catch (const std::bad_alloc&) {
    return PSELINV_ERR_OOM;
  }
}

}  // namespace pselinv
