// Host symbolic analysis of a GENERAL pattern with static pivoting (no
// CUDA): Atilde = P A Q (row ordering P from `rperm`, column ordering Q from
// `cperm`, both new -> old), the structures of the LU factors without
// pivoting, supernodes, their two row structures (Section 2: C_L, the rows
// of the L panel, and C_U, the columns of the U panel, which need not
// agree), the dependency levels of the sweep and the factorisation, and the
// block index maps of the gather (Algorithm 1 steps 3-5) and of the
// factorisation's Schur scatter.
//
// Scalar structures by the fill rule of Gaussian elimination: eliminating
// column k adds every (i, m) with i in C_L(k), m in C_U(k).  Supernodes:
// column j + 1 joins the supernode ending at j when j + 1 lies in both C_L(j)
// and C_U(j) (the diagonal block stays connected), the width stays within
// max_sn, and storing the union structures densely keeps the explicit
// zeros within relax_pct percent (relax_pct = 0: the strict rule, both
// structures nested with sizes one apart).  The supernodal structures are
// then closed under the supernodal updates: R_L(K) and R_U(K) collect,
// besides K's own columns' structures, R_L(J) and R_U(J) of every earlier J
// whose update reaches K, so the Schur complement of every supernode and
// every operand of the selected inversion lies in the stored pattern (the
// fill argument of Theorem 1 at the supernode level).
#include <algorithm>
#include <new>

#include "internal.h"

namespace pselinv {

namespace {

// sorted union of `extra` into the sorted list `v`, keeping entries > bound
void merge_into(std::vector<int64_t>& v, const int64_t* b, const int64_t* e, int64_t bound,
                std::vector<int64_t>& tmp) {
  tmp.clear();
  size_t i = 0;
  while (b != e && *b <= bound) b++;
  while (i < v.size() || b != e) {
    int64_t x;
    if (b == e || (i < v.size() && v[i] < *b)) {
      x = v[i++];
    } else if (i < v.size() && v[i] == *b) {
      x = v[i++];
      b++;
    } else {
      x = *b++;
    }
    tmp.push_back(x);
  }
  v.swap(tmp);
}

// position of r in the sorted range [b, e), or -1
int64_t find_pos(const int64_t* b, const int64_t* e, int64_t r) {
  const int64_t* it = std::lower_bound(b, e, r);
  return (it != e && *it == r) ? (int64_t)(it - b) : -1;
}

}  // namespace

int analyze_general_host(int64_t n, const int64_t* colptr, const int64_t* rowind,
                         const int64_t* rperm, const int64_t* cperm, int64_t max_sn,
                         int64_t relax_pct, HostSym& S) {
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
    S.general = true;
    S.n = n;
    S.nnz = nnz;
    S.max_sn = max_sn;
    S.relax_pct = relax_pct;
    auto set_perm = [&](const int64_t* pm, std::vector<int64_t>& fwd, std::vector<int64_t>& inv) {
      fwd.resize(n);
      inv.assign(n, -1);
      for (int64_t k = 0; k < n; k++) {
        const int64_t o = pm ? pm[k] : k;
        if (o < 0 || o >= n || inv[o] >= 0) return false;
        fwd[k] = o;
        inv[o] = k;
      }
      return true;
    };
    if (!set_perm(rperm, S.rperm, S.irperm) || !set_perm(cperm, S.perm, S.iperm))
      return PSELINV_ERR_ARG;

    // Atilde's off-diagonal pattern by new column (rows below) and new row
    // (columns right of the diagonal)
    std::vector<std::vector<int64_t>> acol(n), arow(n);
    for (int64_t oc = 0; oc < n; oc++)
      for (int64_t p = colptr[oc]; p < colptr[oc + 1]; p++) {
        const int64_t i = S.irperm[rowind[p]], k = S.iperm[oc];
        if (i > k) acol[k].push_back(i);
        if (i < k) arow[i].push_back(k);
      }

    // scalar structures C_L(k), C_U(k) by the fill rule
    std::vector<int64_t> lptr(n + 1, 0), lidx, uptr(n + 1, 0), uidx;
    {
      std::vector<std::vector<int64_t>> ul(n), lu(n);  // steps j reaching column / row k
      std::vector<int64_t> mark(n, -1), buf;
      for (int64_t k = 0; k < n; k++) {
        buf.clear();
        for (int64_t i : acol[k])
          if (mark[i] != 2 * k) {
            mark[i] = 2 * k;
            buf.push_back(i);
          }
        for (int64_t j : ul[k])
          for (int64_t p = lptr[j]; p < lptr[j + 1]; p++)
            if (lidx[p] > k && mark[lidx[p]] != 2 * k) {
              mark[lidx[p]] = 2 * k;
              buf.push_back(lidx[p]);
            }
        std::sort(buf.begin(), buf.end());
        lidx.insert(lidx.end(), buf.begin(), buf.end());
        lptr[k + 1] = (int64_t)lidx.size();
        buf.clear();
        for (int64_t m : arow[k])
          if (mark[m] != 2 * k + 1) {
            mark[m] = 2 * k + 1;
            buf.push_back(m);
          }
        for (int64_t j : lu[k])
          for (int64_t p = uptr[j]; p < uptr[j + 1]; p++)
            if (uidx[p] > k && mark[uidx[p]] != 2 * k + 1) {
              mark[uidx[p]] = 2 * k + 1;
              buf.push_back(uidx[p]);
            }
        std::sort(buf.begin(), buf.end());
        uidx.insert(uidx.end(), buf.begin(), buf.end());
        uptr[k + 1] = (int64_t)uidx.size();
        for (int64_t p = uptr[k]; p < uptr[k + 1]; p++) ul[uidx[p]].push_back(k);
        for (int64_t p = lptr[k]; p < lptr[k + 1]; p++) lu[lidx[p]].push_back(k);
        std::vector<int64_t>().swap(ul[k]);
        std::vector<int64_t>().swap(lu[k]);
      }
    }
    auto in_list = [&](const std::vector<int64_t>& ptr, const std::vector<int64_t>& idx,
                       int64_t k, int64_t x) {
      return find_pos(idx.data() + ptr[k], idx.data() + ptr[k + 1], x) >= 0;
    };

    // supernodes
    std::vector<int64_t> first{0};
    if (n > 0) {
      int64_t f = 0;
      std::vector<int64_t> RL, RU, tmp;  // union structures of [f, l-1] beyond l-1
      RL.assign(lidx.begin() + lptr[0], lidx.begin() + lptr[1]);
      RU.assign(uidx.begin() + uptr[0], uidx.begin() + uptr[1]);
      int64_t nzl = lptr[1] - lptr[0], nzu = uptr[1] - uptr[0];  // structural entries stored
      for (int64_t l = 1; l < n; l++) {
        const int64_t w = l - f + 1;
        bool join = w <= max_sn && in_list(lptr, lidx, l - 1, l) && in_list(uptr, uidx, l - 1, l);
        std::vector<int64_t> nl, nu;
        if (join) {
          nl = RL;
          merge_into(nl, lidx.data() + lptr[l], lidx.data() + lptr[l + 1], l, tmp);
          nu = RU;
          merge_into(nu, uidx.data() + uptr[l], uidx.data() + uptr[l + 1], l, tmp);
          // drop column l itself from the union structures (now in the block)
          nl.erase(std::remove(nl.begin(), nl.end(), l), nl.end());
          nu.erase(std::remove(nu.begin(), nu.end(), l), nu.end());
          const int64_t total = w * (w - 1) + w * (int64_t)(nl.size() + nu.size());
          const int64_t have = nzl + nzu + (lptr[l + 1] - lptr[l]) + (uptr[l + 1] - uptr[l]);
          const int64_t zeros = total - have;
          join = 100 * zeros <= relax_pct * total;
        }
        if (join) {
          RL.swap(nl);
          RU.swap(nu);
          nzl += lptr[l + 1] - lptr[l];
          nzu += uptr[l + 1] - uptr[l];
        } else {
          first.push_back(l);
          f = l;
          RL.assign(lidx.begin() + lptr[l], lidx.begin() + lptr[l + 1]);
          RU.assign(uidx.begin() + uptr[l], uidx.begin() + uptr[l + 1]);
          nzl = lptr[l + 1] - lptr[l];
          nzu = uptr[l + 1] - uptr[l];
        }
      }
      first.push_back(n);
    }
    const int64_t ns = (int64_t)first.size() - 1;
    S.ns = ns;
    S.sn_first.assign(first.begin(), first.end() - 1);
    S.sn_width.resize(ns);
    S.sup_of.resize(n);
    for (int64_t k = 0; k < ns; k++) {
      S.sn_width[k] = first[k + 1] - first[k];
      for (int64_t j = first[k]; j < first[k + 1]; j++) S.sup_of[j] = k;
    }

    // supernodal structures closed under the supernodal updates
    S.rows_ptr.assign(ns + 1, 0);
    S.urows_ptr.assign(ns + 1, 0);
    S.rows.clear();
    S.urows.clear();
    std::vector<std::vector<int64_t>> reach_l(ns), reach_u(ns);  // J whose R_U / R_L reach K
    std::vector<int64_t> dep_height(ns, 0);
    {
      std::vector<int64_t> RL, RU, tmp;
      for (int64_t k = 0; k < ns; k++) {
        const int64_t f = first[k], l = first[k + 1] - 1;
        RL.clear();
        RU.clear();
        for (int64_t j = f; j <= l; j++) {
          merge_into(RL, lidx.data() + lptr[j], lidx.data() + lptr[j + 1], l, tmp);
          merge_into(RU, uidx.data() + uptr[j], uidx.data() + uptr[j + 1], l, tmp);
        }
        // updates of earlier supernodes J that reach K: J's Schur block
        // R_L(J) x R_U(J) has entries in K's columns (R_U(J) meets K: rows of
        // R_L(J) below K join R_L(K)) or in K's rows (R_L(J) meets K:
        // columns of R_U(J) right of K join R_U(K))
        for (int64_t J : reach_l[k])
          merge_into(RL, S.rows.data() + S.rows_ptr[J], S.rows.data() + S.rows_ptr[J + 1], l, tmp);
        for (int64_t J : reach_u[k])
          merge_into(RU, S.urows.data() + S.urows_ptr[J], S.urows.data() + S.urows_ptr[J + 1], l,
                     tmp);
        S.rows.insert(S.rows.end(), RL.begin(), RL.end());
        S.rows_ptr[k + 1] = (int64_t)S.rows.size();
        S.urows.insert(S.urows.end(), RU.begin(), RU.end());
        S.urows_ptr[k + 1] = (int64_t)S.urows.size();
        // the supernodes K's own update reaches, each once; they depend on K
        // in the factorisation (height) and K depends on them in the sweep
        int64_t last = -1;
        for (int64_t m : RU) {
          const int64_t T = S.sup_of[m];
          if (T != last) reach_l[T].push_back(k);
          last = T;
        }
        last = -1;
        for (int64_t i : RL) {
          const int64_t T = S.sup_of[i];
          if (T != last) reach_u[T].push_back(k);
          last = T;
        }
      }
    }
    // factorisation height (leaves 0): K after every J whose update reaches it;
    // sweep depth (roots 0): K after every supernode of R_L(K) and R_U(K)
    S.sn_height.assign(ns, 0);
    for (int64_t k = 0; k < ns; k++) {
      for (int64_t J : reach_l[k]) S.sn_height[k] = std::max(S.sn_height[k], S.sn_height[J] + 1);
      for (int64_t J : reach_u[k]) S.sn_height[k] = std::max(S.sn_height[k], S.sn_height[J] + 1);
    }
    S.sn_depth.assign(ns, 0);
    S.sn_parent.assign(ns, -1);
    for (int64_t k = ns - 1; k >= 0; k--) {
      int64_t d = -1, par = -1;
      for (int64_t p = S.rows_ptr[k]; p < S.rows_ptr[k + 1]; p++)
        d = std::max(d, S.sn_depth[S.sup_of[S.rows[p]]]);
      for (int64_t p = S.urows_ptr[k]; p < S.urows_ptr[k + 1]; p++)
        d = std::max(d, S.sn_depth[S.sup_of[S.urows[p]]]);
      const int64_t a = S.rows_ptr[k + 1] > S.rows_ptr[k] ? S.sup_of[S.rows[S.rows_ptr[k]]] : ns;
      const int64_t b = S.urows_ptr[k + 1] > S.urows_ptr[k] ? S.sup_of[S.urows[S.urows_ptr[k]]] : ns;
      par = std::min(a, b);
      S.sn_depth[k] = d + 1;
      S.sn_parent[k] = par < ns ? par : -1;
    }
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
    // the column elimination tree is not defined for a general pattern:
    // report each column's first structure row (its parent in the tree of
    // the L structures)
    S.etree.assign(n, -1);
    S.colcount.assign(n, 0);
    for (int64_t k = 0; k < n; k++) {
      if (lptr[k + 1] > lptr[k]) S.etree[k] = lidx[lptr[k]];
      S.colcount[k] = lptr[k + 1] - lptr[k];
    }

    // storage: per supernode [diag s*s | L panel c_L*s | U^T panel c_U*s]
    S.sn_offset.resize(ns);
    int64_t off = 0;
    S.flops_selinv = S.flops_factor = 0;
    for (int64_t k = 0; k < ns; k++) {
      const int64_t s = S.sn_width[k];
      const int64_t cl = S.rows_ptr[k + 1] - S.rows_ptr[k], cu = S.urows_ptr[k + 1] - S.urows_ptr[k];
      S.sn_offset[k] = off;
      off += s * s + (cl + cu) * s;
      const double ds = (double)s, dl = (double)cl, du = (double)cu;
      S.flops_selinv += 4 * dl * du * ds + 2 * (dl + du) * ds * ds + 4.0 / 3.0 * ds * ds * ds;
      S.flops_factor += 2 * dl * du * ds + (dl + du) * ds * ds + 2.0 / 3.0 * ds * ds * ds;
    }
    S.storage = off;
    // the same count on the scalar structures (strict supernodes of width 1)
    S.flops_selinv_exact = 0;
    for (int64_t k = 0; k < n; k++) {
      const double dl = (double)(lptr[k + 1] - lptr[k]), du = (double)(uptr[k + 1] - uptr[k]);
      S.flops_selinv_exact += 4 * dl * du + 2 * (dl + du) + 4.0 / 3.0;
    }

    // blocks and relative index maps.  A block of R_L(K) (rows in supernode
    // J) maps every position of R_U(K) from the first row >= first(J): to
    // the local index in J, or to the position in R_U(J).  A block of
    // R_U(K) likewise maps the positions of R_L(K) into J / R_L(J).
    auto build_blocks = [&](const std::vector<int64_t>& own_ptr, const std::vector<int64_t>& own,
                            const std::vector<int64_t>& oth_ptr, const std::vector<int64_t>& oth,
                            const std::vector<int64_t>& tgt_ptr, const std::vector<int64_t>& tgt,
                            std::vector<int32_t>& sn_blk, std::vector<int32_t>& blk_sn,
                            std::vector<int32_t>& blk_pb, std::vector<int32_t>& blk_pe,
                            std::vector<int32_t>& blk_q0, std::vector<int64_t>& blk_rel,
                            std::vector<int32_t>& rows_blk, std::vector<int32_t>& rel) -> bool {
      sn_blk.assign(ns + 1, 0);
      rows_blk.assign(own.size(), 0);
      for (int64_t k = 0; k < ns; k++) {
        const int64_t rb = own_ptr[k], c = own_ptr[k + 1] - rb;
        const int64_t ob = oth_ptr[k], oc = oth_ptr[k + 1] - ob;
        sn_blk[k] = (int32_t)blk_sn.size();
        int64_t p = 0;
        while (p < c) {
          const int64_t J = S.sup_of[own[rb + p]];
          int64_t pe = p;
          while (pe < c && S.sup_of[own[rb + pe]] == J) pe++;
          const int32_t b = (int32_t)blk_sn.size();
          for (int64_t q = p; q < pe; q++) rows_blk[rb + q] = b;
          const int64_t q0 =
              std::lower_bound(oth.begin() + ob, oth.begin() + ob + oc, first[J]) - (oth.begin() + ob);
          blk_sn.push_back((int32_t)J);
          blk_pb.push_back((int32_t)p);
          blk_pe.push_back((int32_t)pe);
          blk_q0.push_back((int32_t)q0);
          blk_rel.push_back((int64_t)rel.size());
          const int64_t lastJ = first[J + 1] - 1;
          for (int64_t q = q0; q < oc; q++) {
            const int64_t x = oth[ob + q];
            if (x <= lastJ) {
              rel.push_back((int32_t)(x - first[J]));
            } else {
              const int64_t pos = find_pos(tgt.data() + tgt_ptr[J], tgt.data() + tgt_ptr[J + 1], x);
              if (pos < 0) return false;  // outside the closed structure
              rel.push_back((int32_t)pos);
            }
          }
          p = pe;
        }
      }
      sn_blk[ns] = (int32_t)blk_sn.size();
      return true;
    };
    S.blk_sn.clear();
    S.blk_pb.clear();
    S.blk_pe.clear();
    S.blk_q0.clear();
    S.blk_rel.clear();
    S.relidx.clear();
    // blocks of R_L(K) map R_U(K) into R_U(J)
    if (!build_blocks(S.rows_ptr, S.rows, S.urows_ptr, S.urows, S.urows_ptr, S.urows, S.sn_blk,
                      S.blk_sn, S.blk_pb, S.blk_pe, S.blk_q0, S.blk_rel, S.rows_blk, S.relidx))
      return PSELINV_ERR_ARG;
    S.ublk_sn.clear();
    S.ublk_pb.clear();
    S.ublk_pe.clear();
    S.ublk_q0.clear();
    S.ublk_rel.clear();
    // blocks of R_U(K) map R_L(K) into R_L(J) (indices continue in relidx)
    if (!build_blocks(S.urows_ptr, S.urows, S.rows_ptr, S.rows, S.rows_ptr, S.rows, S.usn_blk,
                      S.ublk_sn, S.ublk_pb, S.ublk_pe, S.ublk_q0, S.ublk_rel, S.urows_blk,
                      S.relidx))
      return PSELINV_ERR_ARG;

    // storage slots: the factor entry of every input entry (Atilde_{i,k},
    // i = irperm[row], k = iperm[col]) and the selected entry returned for it
    // ((Atilde^{-1})_{k,i} = (A^{-1})_{col,row}, Theorem 2), which lies on
    // the pattern of (L+U)^T: the slot of the factor entry's transpose
    auto slot_lu = [&](int64_t i, int64_t j) -> int64_t {  // entry (i, j) of L+U
      const int64_t I = S.sup_of[i], J = S.sup_of[j];
      if (I == J) return S.sn_offset[J] + (i - first[J]) + (j - first[J]) * S.sn_width[J];
      if (I > J) {  // L_{i,j}: L panel of J
        const int64_t cl = S.rows_ptr[J + 1] - S.rows_ptr[J];
        const int64_t pos = find_pos(S.rows.data() + S.rows_ptr[J], S.rows.data() + S.rows_ptr[J + 1], i);
        if (pos < 0) return -1;
        return S.sn_offset[J] + S.sn_width[J] * S.sn_width[J] + pos + (j - first[J]) * cl;
      }
      // U_{i,j}: U^T panel of I
      const int64_t cl = S.rows_ptr[I + 1] - S.rows_ptr[I], cu = S.urows_ptr[I + 1] - S.urows_ptr[I];
      const int64_t pos =
          find_pos(S.urows.data() + S.urows_ptr[I], S.urows.data() + S.urows_ptr[I + 1], j);
      if (pos < 0) return -1;
      return S.sn_offset[I] + S.sn_width[I] * S.sn_width[I] + cl * S.sn_width[I] + pos +
             (i - first[I]) * cu;
    };
    S.value_map.resize(nnz);
    S.inv_map.resize(nnz);
    for (int64_t oc = 0; oc < n; oc++)
      for (int64_t p = colptr[oc]; p < colptr[oc + 1]; p++) {
        const int64_t i = S.irperm[rowind[p]], k = S.iperm[oc];
        S.value_map[p] = slot_lu(i, k);
        // (Atilde^{-1})_{k,i} is stored where (L+U)_{i,k} is, but transposed
        // inside the blocks: the diagonal block holds Ainv_KK itself, the L
        // panel of J holds Ainv(J, R_L(J))^T, the U^T panel Ainv(R_U(J), J)
        const int64_t I = S.sup_of[i], Kk = S.sup_of[k];
        int64_t slot;
        if (I == Kk) {
          slot = S.sn_offset[I] + (k - first[I]) + (i - first[I]) * S.sn_width[I];
        } else {
          slot = S.value_map[p];
        }
        if (S.value_map[p] < 0) return PSELINV_ERR_ARG;
        S.inv_map[p] = slot;
      }
    return PSELINV_OK;
  } catch (const std::bad_alloc&) {
    return PSELINV_ERR_OOM;
  }
}

}  // namespace pselinv
