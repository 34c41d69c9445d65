// Fill-reducing ordering by nested dissection of the graph of A (host only).
//
// The paper takes its orderings from graph partitioners (Section 4); this
// is the automatic nested dissection of George and Liu (Computer Solution
// of Large Sparse Positive Definite Systems, 1981, ch. 8): a part of the
// graph is split by a separator drawn from the rooted level structure of a
// pseudo-peripheral vertex, the two sides are ordered first and the
// separator after them, recursively, down to parts of at most `leaf`
// vertices.  Written here from that description:
//   * parts are processed from an explicit stack; each owns a contiguous
//     range of positions of the new order and puts its separator at the end
//     of the range, so every separator follows the parts it separates;
//   * a disconnected part becomes one part per connected component;
//   * pseudo-peripheral vertex: from a vertex of least degree, repeatedly
//     re-root the level structure at a least-degree vertex of its last
//     level while that makes the structure deeper;
//   * separator: a level strictly inside the structure, restricted to the
//     vertices that have a neighbour in the next level (the rest of that
//     level stays with the lower side): the smallest such separator among
//     the levels that leave at least a fifth of the part on each side,
//     else the level where the count of vertices up to it reaches half;
//   * a part at most `leaf` large, or too shallow to split (fewer than three
//     levels), is ordered by its breadth-first order.
#include <algorithm>
#include <cstdlib>
#include <new>
#include <utility>
#include <vector>

#include "pselinv.h"

namespace {

struct Graph {
  std::vector<int64_t> ptr, adj;  // symmetric adjacency without the diagonal
};

// Breadth-first search of the part tagged `tag` from `root`; fills `order`
// (visit order) and `lev` (level of every visited vertex); returns the
// number of levels.
int64_t bfs(const Graph& g, const std::vector<int64_t>& part, int64_t tag, int64_t root,
            std::vector<int64_t>& lev, std::vector<int64_t>& order, std::vector<int64_t>& seen,
            int64_t stamp) {
  order.clear();
  order.push_back(root);
  seen[root] = stamp;
  lev[root] = 0;
  int64_t depth = 1;
  for (size_t h = 0; h < order.size(); h++) {
    const int64_t v = order[h];
    for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; p++) {
      const int64_t u = g.adj[p];
      if (part[u] != tag || seen[u] == stamp) continue;
      seen[u] = stamp;
      lev[u] = lev[v] + 1;
      depth = std::max(depth, lev[u] + 1);
      order.push_back(u);
    }
  }
  return depth;
}

int64_t degree_in(const Graph& g, const std::vector<int64_t>& part, int64_t tag, int64_t v) {
  int64_t d = 0;
  for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; p++) d += part[g.adj[p]] == tag;
  return d;
}

}  // namespace

extern "C" int pselinv_order_nd(int64_t n, const int64_t* colptr, const int64_t* rowind,
                                int64_t leaf, int64_t* perm_out) {
  if (n < 0 || !colptr || (n > 0 && (!rowind || !perm_out)) || leaf < 1) return PSELINV_ERR_ARG;
  try {
    if (colptr[0] != 0) return PSELINV_ERR_ARG;
    for (int64_t j = 0; j < n; j++) {
      if (colptr[j + 1] < colptr[j]) return PSELINV_ERR_ARG;
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) {
        if (rowind[p] < 0 || rowind[p] >= n) return PSELINV_ERR_ARG;
        if (p > colptr[j] && rowind[p] <= rowind[p - 1]) return PSELINV_ERR_ARG;
      }
    }
    const int64_t nnz = colptr[n];
    // the pattern must equal its transpose (then the columns are the
    // adjacency lists)
    {
      std::vector<int64_t> tptr(n + 1, 0), tidx(nnz), fill(n);
      for (int64_t p = 0; p < nnz; p++) tptr[rowind[p] + 1]++;
      for (int64_t j = 0; j < n; j++) tptr[j + 1] += tptr[j];
      for (int64_t j = 0; j < n; j++) fill[j] = tptr[j];
      for (int64_t j = 0; j < n; j++)
        for (int64_t p = colptr[j]; p < colptr[j + 1]; p++) tidx[fill[rowind[p]]++] = j;
      if (!std::equal(tptr.begin(), tptr.end(), colptr) ||
          !std::equal(tidx.begin(), tidx.end(), rowind))
        return PSELINV_ERR_NOT_STRUCT_SYM;
    }
    Graph g;
    g.ptr.assign(n + 1, 0);
    g.adj.reserve(nnz);
    for (int64_t j = 0; j < n; j++) {
      for (int64_t p = colptr[j]; p < colptr[j + 1]; p++)
        if (rowind[p] != j) g.adj.push_back(rowind[p]);
      g.ptr[j + 1] = (int64_t)g.adj.size();
    }

    std::vector<int64_t> part(n, 0), seen(n, -1), lev(n, 0), order, comp;
    int64_t tags = 0, stamps = 0;
    struct Part {
      std::vector<int64_t> v;
      int64_t lo;  // first position of the part's range
    };
    std::vector<Part> stack;
    {
      Part all;
      all.v.resize(n);
      for (int64_t i = 0; i < n; i++) all.v[i] = i;
      all.lo = 0;
      if (n > 0) stack.push_back(std::move(all));
    }
    while (!stack.empty()) {
      Part P = std::move(stack.back());
      stack.pop_back();
      const int64_t tag = ++tags;
      for (int64_t v : P.v) part[v] = tag;
      const int64_t m = (int64_t)P.v.size();
      // connected components of the part, in order of their lowest vertex
      std::vector<std::vector<int64_t>> comps;
      const int64_t stamp = ++stamps;
      std::vector<int64_t> sorted_v = P.v;
      std::sort(sorted_v.begin(), sorted_v.end());
      for (int64_t s0 : sorted_v) {
        if (seen[s0] == stamp) continue;
        comp.clear();
        comp.push_back(s0);
        seen[s0] = stamp;
        for (size_t h = 0; h < comp.size(); h++) {
          const int64_t v = comp[h];
          for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; p++) {
            const int64_t u = g.adj[p];
            if (part[u] == tag && seen[u] != stamp) {
              seen[u] = stamp;
              comp.push_back(u);
            }
          }
        }
        comps.push_back(comp);
      }
      if (comps.size() > 1) {
        int64_t lo = P.lo;
        for (auto& c : comps) {
          Part Q;
          Q.lo = lo;
          lo += (int64_t)c.size();
          Q.v = std::move(c);
          stack.push_back(std::move(Q));
        }
        continue;
      }
      // one connected part: level structure from a pseudo-peripheral vertex
      int64_t root = P.v[0], dmin = -1;
      for (int64_t v : sorted_v) {
        const int64_t d = degree_in(g, part, tag, v);
        if (dmin < 0 || d < dmin) {
          dmin = d;
          root = v;
        }
      }
      int64_t depth = bfs(g, part, tag, root, lev, order, seen, ++stamps);
      for (int it = 0; it < 8 && m > leaf; it++) {
        int64_t cand = -1, cd = -1;
        for (int64_t v : order)
          if (lev[v] == depth - 1) {
            const int64_t d = degree_in(g, part, tag, v);
            if (cand < 0 || d < cd || (d == cd && v < cand)) {
              cand = v;
              cd = d;
            }
          }
        std::vector<int64_t> o2;
        const int64_t d2 = bfs(g, part, tag, cand, lev, o2, seen, ++stamps);
        if (d2 <= depth) {
          bfs(g, part, tag, root, lev, order, seen, ++stamps);  // restore root's levels
          break;
        }
        root = cand;
        depth = d2;
        order.swap(o2);
      }
      if (m <= leaf || depth < 3) {
        for (int64_t i = 0; i < m; i++) perm_out[P.lo + i] = order[i];
        continue;
      }
      // separator level j in [1, depth - 2]: the smallest separator (below)
      // among the levels that leave at least a fifth of the part on each
      // side, else the level where the count reaches half the part
      std::vector<int64_t> cnt(depth, 0), scnt(depth, 0);
      for (int64_t v : order) {
        cnt[lev[v]]++;
        for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; p++) {
          const int64_t u = g.adj[p];
          if (part[u] == tag && lev[u] == lev[v] + 1) {
            scnt[lev[v]]++;
            break;
          }
        }
      }
      int64_t j = 1, acc = cnt[0];
      while (j < depth - 2 && acc + cnt[j] < (m + 1) / 2) acc += cnt[j++];
      {
        int64_t below = cnt[0], best = -1;
        for (int64_t l = 1; l <= depth - 2; l++) {
          const int64_t lower = below + cnt[l] - scnt[l], upper = m - lower - scnt[l];
          below += cnt[l];
          if (5 * std::min(lower, upper) < m) continue;
          if (best < 0 || scnt[l] < scnt[best] ||
              (scnt[l] == scnt[best] && std::llabs(l - j) < std::llabs(best - j)))
            best = l;
        }
        if (best >= 0) j = best;
      }
      // separator: the vertices of level j with a neighbour in level j + 1
      std::vector<int64_t> sep, rest;
      for (int64_t v : order) {
        bool in_sep = false;
        if (lev[v] == j)
          for (int64_t p = g.ptr[v]; p < g.ptr[v + 1] && !in_sep; p++) {
            const int64_t u = g.adj[p];
            in_sep = part[u] == tag && lev[u] == j + 1;
          }
        (in_sep ? sep : rest).push_back(v);
      }
      const int64_t ns = (int64_t)sep.size();
      for (int64_t i = 0; i < ns; i++) perm_out[P.lo + m - ns + i] = sep[i];
      for (int64_t v : sep) part[v] = 0;
      Part R;
      R.lo = P.lo;
      R.v = std::move(rest);
      if (!R.v.empty()) stack.push_back(std::move(R));
    }
    return PSELINV_OK;
  } catch (const std::bad_alloc&) {
    return PSELINV_ERR_OOM;
  }
}
