// Internal declarations shared by the host analysis and the CUDA sources.
#pragma once
#include <cstdint>
#include <vector>

#include "pselinv.h"

namespace pselinv {

// Host-side symbolic structure (permuted indices).  Built by analyze_host().
struct HostSym {
  int64_t n = 0, nnz = 0;
  int64_t max_sn = 256, relax_pct = 20;
  std::vector<int64_t> perm, iperm;
  std::vector<int64_t> etree;     // column elimination tree of the exact fill
  std::vector<int64_t> colcount;  // exact |struct(j)|
  // supernodes
  int64_t ns = 0;
  std::vector<int64_t> sn_first, sn_width, sn_parent, sn_depth, sn_height, sn_offset;
  std::vector<int64_t> rows_ptr, rows;  // R_K
  std::vector<int64_t> sup_of;          // column -> supernode
  // levels: by depth from the roots (selected inversion) and by height
  // from the leaves (factorisation)
  std::vector<int64_t> level_ptr, level_sn;
  std::vector<int64_t> hlevel_ptr, hlevel_sn;
  // block index maps.  R_K is cut into blocks of consecutive rows that fall
  // in the same supernode J.  For block b of K covering positions [pb, pe):
  //   relidx[blk_rel[b] + (p - pb)], p in [pb, c_K):
  //     p <  pe : R_K[p] - first(J)          (local column of row R_K[p] in J)
  //     p >= pe : position of R_K[p] in R_J   (fill argument: R_K[p] in R_J)
  std::vector<int32_t> sn_blk;    // [ns + 1] first block of K
  std::vector<int32_t> blk_sn, blk_pb, blk_pe;
  std::vector<int64_t> blk_rel;
  std::vector<int32_t> rows_blk;  // global block index of each position of each R_K
  std::vector<int32_t> relidx;
  std::vector<int64_t> value_map;  // storage slot of each input entry
  int64_t storage = 0;             // scalars per instance
  // general patterns (analyze_general_host): rows / rows_ptr hold R_L(K)
  // (the L panel's rows) and urows / urows_ptr R_U(K) (the U^T panel's
  // rows, the columns of U right of K), which need not agree.  Row ordering
  // rperm (new -> old; perm above is the column ordering).  Blocks of R_L(K)
  // (blk_*) map the positions of R_U(K) from blk_q0 on (relidx at blk_rel)
  // to the local index in J or the position in R_U(J); blocks of R_U(K)
  // (ublk_*) map the positions of R_L(K) into J / R_L(J).  inv_map: slot of
  // the selected entry (A^{-1})_{col,row} returned for each input entry.
  bool general = false;
  std::vector<int64_t> rperm, irperm;
  std::vector<int64_t> urows_ptr, urows;
  std::vector<int32_t> blk_q0;
  std::vector<int32_t> usn_blk, ublk_sn, ublk_pb, ublk_pe, ublk_q0, urows_blk;
  std::vector<int64_t> ublk_rel;
  std::vector<int64_t> inv_map;
  double flops_selinv = 0, flops_selinv_exact = 0, flops_factor = 0;
};

// Host analysis; returns a PSELINV_* status.  No CUDA calls.
int analyze_host(int64_t n, const int64_t* colptr, const int64_t* rowind, const int64_t* perm,
                 int64_t max_sn, int64_t relax_pct, HostSym& out);
// The same for a general pattern with row ordering rperm and column
// ordering cperm (static pivoting, P A Q with P != Q^T).
int analyze_general_host(int64_t n, const int64_t* colptr, const int64_t* rowind,
                         const int64_t* rperm, const int64_t* cperm, int64_t max_sn,
                         int64_t relax_pct, HostSym& out);

}  // namespace pselinv
