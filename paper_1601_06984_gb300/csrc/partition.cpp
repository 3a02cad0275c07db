// Halo plan of a partitioned mesh (Sec. 3.1 weight-based decomposition along
// the space-filling curve, Sec. 3.2 halo elements), host only.
//
// Given the owner of every element (for instance the split of
// lbm_sfc_partition), the part `rank` computes its own fluid elements and the
// ghost elements they depend on.  What it must receive from other parts are
// the fluid elements those computations read: the pull sources of its
// stream-collide (including the second node of interpolated bounce-back and
// the outlet's extrapolation sources), the GhostFromCoarser sources and the
// GhostFromFiner children of the ghosts it fills, and the pull sources of the
// ghosts the time mode advances (the inner GhostFromFiner layer in
// LBM_TIME_LINEAR, the inner GhostFromCoarser layer in LBM_TIME_TWO_LAYER, the
// inner three of the four GhostFromCoarser layers in LBM_TIME_DIFFUSIVE).
// Every such read takes the current state of the read element's level, so one
// exchange of a level's halo after each stream-collide of that level (and one
// after lbm_init) keeps every read current.  Ghosts are computed by every
// part that needs them; their inputs being the same, so are their values.
#include <algorithm>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_internal.h"

using namespace lbm;

extern "C" lbm_status lbm_halo_plan(const lbm_ctx* c, const int32_t* part, int32_t nparts, int32_t rank,
                                    int64_t* recv_count, int64_t* recv, int64_t recv_cap, int64_t* n_ghosts,
                                    int64_t* ghosts, int64_t ghost_cap) {
  if (!c || !part || nparts < 1 || rank < 0 || rank >= nparts || !recv_count || !n_ghosts) return LBM_ERR_ARG;
  if (recv_cap < 0 || ghost_cap < 0 || (recv_cap > 0 && !recv) || (ghost_cap > 0 && !ghosts)) return LBM_ERR_ARG;
  const HostMesh& M = c->M;
  if (M.lv.empty()) return LBM_ERR_STATE;
  const int64_t n = M.n_user, Ntot = M.Ntot;
  const int Q = M.Q, nch = 1 << M.d;
  for (int64_t u = 0; u < n; ++u)
    if (part[u] < 0 || part[u] >= nparts) return LBM_ERR_ARG;
  const bool linear = c->p.time_mode == LBM_TIME_LINEAR;
  // GhostFromCoarser layers whose advanced values reach fluid
  const int gfc_adv = c->p.time_mode == LBM_TIME_DIFFUSIVE ? 3 : 1;
  // per slot: level index, position within its level's ghost rows (-1: not a ghost)
  std::vector<int8_t> lev(Ntot, -1);
  std::vector<int64_t> ghost_row(Ntot, -1);
  int64_t row0 = 0;
  for (int li = 0; li < (int)M.lv.size(); ++li) {
    const HostLevel& H = M.lv[li];
    for (int64_t e = 0; e < H.N; ++e) lev[H.base + e] = (int8_t)li;
    for (int64_t k = 0; k < H.nC; ++k) ghost_row[H.base + H.oC + k] = row0 + k;
    for (int64_t k = 0; k < H.nG1; ++k) ghost_row[H.base + H.oG1 + k] = row0 + H.nC + k;
    for (int64_t k = 0; k < H.nG2; ++k) ghost_row[H.base + H.oG2 + k] = row0 + H.nC + H.nG1 + k;
    row0 += H.nC + H.nG1 + H.nG2;
  }
  // boundary-value index -> extrapolation / second-node sources
  std::vector<uint8_t> computed(Ntot, 0), halo(n, 0);
  std::vector<int64_t> work;
  auto read = [&](int64_t slot) {
    if (slot < 0 || slot >= Ntot) return;
    const uint8_t k = M.kind[slot];
    if (k == K_FLUID) {
      const int32_t u = M.slot_user[slot];
      if (u >= 0 && part[u] != rank) halo[u] = 1;
    } else if ((k == K_GFC || k == K_GFF) && !computed[slot]) {
      computed[slot] = 1;
      work.push_back(slot);
    }
  };
  // the pull sources of an element the stream-collide processes
  auto pulls = [&](int64_t slot) {
    for (int i = 1; i < Q; ++i) {
      const uint32_t code = M.nbr[(size_t)(i - 1) * Ntot + slot];
      if (code < NB_FLAG30) {
        read((int64_t)code);
      } else if (!(code & NB_BOUNCE)) {  // boundary value: outlet or interpolated bounce-back
        const int64_t v = code & NB_INDEX;
        read(M.out_a[v]);
        read(M.out_b[v]);
      }
    }
  };
  for (int64_t u = 0; u < n; ++u)
    if (part[u] == rank) {
      computed[M.uslot[u]] = 1;
      pulls(M.uslot[u]);
    }
  while (!work.empty()) {
    const int64_t g = work.back();
    work.pop_back();
    const HostLevel& H = M.lv[lev[g]];
    const int64_t e = g - H.base;
    if (M.kind[g] == K_GFC) {
      const int64_t k = e - H.oC;
      const HostLevel& Hc = M.lv[lev[g] - 1];
      for (int s = 0; s < 4; ++s) read(Hc.src_elem[H.gfc_src[(size_t)s * H.nC + k]]);
      if (!linear && H.ghost_layer[k] <= gfc_adv) pulls(g);  // advanced by the fine stream-collide
    } else {
      const bool inner = e >= H.oG1 && e < H.oG1 + H.nG1;
      const int64_t k = inner ? e - H.oG1 : H.nG1 + (e - H.oG2);
      for (int b = 0; b < nch; ++b) read((int64_t)H.gff_child0[k] + b);
      if (linear && inner) pulls(g);  // advanced by the coarse stream-collide
    }
  }
  // receive lists: by sending part, caller indices ascending
  std::fill(recv_count, recv_count + nparts, 0);
  for (int64_t u = 0; u < n; ++u)
    if (halo[u]) recv_count[part[u]]++;
  std::vector<int64_t> start(nparts + 1, 0);
  for (int p = 0; p < nparts; ++p) start[p + 1] = start[p] + recv_count[p];
  if (recv_cap > 0) {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t u = 0; u < n; ++u)
      if (halo[u]) {
        const int64_t pos = fill[part[u]]++;
        if (pos < recv_cap) recv[pos] = u;
      }
  }
  int64_t ng = 0;
  for (int64_t s = 0; s < Ntot; ++s)
    if (computed[s] && ghost_row[s] >= 0) {
      if (ng < ghost_cap) ghosts[ng] = ghost_row[s];
      ++ng;
    }
  if (ng <= ghost_cap) std::sort(ghosts, ghosts + ng);
  *n_ghosts = ng;
  return LBM_OK;
}
