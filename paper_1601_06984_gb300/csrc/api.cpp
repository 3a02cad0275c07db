// C ABI of liblbm (include/lbm.h): context, device workspace layout, the
// recursive level time stepping driver (Sec. 2.2) and the host<->device
// transfers of the public calls.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_ctx.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }


}  // namespace

using lbm::LevelDev;

void lbm_ctx::layout() {
  const HostMesh& m = M;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += align_up(std::max<size_t>(b, 1));
    return r;
  };
  const size_t sb = ops->storage_bytes, cb = ops->compute_bytes;
  const size_t N = (size_t)m.Ntot;
  oA = take(Q * N * sb);
  oB = take(Q * N * sb);
  oNbr = take((size_t)(Q - 1) * N * 4);
  oBrickNb = take(m.brick_nb.size() * 4);
  oBrickTab = take(m.brick_tab.size() * 2);
  oInletS = take(m.inlet_s.size() * 8);
  oOutQ = take(m.out_q.size() * 8);
  oObsA = take(m.obs_a.size() * 4);
  oObsQ = take(m.obs_q.size() * 8);
  oF = p.use_force ? take((size_t)d * N * cb) : 0;
  ld.assign(nlev, LevelDev());
  const size_t M_ = mom_stride(Q);
  for (int li = 0; li < nlev; ++li) {
    const HostLevel& H = m.lv[li];
    LevelDev& L = ld[li];
    L.gff_child0 = take(H.gff_child0.size() * 4);
    L.gfc_src = take(H.gfc_src.size() * 4);
    L.gfc_oct = take(H.gfc_oct.size());
    L.src_elem = take(H.src_elem.size() * 4);
    L.nsrc = (int64_t)H.src_elem.size();
    L.gsrc_elem = take(H.gsrc_elem.size() * 4);
    L.gsrc_rec = take(H.gsrc_rec.size() * 4);
    L.n_gsrc = (int64_t)H.gsrc_elem.size();
    L.n_gsrc_inner = H.n_gsrc_inner;
    L.momA[0] = take(M_ * L.nsrc * cb);
    L.momA[1] = take(M_ * L.nsrc * cb);
  }
  const size_t nout = m.out_elem.size(), nobs = m.obs_elem.size();
  oOutElem = take(nout * 4);
  oOutA = take(nout * 4);
  oOutB = take(nout * 4);
  oOutDir = take(nout);
  oOutKind = take(nout);
  oSide = take(nout * cb);
  oObsElem = take(nobs * 4);
  oObsDir = take(nobs);
  oUslot = take((size_t)m.n_user * 4);
  oUlev = take((size_t)m.n_user);
  oSlotUser = take((size_t)N * 4);
  oSrcMask = take(m.src_mask.size() * 4);
  oSrcFirst = take(m.src_first.size() * 4);
  chunk = std::min<int64_t>(m.n_user, (int64_t)1 << 20);
  oStage = take((size_t)chunk * (1 + d + nS + Q + Q) * 8);
  oPartial = take((size_t)nlev * kReduceBlocks * 8 * 8);
  oRed = take(8 * 8);
  bytes = o;
}

// ---------------------------------------------------------------- driver
void lbm_ctx::fill_gff(int li) {
  const HostLevel& H = M.lv[li];
  const HostLevel& Hf = M.lv[li + 1];
  if (H.nG1 + H.nG2 == 0) return;
  GffArgs a{};
  a.src_fine = cur(li + 1);
  a.force = force_ptr();
  a.child0 = at<int32_t>(ld[li].gff_child0);
  a.ng = H.nG1 + H.nG2;
  a.n_inner = H.nG1;
  a.dest0 = H.base + H.oG1;
  a.dest_outer = H.base + H.oG2;
  a.dst = cur(li);
  a.Ntot = M.Ntot;
  a.omega_c = H.omega;
  a.omega_f = Hf.omega;
  a.rho_off = rho_off;
  // fine -> coarse lattice units: u_c = (dt_c / dt_f) / 2 u_f, the density
  // deviation with the square of that factor (1 in acoustic scaling)
  a.tratio = time_ratio(p.time_mode);
  a.u_scale = a.tratio / 2.0;
  a.r_scale = a.u_scale * a.u_scale;
  a.r_shift = (1.0 - a.r_scale) * (p.rho0 - rho_off);
  a.odd_ratio = odd_fneq_ratio(p.time_mode, true);
  timed_launch(li, TK_GFF, [&] { ops->fill_gff(Q, a, st); });
  ++launches;
}

void lbm_ctx::source_moments(int li, size_t mom_off, size_t prev_off, cudaStream_t s, int subset) {
  const LevelDev& L = ld[li];
  const int64_t n = subset == SRC_ALL ? L.nsrc : subset == SRC_GFF ? L.n_gsrc : L.n_gsrc - L.n_gsrc_inner;
  if (n == 0) return;
  if (!s) s = st;
  MomentsArgs a{};
  a.src = cur(li);
  a.force = force_ptr();
  if (subset == SRC_ALL) {
    a.elem = at<int32_t>(L.src_elem);
  } else {
    const int64_t skip = subset == SRC_GFF ? 0 : L.n_gsrc_inner;
    a.elem = at<int32_t>(L.gsrc_elem) + skip;
    a.rec = at<int32_t>(L.gsrc_rec) + skip;
  }
  a.mom = at(mom_off);
  a.prev = prev_off ? at(prev_off) : nullptr;
  a.Ntot = M.Ntot;
  a.nsrc = n;
  a.omega = M.lv[li].omega;
  a.rho_off = rho_off;
  timed_launch(li, TK_MOM, [&] { ops->source_moments(Q, a, s); }, s);
  ++launches;
}

void lbm_ctx::fill_gfc(int lf, bool two_times, bool all_layers, cudaStream_t s, bool next_buffer) {
  const HostLevel& H = M.lv[lf];
  if (H.nC == 0) return;
  if (!s) s = st;
  const int lc = lf - 1;
  GfcArgs a{};
  // at t + 1/2 (after the coarse stream-collide): the means of the records
  // at t and t + 1, which the two buffers hold
  a.mom = at(ld[lc].momA[parity[lc] ^ (two_times ? 1 : 0)]);
  a.mom2 = two_times ? at(ld[lc].momA[parity[lc]]) : nullptr;
  a.nsrc = ld[lc].nsrc;
  a.gsrc = at<int32_t>(ld[lf].gfc_src);
  a.oct = at<uint8_t>(ld[lf].gfc_oct);
  a.ng = H.nC;
  a.dest0 = H.base + H.oC;
  a.dst = next_buffer ? nxt(lf) : cur(lf);
  a.Ntot = M.Ntot;
  a.omega_c = M.lv[lc].omega;
  a.omega_f = H.omega;
  a.rho_off = rho_off;
  a.skip_outer = !all_layers && p.time_mode == LBM_TIME_LINEAR;
  // coarse -> fine lattice units, the inverse of the GhostFromFiner conversion
  a.tratio = time_ratio(p.time_mode);
  a.u_scale = 2.0 / a.tratio;
  a.r_scale = a.u_scale * a.u_scale;
  a.r_shift = (1.0 - a.r_scale) * (p.rho0 - rho_off);
  a.odd_ratio = odd_fneq_ratio(p.time_mode, false);
  timed_launch(lf, TK_GFC, [&] { ops->fill_gfc(Q, a, s); }, s);
  ++launches;
}

void lbm_ctx::stream_collide(int li, cudaStream_t s0) {
  if (!s0) s0 = st;
  const HostLevel& H = M.lv[li];
  if (H.out_end > H.out_begin) {
    OutletArgs o{};
    o.src = cur(li);
    o.side = at(oSide);
    o.elem = at<int32_t>(oOutElem);
    o.a = at<int32_t>(oOutA);
    o.b = at<int32_t>(oOutB);
    o.dir = at<int8_t>(oOutDir);
    o.kind = at<int8_t>(oOutKind);
    o.force = force_ptr();
    o.Ntot = M.Ntot;
    o.begin = H.out_begin;
    o.end = H.out_end;
    o.omega = H.omega;
    o.rho_off = rho_off;
    o.rho0 = p.rho0;
    o.zero_gradient = p.outlet == LBM_OUTLET_ZERO_GRADIENT;
    o.q = at<double>(oOutQ);
    timed_launch(li, TK_OUTLET, [&] { ops->outlet(Q, o, s0); }, s0);
    ++launches;
  }
  // interior bricks, then boundary bricks (the first 64 (nB + nBb) fluid
  // elements) through the brick tables
  const int64_t nbnd = ops->boundary_bricks ? H.nBb : 0;
  const int64_t nbrick = 64 * (H.nB + nbnd);
  BrickArgs b{};
  b.src = cur(li);
  b.dst = nxt(li);
  b.force = force_ptr();
  b.nb = at<int32_t>(oBrickNb) + (size_t)H.brick_first * 27;
  b.tab = at<uint16_t>(oBrickTab);
  b.Ntot = M.Ntot;
  b.begin = H.base + H.oF;
  b.nB = H.nB;
  b.omega = H.omega;
  b.rho_off = rho_off;
  b.nbr = at<uint32_t>(oNbr);
  b.side = at(oSide);
  b.inlet_s = at<double>(oInletS);
  // the inlet velocity in this level's lattice units
  const double uin_unit = level_velocity_ratio(li, p.time_mode);
  for (int i = 0; i < kQmax; ++i) b.inlet[i] = inlet[i] * uin_unit;
  // the level's GFC source records at t + 1 from the new state
  SourceOut so{};
  if (li + 1 < nlev && ld[li].nsrc > 0) {
    so.mask = at<uint32_t>(oSrcMask);
    so.first = at<int32_t>(oSrcFirst);
    so.rec_out = at(ld[li].momA[parity[li] ^ 1]);
  }
  b.so = so;
  BrickArgs bb = b;
  bb.nb = b.nb + (size_t)H.nB * 27;
  bb.begin = b.begin + 64 * H.nB;
  bb.nB = nbnd;
  // the rest through the neighbour list; processed range: TWO_LAYER and
  // DIFFUSIVE [GFC | fluid], LINEAR [fluid | GFF inner], minus the bricks
  StreamCollideArgs a{};
  a.src = cur(li);
  a.dst = nxt(li);
  a.nbr = at<uint32_t>(oNbr);
  a.force = force_ptr();
  a.side = at(oSide);
  a.inlet_s = at<double>(oInletS);
  a.Ntot = M.Ntot;
  if (p.time_mode != LBM_TIME_LINEAR) {
    a.begin = H.base + H.oC;
    a.end = H.base + H.oG1 - nbrick;
    a.hole_at = H.base + H.oF;
    a.hole_len = nbrick;
  } else {
    a.begin = H.base + H.oF + nbrick;
    a.end = H.base + H.oG2;
    a.hole_at = a.end;
    a.hole_len = 0;
  }
  a.omega = H.omega;
  a.rho_off = rho_off;
  std::memcpy(a.inlet, b.inlet, sizeof(a.inlet));
  a.so = so;
  const bool use_force = p.use_force != 0;
  auto launch = [&](int kernel, cudaStream_t s) {
    if (kernel == TK_INTERIOR) ops->stream_collide_brick(Q, use_force, false, b, s);
    else if (kernel == TK_BOUNDARY) ops->stream_collide_brick(Q, use_force, true, bb, s);
    else ops->stream_collide(Q, use_force, a, s);
    ++launches;
  };
  const bool has[3] = {b.nB > 0, a.end > a.begin, bb.nB > 0};  // by TimedKind 0..2
  // inside a graph capture the kernels run as parallel branches (boundary
  // bricks and neighbour list on the level's two side streams), joined before
  // the next op; launched kernel by kernel they run one after the other
  const bool fork = capturing && concurrent_sc && timing != 1 && !lvs.empty() && (has[TK_BOUNDARY] || has[TK_LIST]);
  auto group = [&] {
    if (fork) {
      cudaEventRecord(lvs[li].fork, s0);
      cudaStreamWaitEvent(lvs[li].side[0], lvs[li].fork, 0);
      cudaStreamWaitEvent(lvs[li].side[1], lvs[li].fork, 0);
    }
    for (int kernel : {TK_INTERIOR, TK_BOUNDARY, TK_LIST}) {
      if (!has[kernel]) continue;
      cudaStream_t s = !fork || kernel == TK_INTERIOR ? s0 : lvs[li].side[kernel == TK_BOUNDARY ? 0 : 1];
      timed_launch(li, kernel, [&] { launch(kernel, s); }, s);
    }
    if (fork) {
      for (int k = 0; k < 2; ++k) {
        cudaEventRecord(lvs[li].join[k], lvs[li].side[k]);
        cudaStreamWaitEvent(s0, lvs[li].join[k], 0);
      }
    }
  };
  // the whole level's stream-collide (fork to join) as one timed span
  timed_launch(li, TK_SC_SPAN, group, s0);
  parity[li] ^= 1;
}

void lbm_ctx::ensure_records() {
  if (recs_valid || dry) return;
  for (int li = 0; li + 1 < nlev; ++li) source_moments(li, ld[li].momA[parity[li]]);
  recs_valid = true;
}

void lbm_ctx::advance(int li) {
  const bool has_finer = li + 1 < nlev;
  const bool linear = p.time_mode == LBM_TIME_LINEAR;
  auto op = [&](int kind, int level) {
    if (hook) hook(kind, level);
    return !dry;
  };
  // Source records (interpolation step 1), two buffers per level: momA[parity]
  // holds those of the current state.  The stream-collide writes the records
  // of the sources it updates into the other buffer (their state at t + 1);
  // the GhostFromFiner sources get theirs at t after their fill, and in
  // LINEAR mode the outer GhostFromFiner layer, which no stream-collide
  // updates, at t + 1 from its stored state.  The fill at t + 1/2 takes the
  // means of the two buffers.
  // In a graph capture the level's stream-collide becomes a branch of its
  // own, forked after the GhostFromFiner fill (the last op it needs) and
  // joined before the finer level's second substep; meanwhile the records at
  // t, the finer level's GhostFromCoarser fill and its first substep run on
  // the main branch (they read this level's current buffer, its records at t
  // or other levels only).  With gfc_b_branch the finer level's fill at
  // t + 1/2 follows the stream-collide on its branch (forked after the
  // records at t), into the fine buffer that the first substep's
  // stream-collide writes, whose ghost slots nothing touches before the
  // second substep.
  const bool branch = has_finer && capturing && concurrent_sc && level_branch && timing != 1 && !lvs.empty() && !dry;
  const bool gfc_b_on_branch = branch && linear && gfc_b_branch;
  if (has_finer) {
    if (op(OP_GFF, li)) fill_gff(li);
    if (branch && !gfc_b_on_branch) cudaEventRecord(lvs[li].fork_sc, st);
    if (op(OP_MOM_A, li)) source_moments(li, ld[li].momA[parity[li]], 0, nullptr, SRC_GFF);
    if (gfc_b_on_branch) cudaEventRecord(lvs[li].fork_sc, st);
    if (op(OP_GFC_A, li + 1)) fill_gfc(li + 1, false);
  }
  if (op(OP_SC, li)) {
    if (branch) {
      cudaStreamWaitEvent(lvs[li].sc, lvs[li].fork_sc, 0);
      stream_collide(li, lvs[li].sc);
      if (gfc_b_on_branch) {
        source_moments(li, ld[li].momA[parity[li]], 0, lvs[li].sc, SRC_GFF_OUTER);
        fill_gfc(li + 1, true, false, lvs[li].sc, true);
      }
    } else {
      stream_collide(li);
    }
  } else {
    parity[li] ^= 1;
  }
  if (has_finer) {
    advance(li + 1);
    if (branch) {
      cudaEventRecord(lvs[li].done_sc, lvs[li].sc);
      cudaStreamWaitEvent(st, lvs[li].done_sc, 0);
    }
    if (linear) {
      if (op(OP_MOM_B, li) && !gfc_b_on_branch)
        source_moments(li, ld[li].momA[parity[li]], 0, nullptr, SRC_GFF_OUTER);
      if (op(OP_GFC_B, li + 1) && !gfc_b_on_branch) fill_gfc(li + 1, true);
    }
    // the remaining substeps (one in acoustic scaling; three with diffusive
    // scaling, whose four ghost layers filled at t last all four)
    for (int k = 1; k < time_ratio(p.time_mode); ++k) advance(li + 1);
  }
}

bool lbm_ctx::make_level_streams() {
  if (!lvs.empty()) return true;
  std::vector<LevelStreams> v(nlev);
  bool ok = true;
  for (auto& L : v) {
    for (cudaStream_t* s : {&L.sc, &L.side[0], &L.side[1]})
      ok = ok && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t* e : {&L.fork_sc, &L.done_sc, &L.fork, &L.join[0], &L.join[1]})
      ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  }
  lvs.swap(v);  // created handles are released by the destructor either way
  if (!ok) cudaGetLastError();
  return ok;
}

const lbm_ctx::StepGraph* lbm_ctx::step_graph(int nsteps) {
  for (const StepGraph& g : graphs)
    if (g.parity == parity && g.steps == nsteps) return &g;
  if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    graphs_on = false;
    return nullptr;
  }
  // no branch streams: the captured steps stay sequential
  if (concurrent_sc && !make_level_streams()) concurrent_sc = false;
  // capture on a private stream (the bound stream may be the legacy default
  // stream, which cannot be captured); host bookkeeping is restored afterwards
  const std::vector<int> p0 = parity;
  const int64_t l0 = launches;
  if (timing == 2) {
    // events for the finest level's stream-collide launches and their span
    // (up to four pairs per substep, m^(nlev-1) substeps per coarse step, m
    // the time-step ratio), made before the capture begins (at most 2^16;
    // further ones are made as they are needed)
    int64_t nev = (int64_t)nsteps * 4 * 2;
    for (int li = 1; li < nlev && nev < (1 << 16); ++li) nev *= time_ratio(p.time_mode);
    for (int64_t k = 0; k < std::min<int64_t>(nev, 1 << 16); ++k) event_pool.push_back(get_event());
  }
  const size_t t0 = timed.size();
  cudaStream_t user = st;
  st = cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    capturing = true;
    for (int k = 0; k < nsteps; ++k) advance(0);
    capturing = false;
    e = cudaStreamEndCapture(cap_stream, &graph);
  }
  st = user;
  std::vector<Timed> gt(timed.begin() + t0, timed.end());
  timed.resize(t0);
  const int64_t nl = launches - l0;
  launches = l0;
  // two steps bring every level back to its buffer; one step flips the
  // coarsest level's (the finer levels take an even number of substeps)
  std::vector<int> expect = p0;
  if (nsteps == 1) expect[0] ^= 1;
  const std::vector<int> p1 = parity;
  const bool same = p1 == expect;
  parity = p0;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && graph && same) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || !exec || !same) {
    cudaGetLastError();
    for (auto& t : gt) {
      event_pool.push_back(t.a);
      event_pool.push_back(t.b);
    }
    graphs_on = false;
    return nullptr;
  }
  graphs.push_back({p0, p1, nsteps, exec, nl, std::move(gt)});
  return &graphs.back();
}

// ---------------------------------------------------------------- internal accessors
namespace lbm {

lbm_status reduce_plan(lbm_ctx* c, ReducePlan* plan) {
  if (!c || !plan) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "reduction before lbm_bind");
  plan->ops = c->ops;
  plan->Q = c->Q;
  plan->stream = c->st;
  plan->workspace = c->ws;
  plan->levels.clear();
  const int d = c->d;
  for (int li = 0; li < c->nlev; ++li) {
    const HostLevel& H = c->M.lv[li];
    ReduceArgs a{};
    a.pdf = c->cur(li);
    a.force = c->force_ptr();
    a.Ntot = c->M.Ntot;
    a.begin = H.base + H.oF;
    a.end = H.base + H.oF + H.nF;
    a.omega = H.omega;
    a.rho_off = c->rho_off;
    a.vol = std::ldexp(1.0, -d * li);
    // diffusive scaling: mass, momentum and kinetic energy in the coarsest
    // level's units (a lattice velocity of level li is 2^li of the
    // coarsest's), forces in the finest level's (a force unit goes with
    // dx^(d+1) / dt^2)
    const double us = 1.0 / level_velocity_ratio(li, c->p.time_mode);
    a.vol_m = a.vol * us;
    a.vol_k = a.vol * us * us;
    a.r_scale = us * us;
    a.rho0 = c->p.rho0;
    a.partial = nullptr;
    a.nblocks = kReduceBlocks;
    a.obs_elem = c->at<int32_t>(c->oObsElem) + H.obs_begin;
    a.obs_dir = c->at<int8_t>(c->oObsDir) + H.obs_begin;
    a.obs_a = c->at<int32_t>(c->oObsA) + H.obs_begin;
    a.obs_q = c->at<double>(c->oObsQ) + H.obs_begin;
    a.obs_n = H.obs_end - H.obs_begin;
    a.fscale = std::ldexp(1.0, (c->p.time_mode == LBM_TIME_DIFFUSIVE ? d - 3 : d - 1) * (c->nlev - 1 - li));
    plan->levels.push_back(a);
  }
  return LBM_OK;
}

lbm_status set_error(lbm_ctx* c, lbm_status s, const std::string& msg) { return c->fail(s, msg); }

void count_launches(lbm_ctx* c, int64_t n) { c->launches += n; }

}  // namespace lbm

// ---------------------------------------------------------------- C ABI
extern "C" {

lbm_status lbm_build_mesh(const int64_t* tree_ids, const int8_t* levels, int64_t n, const lbm_params* params,
                          lbm_ctx** out) {
  if (!out || !params) return LBM_ERR_ARG;
  *out = nullptr;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_OOM;
  c->p = *params;
  if (params->precision == LBM_FP64) c->ops = ops_fp64();
  else if (params->precision == LBM_FP32DEV) c->ops = ops_fp32dev();
  else if (params->precision == LBM_BF16DEV) c->ops = ops_bf16dev();
  else {
    c->err = "bad precision";
    *out = c;
    return LBM_ERR_ARG;
  }
  if (params->outlet != LBM_OUTLET_LINEAR && params->outlet != LBM_OUTLET_ZERO_GRADIENT) {
    c->err = "bad outlet extrapolation";
    *out = c;
    return LBM_ERR_ARG;
  }
  if (params->check_every < 0 || !(params->mass_band >= 0.0) || !std::isfinite(params->mass_band)) {
    c->err = "check_every must be >= 0 and mass_band finite and >= 0";
    *out = c;
    return LBM_ERR_ARG;
  }
  if (params->adjoint_tape < 0 || params->adjoint_tape > 2) {
    c->err = "adjoint_tape must be 0, 1 or 2";
    *out = c;
    return LBM_ERR_ARG;
  }
  lbm_status s;
  try {
    s = build_host_mesh(tree_ids, levels, n, c->p, &c->M, &c->err);
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    s = LBM_ERR_OOM;
  }
  *out = c;
  if (s != LBM_OK) return s;
  c->Q = c->M.Q;
  c->d = c->M.d;
  c->nS = c->M.nS;
  c->nlev = (int)c->M.lv.size();
  c->rho_off = params->precision == LBM_FP64 ? 0.0 : params->rho0;
  int cc[kQmax][3];
  double w[kQmax];
  host_lattice(c->Q, cc, w);
  for (int i = 0; i < c->Q; ++i) {
    double cu = 0;
    for (int a = 0; a < c->d; ++a) cu += cc[i][a] * params->u_in[a];
    c->inlet[i] = 6.0 * w[i] * params->rho0 * cu;
  }
  c->layout();
  c->parity.assign(c->nlev, 0);
  return LBM_OK;
}

lbm_status lbm_mesh_info(const lbm_ctx* c, int64_t* info, int32_t cap, int32_t* nlevels) {
  if (!c || !info) return LBM_ERR_ARG;
  int n = 0;
  for (const HostLevel& H : c->M.lv) {
    if (n >= cap) break;
    int64_t r[10] = {H.L, H.nF, H.nC, H.nG1, H.nG2, H.N, H.out_end - H.out_begin, H.obs_end - H.obs_begin,
                     H.nB, H.nBb};
    std::memcpy(info + 10 * n, r, sizeof(r));
    ++n;
  }
  if (nlevels) *nlevels = (int32_t)c->M.lv.size();
  return LBM_OK;
}

lbm_status lbm_obstacle_links(const lbm_ctx* c, int64_t* elem, int8_t* dir, int64_t cap, int64_t* n) {
  if (!c || !n || cap < 0 || (cap > 0 && (!elem || !dir))) return LBM_ERR_ARG;
  const HostMesh& m = c->M;
  const int64_t cnt = (int64_t)m.obs_elem.size();
  *n = cnt;
  if (cap == 0 || cnt == 0) return LBM_OK;
  // global element slot -> caller index
  std::vector<int64_t> user_of(m.Ntot, -1);
  for (int64_t k = 0; k < m.n_user; ++k) user_of[m.uslot[k]] = k;
  for (int64_t l = 0; l < std::min(cap, cnt); ++l) {
    elem[l] = user_of[m.obs_elem[l]];
    dir[l] = m.obs_dir[l];
  }
  return LBM_OK;
}

lbm_status lbm_set_link_q(lbm_ctx* c, const double* q, int64_t n) {
  if (!c || (n > 0 && !q)) return LBM_ERR_ARG;
  if (!c->p.bouzidi) return c->fail(LBM_ERR_STATE, "params.bouzidi is 0");
  HostMesh& m = c->M;
  if (n != (int64_t)m.obs_elem.size()) return c->fail(LBM_ERR_ARG, "n differs from the obstacle link count");
  for (int64_t l = 0; l < n; ++l)
    if (!(q[l] > 0.0 && q[l] <= 1.0)) return c->fail(LBM_ERR_ARG, "wall distance outside (0, 1]");
  for (int64_t l = 0; l < n; ++l) {
    m.obs_q[l] = q[l];
    if (m.obs_side[l] >= 0) m.out_q[m.obs_side[l]] = q[l];
  }
  if (!c->bound) return LBM_OK;  // uploaded by lbm_bind
  lbm_status s = c->cuda_check(
      cudaMemcpyAsync(c->ws + c->oObsQ, m.obs_q.data(), m.obs_q.size() * 8, cudaMemcpyHostToDevice, c->st), "link q");
  if (s == LBM_OK)
    s = c->cuda_check(
        cudaMemcpyAsync(c->ws + c->oOutQ, m.out_q.data(), m.out_q.size() * 8, cudaMemcpyHostToDevice, c->st), "link q");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "link q");
  return s;
}

lbm_status lbm_device_bytes(const lbm_ctx* c, uint64_t* bytes) {
  if (!c || !bytes || !c->ops || c->M.lv.empty()) return LBM_ERR_ARG;
  *bytes = c->bytes;
  return LBM_OK;
}

lbm_status lbm_bind(lbm_ctx* c, void* ws, uint64_t bytes, void* stream) {
  if (!c || !ws) return LBM_ERR_ARG;
  if (c->M.lv.empty()) return c->fail(LBM_ERR_STATE, "no mesh");
  if (bytes < c->bytes) return c->fail(LBM_ERR_ARG, "device workspace too small");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return c->fail(LBM_ERR_ARG, "device workspace not 256-byte aligned");
  c->drop_graphs();  // captured steps point into the previous workspace
  c->ws = static_cast<char*>(ws);
  c->st = static_cast<cudaStream_t>(stream);
  const HostMesh& m = c->M;
  auto up = [&](size_t off, const void* src, size_t b) -> lbm_status {
    if (b == 0) return LBM_OK;
    return c->cuda_check(cudaMemcpyAsync(c->ws + off, src, b, cudaMemcpyHostToDevice, c->st), "upload");
  };
  lbm_status s = up(c->oNbr, m.nbr.data(), m.nbr.size() * 4);
  if (s == LBM_OK) s = up(c->oBrickNb, m.brick_nb.data(), m.brick_nb.size() * 4);
  if (s == LBM_OK) s = up(c->oBrickTab, m.brick_tab.data(), m.brick_tab.size() * 2);
  if (s == LBM_OK) s = up(c->oInletS, m.inlet_s.data(), m.inlet_s.size() * 8);
  if (s == LBM_OK) s = up(c->oOutQ, m.out_q.data(), m.out_q.size() * 8);
  if (s == LBM_OK) s = up(c->oObsA, m.obs_a.data(), m.obs_a.size() * 4);
  if (s == LBM_OK) s = up(c->oObsQ, m.obs_q.data(), m.obs_q.size() * 8);
  for (int li = 0; li < c->nlev && s == LBM_OK; ++li) {
    const HostLevel& H = m.lv[li];
    s = up(c->ld[li].gff_child0, H.gff_child0.data(), H.gff_child0.size() * 4);
    if (s == LBM_OK) s = up(c->ld[li].gfc_src, H.gfc_src.data(), H.gfc_src.size() * 4);
    if (s == LBM_OK) s = up(c->ld[li].gfc_oct, H.gfc_oct.data(), H.gfc_oct.size());
    if (s == LBM_OK) s = up(c->ld[li].src_elem, H.src_elem.data(), H.src_elem.size() * 4);
    if (s == LBM_OK) s = up(c->ld[li].gsrc_elem, H.gsrc_elem.data(), H.gsrc_elem.size() * 4);
    if (s == LBM_OK) s = up(c->ld[li].gsrc_rec, H.gsrc_rec.data(), H.gsrc_rec.size() * 4);
  }
  if (s == LBM_OK) s = up(c->oSrcMask, m.src_mask.data(), m.src_mask.size() * 4);
  if (s == LBM_OK) s = up(c->oSrcFirst, m.src_first.data(), m.src_first.size() * 4);
  if (s == LBM_OK) s = up(c->oOutElem, m.out_elem.data(), m.out_elem.size() * 4);
  if (s == LBM_OK) s = up(c->oOutA, m.out_a.data(), m.out_a.size() * 4);
  if (s == LBM_OK) s = up(c->oOutB, m.out_b.data(), m.out_b.size() * 4);
  if (s == LBM_OK) s = up(c->oOutDir, m.out_dir.data(), m.out_dir.size());
  if (s == LBM_OK) s = up(c->oOutKind, m.out_kind.data(), m.out_kind.size());
  if (s == LBM_OK) s = up(c->oObsElem, m.obs_elem.data(), m.obs_elem.size() * 4);
  if (s == LBM_OK) s = up(c->oObsDir, m.obs_dir.data(), m.obs_dir.size());
  if (s == LBM_OK) s = up(c->oUslot, m.uslot.data(), m.uslot.size() * 4);
  if (s == LBM_OK) s = up(c->oUlev, m.ulev.data(), m.ulev.size());
  if (s == LBM_OK) s = up(c->oSlotUser, m.slot_user.data(), m.slot_user.size() * 4);
  if (s != LBM_OK) return s;
  if (c->p.use_force) {
    s = c->cuda_check(cudaMemsetAsync(c->ws + c->oF, 0, (size_t)c->d * m.Ntot * c->ops->compute_bytes, c->st),
                      "force clear");
    if (s != LBM_OK) return s;
  }
  for (size_t off : {c->oA, c->oB}) {
    FillArgs f{c->ws + off, m.Ntot, c->p.rho0, c->rho_off};
    c->ops->fill_rest(c->Q, f, c->st);
    ++c->launches;
  }
  s = c->launched("bind");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "bind sync");
  if (s != LBM_OK) return s;
  std::fill(c->parity.begin(), c->parity.end(), 0);
  c->reset_check();
  c->bound = true;
  return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* c, const double* rho, const double* u, const double* S, const double* df) {
  if (!c || !rho || !u) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_init before lbm_bind");
  const int64_t n = c->M.n_user;
  const int d = c->d, nS = c->nS, Q = c->Q;
  // Every level starts in A.  The chunks are computed in caller order into B
  // (coalesced writes, B holds nothing that survives an init), then placed
  // into the element slots of A in slot order, and B is reset to rest.
  // The staging area is used as two halves: the host copies of one half-chunk
  // (on the context's copy stream) overlap the init kernel of the other.
  std::fill(c->parity.begin(), c->parity.end(), 0);
  c->reset_check();
  const bool two = c->copy_stream_ready();
  const int64_t CH = two ? (c->chunk + 1) / 2 : c->chunk;
  const int64_t per = 1 + d + nS + Q;  // staged doubles per element
  cudaStream_t cs = two ? c->copy_st : c->st;
  if (two) {
    // the staging area may still be read by earlier work on the bound stream
    cudaEventRecord(c->copy_ev[2], c->st);
    cudaStreamWaitEvent(cs, c->copy_ev[2], 0);
  }
  int64_t i = 0;
  for (int64_t first = 0; first < n; first += CH, ++i) {
    const int64_t cnt = std::min(CH, n - first);
    const int half = two ? (int)(i & 1) : 0;
    double* sr = c->at<double>(c->oStage) + (size_t)half * CH * per;
    double* su = sr + CH;
    double* sS = su + CH * d;
    double* sdf = sS + CH * nS;
    // this half's previous init kernel has read it
    if (two && i >= 2) cudaStreamWaitEvent(cs, c->copy_ev[half], 0);
    lbm_status s = c->cuda_check(cudaMemcpyAsync(sr, rho + first, cnt * 8, cudaMemcpyHostToDevice, cs), "init copy");
    if (s == LBM_OK)
      s = c->cuda_check(cudaMemcpyAsync(su, u + first * d, cnt * d * 8, cudaMemcpyHostToDevice, cs), "init copy");
    if (s == LBM_OK && S)
      s = c->cuda_check(cudaMemcpyAsync(sS, S + first * nS, cnt * nS * 8, cudaMemcpyHostToDevice, cs), "init copy");
    if (s == LBM_OK && df)
      s = c->cuda_check(cudaMemcpyAsync(sdf, df + first * Q, cnt * Q * 8, cudaMemcpyHostToDevice, cs), "init copy");
    if (s != LBM_OK) return s;
    if (two) {
      cudaEventRecord(c->copy_ev[3], cs);
      cudaStreamWaitEvent(c->st, c->copy_ev[3], 0);
    }
    InitArgs a{};
    a.temp = c->at(c->oB);
    a.ulev = c->at<uint8_t>(c->oUlev);
    a.rho = sr;
    a.u = su;
    a.S = S ? sS : nullptr;
    a.df = df ? sdf : nullptr;
    a.first = first;
    a.cnt = cnt;
    a.n_user = n;
    for (int li = 0; li < c->nlev; ++li) a.omega[li] = c->M.lv[li].omega;
    a.rho_off = c->rho_off;
    c->ops->init(Q, a, c->st);
    ++c->launches;
    if (two) cudaEventRecord(c->copy_ev[half], c->st);
  }
  PlaceArgs pl{c->at(c->oB), c->at(c->oA), c->at<int32_t>(c->oSlotUser), n, c->M.Ntot};
  c->ops->init_place(Q, pl, c->st);
  ++c->launches;
  FillArgs f{c->at(c->oB), c->M.Ntot, c->p.rho0, c->rho_off};
  c->ops->fill_rest(Q, f, c->st);
  ++c->launches;
  lbm_status s = c->launched("init");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "init sync");
  return s;
}

lbm_status lbm_set_force(lbm_ctx* c, const double* F) {
  if (!c || !F) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_set_force before lbm_bind");
  if (!c->p.use_force) return c->fail(LBM_ERR_STATE, "params.use_force is 0");
  const int64_t n = c->M.n_user, CH = c->chunk;
  double* sf = c->at<double>(c->oStage);
  for (int64_t first = 0; first < n; first += CH) {
    const int64_t cnt = std::min(CH, n - first);
    lbm_status s = c->cuda_check(
        cudaMemcpyAsync(sf, F + first * c->d, cnt * c->d * 8, cudaMemcpyHostToDevice, c->st), "force copy");
    if (s != LBM_OK) return s;
    ForceArgs a{c->at(c->oF), c->at<int32_t>(c->oUslot), sf, first, cnt, c->M.Ntot, c->d};
    launch_scatter_force(c->p.precision == LBM_FP64, a, c->st);
    ++c->launches;
  }
  c->recs_valid = false;
  lbm_status s = c->launched("set_force");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "force sync");
  return s;
}

static lbm_status step_run(lbm_ctx* c, int64_t n_coarse);

// the FP64 reductions of the current state into out[8] (host), synchronising
static lbm_status reduce_to_host(lbm_ctx* c, double out[8]) {
  // the per-level arguments come from the one plan builder (also used by
  // lbm_reduce_noalloc); only the partial rows differ
  ReducePlan plan;
  lbm_status ps = reduce_plan(c, &plan);
  if (ps != LBM_OK) return ps;
  for (int li = 0; li < c->nlev; ++li) {
    ReduceArgs a = plan.levels[li];
    a.partial = c->at<double>(c->oPartial) + (size_t)li * kReduceBlocks * 8;
    c->ops->reduce(c->Q, a, c->st);
    ++c->launches;
  }
  FinalArgs fa{c->at<double>(c->oPartial), (int64_t)c->nlev * kReduceBlocks, c->at<double>(c->oRed)};
  launch_final_reduce(fa, c->st);
  ++c->launches;
  lbm_status s = c->launched("reduce");
  if (s == LBM_OK) s = c->cuda_check(cudaMemcpyAsync(out, c->at(c->oRed), 64, cudaMemcpyDeviceToHost, c->st), "reduce copy");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "reduce sync");
  return s;
}

// the mass check of params.check_every: finite, and within mass_band of the
// reference mass when a band is set
static lbm_status check_mass(lbm_ctx* c, bool reference) {
  double r[8];
  lbm_status s = reduce_to_host(c, r);
  if (s != LBM_OK) return s;
  const double m = r[0];
  char buf[160];
  if (!std::isfinite(m)) {
    std::snprintf(buf, sizeof buf, "mass check after %lld coarse steps: mass is not finite (%g)",
                  (long long)c->steps_done, m);
    return c->fail(LBM_ERR_NUMERIC, buf);
  }
  if (reference) {
    c->mass_ref = m;
    c->mass_ref_valid = true;
    return LBM_OK;
  }
  if (c->p.mass_band > 0.0 && std::fabs(m / c->mass_ref - 1.0) > c->p.mass_band) {
    std::snprintf(buf, sizeof buf, "mass check after %lld coarse steps: mass %.17g outside %g of %.17g",
                  (long long)c->steps_done, m, c->p.mass_band, c->mass_ref);
    return c->fail(LBM_ERR_NUMERIC, buf);
  }
  return LBM_OK;
}

// n_coarse coarse steps with no check in between
lbm_status lbm_ctx::run_steps(int64_t n_coarse) { return step_run(this, n_coarse); }

static lbm_status step_run(lbm_ctx* c, int64_t n_coarse) {
  int64_t k = 0;
  if (n_coarse > 0) c->ensure_records();  // outside any capture
  // pairs of coarse steps replay a captured two-step graph and a remaining
  // single step a one-step graph; timed steps (mode 1) and the adjoint's
  // recorded steps are issued one kernel at a time
  if (c->graphs_on && c->timing != 1 && !c->hook && !c->dry) {
    while (k < n_coarse) {
      const lbm_ctx::StepGraph* g = c->step_graph(n_coarse - k >= 2 ? 2 : 1);
      if (!g) break;
      lbm_status s = c->cuda_check(cudaGraphLaunch(g->exec, c->st), "graph launch");
      if (s != LBM_OK) return s;
      c->launches += g->launches;
      c->parity = g->end;
      c->last_graph = (int)(g - c->graphs.data());
      c->graph_unread = true;
      k += g->steps;
    }
  }
  for (; k < n_coarse; ++k) c->coarse_step();
  return c->launched("step");
}

lbm_status lbm_step(lbm_ctx* c, int64_t n_coarse) {
  if (!c || n_coarse < 0) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_step before lbm_bind");
  const int64_t M = c->p.check_every;
  if (M <= 0) {
    c->steps_done += n_coarse;
    return step_run(c, n_coarse);
  }
  // the optional mass check: after every M-th coarse step, counted across calls
  if (!c->mass_ref_valid && n_coarse > 0) {
    lbm_status s = check_mass(c, true);
    if (s != LBM_OK) return s;
  }
  int64_t done = 0;
  while (done < n_coarse) {
    const int64_t chunk = std::min(n_coarse - done, M - c->steps_since_check);
    lbm_status s = step_run(c, chunk);
    if (s != LBM_OK) return s;
    done += chunk;
    c->steps_done += chunk;
    c->steps_since_check += chunk;
    if (c->steps_since_check == M) {
      c->steps_since_check = 0;
      s = check_mass(c, false);
      if (s != LBM_OK) return s;
    }
  }
  return LBM_OK;
}

lbm_status lbm_fill_ghosts(lbm_ctx* c) {
  if (!c) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_fill_ghosts before lbm_bind");
  for (int li = 0; li + 1 < c->nlev; ++li) {
    c->fill_gff(li);
    c->source_moments(li, c->ld[li].momA[c->parity[li]]);
    c->fill_gfc(li + 1, false, true);
  }
  c->recs_valid = true;  // every record now holds the current state's moments
  return c->launched("fill_ghosts");
}

static lbm_status out_chunks(lbm_ctx* c, double* rho, double* u, double* S, double* f) {
  const int64_t n = c->M.n_user, CH = c->chunk;
  const int d = c->d, nS = c->nS, Q = c->Q;
  double* sr = c->at<double>(c->oStage);
  double* su = sr + CH;
  double* sS = su + CH * d;
  double* sf = sS + CH * nS;
  for (int64_t first = 0; first < n; first += CH) {
    const int64_t cnt = std::min(CH, n - first);
    OutArgs a{};
    a.A = c->at(c->oA);
    a.B = c->at(c->oB);
    a.force = c->force_ptr();
    a.uslot = c->at<int32_t>(c->oUslot);
    a.ulev = c->at<uint8_t>(c->oUlev);
    a.parity = c->parity_mask();
    a.rho = rho ? sr : nullptr;
    a.u = u ? su : nullptr;
    a.S = S ? sS : nullptr;
    a.f = f ? sf : nullptr;
    a.first = first;
    a.cnt = cnt;
    a.Ntot = c->M.Ntot;
    for (int li = 0; li < c->nlev; ++li) a.omega[li] = c->M.lv[li].omega;
    a.rho_off = c->rho_off;
    c->ops->out(Q, a, c->st);
    ++c->launches;
    lbm_status s = c->launched("output");
    auto down = [&](double* dst, const double* src, size_t b) {
      if (s == LBM_OK) s = c->cuda_check(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, c->st), "output copy");
    };
    if (rho) down(rho + first, sr, cnt * 8);
    if (u) down(u + first * d, su, cnt * d * 8);
    if (S) down(S + first * nS, sS, cnt * nS * 8);
    if (f) down(f + first * Q, sf, cnt * Q * 8);
    if (s != LBM_OK) return s;
  }
  return c->cuda_check(cudaStreamSynchronize(c->st), "output sync");
}

lbm_status lbm_moments(lbm_ctx* c, double* rho, double* u, double* S) {
  if (!c) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_moments before lbm_bind");
  return out_chunks(c, rho, u, S, nullptr);
}

lbm_status lbm_get_state(lbm_ctx* c, double* f) {
  if (!c || !f) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_get_state before lbm_bind");
  return out_chunks(c, nullptr, nullptr, nullptr, f);
}

lbm_status lbm_set_state(lbm_ctx* c, const double* f) {
  if (!c || !f) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_set_state before lbm_bind");
  const int64_t n = c->M.n_user, CH = c->chunk;
  double* sf = c->at<double>(c->oStage);
  c->reset_check();
  for (int64_t first = 0; first < n; first += CH) {
    const int64_t cnt = std::min(CH, n - first);
    lbm_status s = c->cuda_check(
        cudaMemcpyAsync(sf, f + first * c->Q, cnt * c->Q * 8, cudaMemcpyHostToDevice, c->st), "state copy");
    if (s != LBM_OK) return s;
    SetStateArgs a{c->at(c->oA), c->at(c->oB), c->at<int32_t>(c->oUslot), c->at<uint8_t>(c->oUlev),
                   c->parity_mask(), sf, first, cnt, c->M.Ntot, c->rho_off};
    c->ops->set_state(c->Q, a, c->st);
    ++c->launches;
  }
  lbm_status s = c->launched("set_state");
  if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "state sync");
  return s;
}

lbm_status lbm_reduce(lbm_ctx* c, double out[8]) {
  if (!c || !out) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_reduce before lbm_bind");
  return reduce_to_host(c, out);
}

lbm_status lbm_ghost_count(const lbm_ctx* c, int64_t* n) {
  if (!c || !n) return LBM_ERR_ARG;
  int64_t t = 0;
  for (const HostLevel& H : c->M.lv) t += H.nC + H.nG1 + H.nG2;
  *n = t;
  return LBM_OK;
}

lbm_status lbm_get_ghosts(lbm_ctx* c, int64_t* info, double* f) {
  if (!c || !info || !f) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_get_ghosts before lbm_bind");
  const int Q = c->Q;
  int64_t row = 0;
  double* stage = c->at<double>(c->oStage);
  for (int li = 0; li < c->nlev; ++li) {
    const HostLevel& H = c->M.lv[li];
    const int64_t ng = H.nC + H.nG1 + H.nG2;
    for (int64_t k = 0; k < ng; ++k) {
      int64_t* r = info + 6 * (row + k);
      r[0] = H.L;
      r[1] = k < H.nC ? 1 : 2;
      r[2] = H.ghost_layer[k];
      for (int a = 0; a < 3; ++a) r[3 + a] = H.ghost_xyz[3 * k + a];
    }
    const int64_t seg_first[3] = {H.base + H.oC, H.base + H.oG1, H.base + H.oG2};
    const int64_t seg_cnt[3] = {H.nC, H.nG1, H.nG2};
    for (int sgi = 0; sgi < 3; ++sgi) {
      for (int64_t done = 0; done < seg_cnt[sgi]; done += c->chunk) {
        const int64_t cnt = std::min<int64_t>(c->chunk, seg_cnt[sgi] - done);
        GatherGhostArgs a{c->cur(li), seg_first[sgi] + done, cnt, c->M.Ntot, stage, c->rho_off};
        c->ops->gather_ghosts(Q, a, c->st);
        ++c->launches;
        lbm_status s = c->launched("ghosts");
        if (s == LBM_OK)
          s = c->cuda_check(cudaMemcpyAsync(f + (row + done) * Q, stage, cnt * Q * 8, cudaMemcpyDeviceToHost, c->st),
                            "ghost copy");
        if (s == LBM_OK) s = c->cuda_check(cudaStreamSynchronize(c->st), "ghost sync");
        if (s != LBM_OK) return s;
      }
      row += seg_cnt[sgi];
    }
  }
  return LBM_OK;
}

lbm_status lbm_sfc_partition(const int64_t* tree_ids, int64_t n, int32_t d, int32_t nparts, int64_t* order,
                             int64_t* weights, int64_t* cumulative, int32_t* part) {
  std::string msg;
  return sfc_partition(tree_ids, n, d, nparts, order, weights, cumulative, part, &msg);
}

lbm_status lbm_kernel_launches(const lbm_ctx* c, int64_t* count) {
  if (!c || !count) return LBM_ERR_ARG;
  *count = c->launches;
  return LBM_OK;
}

lbm_status lbm_timing_enable(lbm_ctx* c, int32_t mode) {
  if (!c) return LBM_ERR_ARG;
  if (mode < 0 || mode > 2) return c->fail(LBM_ERR_ARG, "timing mode must be 0, 1 or 2");
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_timing_enable before lbm_bind");
  lbm_status s = c->cuda_check(cudaStreamSynchronize(c->st), "timing sync");
  c->recycle_timed();
  // graphs captured with events (mode 2) and without them are not interchangeable
  if ((mode == 2) != (c->timing == 2)) c->drop_graphs();
  c->graph_unread = false;
  c->timing = mode;
  return s;
}

lbm_status lbm_timing_read(lbm_ctx* c, int64_t* launches, double* ms, int32_t cap) {
  if (!c || !launches || !ms) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_timing_read before lbm_bind");
  lbm_status s = c->cuda_check(cudaStreamSynchronize(c->st), "timing sync");
  if (s != LBM_OK) return s;
  for (int k = 0; k < cap; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
  }
  auto add = [&](const lbm_ctx::Timed& t) {
    float e = 0.f;
    if (s == LBM_OK) s = c->cuda_check(cudaEventElapsedTime(&e, t.a, t.b), "timing read");
    const int row = kTimedKinds * t.li + t.kernel;
    if (s == LBM_OK && row < cap) {
      launches[row] += 1;
      ms[row] += e;
    }
  };
  for (auto& t : c->timed) add(t);
  if (c->graph_unread && c->last_graph >= 0)
    for (auto& t : c->graphs[c->last_graph].timed) add(t);
  c->graph_unread = false;
  c->recycle_timed();
  return s;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

void lbm_destroy(lbm_ctx* c) { delete c; }

}  // extern "C"
