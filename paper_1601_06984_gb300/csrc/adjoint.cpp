// Discrete adjoint driver: checkpointed reverse sweep over the multilevel step.
//
// lbm_adjoint runs the forward steps from the current state, keeping a copy of
// the state every K coarse steps.  Going backwards segment by segment, it
// recomputes the segment once to keep every step's starting state, then for
// each step (last to first) recomputes that step once more while recording its
// op sequence (the "tape") together with copies of every level state an op
// read, and applies the reverse kernels to the tape in reverse order.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "lbm_ctx.h"

// run the brick and neighbour-list reverse stream-collide of a level
// concurrently (disjoint elements and scatter targets, rows of their own)
#ifndef LBM_ADJ_CONCURRENT
#define LBM_ADJ_CONCURRENT 1
#endif
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct TapeOp {
  int op = 0, level = 0;
  int snap = -1;       // snapshot of the state the op reads (level, or level+1 for GFF)
  int snap_a = -1;     // GFC: snapshot for the records at t (momA)
  int snap_b = -1;     // GFC B: snapshot for the records at t+1
  std::vector<int> parity;  // parities of all levels before the op
};

struct AdjLayout {
  size_t lamA = 0, lamB = 0, lamF = 0, side_fwd = 0, lam_side = 0, partial = 0, acc = 0, contrib = 0;
  std::vector<size_t> lam_recA, lam_recB, recA, recB, csr_off, csr_item;
  size_t ck = 0, steps = 0, snaps = 0, ends = 0, fin = 0;
  int n_ck = 0, n_steps = 0, n_snaps = 0;
  // tape_all: a segment's recompute records every step's tape (two forward
  // passes per step instead of three); needs K tapes' copies plus, per step but
  // the last, copies of the states the reverse reads in place (both buffers)
  bool tape_all = false;
  size_t state_bytes = 0, total = 0;
  int partial_rows = 0;  // running rows of the parameter sums: the largest grid of a reverse launch
  int side_row0 = 0;     // first row of the neighbour-list reverse, which runs beside the brick reverse
};

// Copies the rows of level li's segment of a [Q][Ntot] state.
void copy_level(lbm_ctx* c, const void* from, void* to, int li) {
  const HostLevel& H = c->M.lv[li];
  const size_t s = c->ops->storage_bytes;
  launch_copy_rows(from, to, (size_t)c->M.Ntot * s, (size_t)H.base * s, (size_t)H.N * s, c->Q, s, c->st);
}

// Walks (dry) or follows (recording) one coarse step and decides, per level
// state an op reads, where the reverse sweep finds it.  A state is identified
// by (level, version); the version of a level is bumped by every op that
// writes it.  A state that no later op of the step overwrites (its buffer
// keeps it until the next restore) is read in place; the others are copied to
// the snapshot store when they are first read.  A copy fills only its level's
// segment of a full-size slot, so copies of different levels share slots: the
// k-th copy of every level goes to slot k.
struct Recorder {
  lbm_ctx* c;
  bool counting = true;
  std::vector<int> version;                    // per level, bumped by every write
  std::map<std::pair<int, int>, int> snap_of;  // (level, version) -> snapshot index
  std::vector<std::pair<int, int>> snap_key;
  std::vector<int> snap_buf;                   // buffer (parity) the state lives in
  std::vector<char> clobbered;                 // a later op of the step wrote that buffer
  std::vector<char> need_copy;                 // from the dry walk: copy instead of reading in place
  std::vector<const void*> where;              // recording: where the reverse reads each state
  std::vector<TapeOp> tape;
  int last_mom_a_snap[16], last_mom_b_snap[16];
  char* snap_base = nullptr;
  size_t state_bytes = 0;
  int max_snaps = 0;
  int n_copies[16] = {};                       // copies taken so far, per level
  bool overflow = false;

  explicit Recorder(lbm_ctx* ctx) : c(ctx), version(ctx->nlev, 0) {
    std::fill(last_mom_a_snap, last_mom_a_snap + 16, -1);
    std::fill(last_mom_b_snap, last_mom_b_snap + 16, -1);
  }


  void wrote(int li, int buf) {
    for (size_t id = 0; id < snap_key.size(); ++id)
      if (snap_key[id].first == li && snap_buf[id] == buf) clobbered[id] = 1;
    version[li]++;
  }

  int snapshot(int li) {
    auto key = std::make_pair(li, version[li]);
    auto it = snap_of.find(key);
    if (it != snap_of.end()) return it->second;
    const int id = (int)snap_key.size();
    snap_of[key] = id;
    snap_key.push_back(key);
    snap_buf.push_back(c->parity[li]);
    clobbered.push_back(0);
    if (!counting) {
      const bool copy = id < (int)need_copy.size() ? need_copy[id] != 0 : true;
      if (!copy) {
        where.push_back(c->cur(li));
      } else if (n_copies[li] >= max_snaps) {
        overflow = true;
        where.push_back(nullptr);
        return id;
      } else {
        char* dst = snap_base + (size_t)n_copies[li]++ * state_bytes;
        copy_level(c, c->cur(li), dst, li);
        where.push_back(dst);
      }
    }
    return id;
  }

  void on(int op, int li) {
    TapeOp t;
    t.op = op;
    t.level = li;
    t.parity = c->parity;
    switch (op) {
      case OP_GFF:
        t.snap = snapshot(li + 1);
        tape.push_back(t);
        wrote(li, c->parity[li]);
        break;
      case OP_MOM_A:
        t.snap = snapshot(li);
        last_mom_a_snap[li] = t.snap;
        tape.push_back(t);
        break;
      case OP_GFC_A:
        t.snap_a = last_mom_a_snap[li - 1];
        tape.push_back(t);
        wrote(li, c->parity[li]);
        break;
      case OP_SC:
        t.snap = snapshot(li);
        tape.push_back(t);
        wrote(li, c->parity[li] ^ 1);
        break;
      case OP_MOM_B:
        t.snap = snapshot(li);
        t.snap_a = last_mom_a_snap[li];
        last_mom_b_snap[li] = t.snap;
        tape.push_back(t);
        break;
      case OP_GFC_B:
        t.snap_a = last_mom_a_snap[li - 1];
        t.snap_b = last_mom_b_snap[li - 1];
        tape.push_back(t);
        wrote(li, c->parity[li]);
        break;
    }
  }
};

// Dry walk of one coarse step from the current parities (launches nothing):
// the states its ops read and which of them a later op overwrites.
void dry_walk(lbm_ctx* c, Recorder& r) {
  r.counting = true;
  std::vector<int> saved = c->parity;
  c->hook = [&](int op, int li) { r.on(op, li); };
  c->dry = true;
  c->advance(0);
  c->dry = false;
  c->hook = nullptr;
  c->parity = saved;
}

// Which of the states the next coarse step's ops read must be copied.
std::vector<char> plan_snapshots(lbm_ctx* c) {
  Recorder r(c);
  dry_walk(c, r);
  return r.clobbered;
}

// Snapshot slots one coarse step's tape needs: the largest number of copies of
// one level (the same for every step: the pattern depends only on which of a
// level's two buffers an op touches).
int count_snapshots(lbm_ctx* c) {
  Recorder r(c);
  dry_walk(c, r);
  std::vector<int> per_level(c->nlev, 0);
  for (size_t id = 0; id < r.snap_key.size(); ++id)
    if (r.clobbered[id]) per_level[r.snap_key[id].first]++;
  return per_level.empty() ? 0 : *std::max_element(per_level.begin(), per_level.end());
}

AdjLayout adj_layout(lbm_ctx* c, int64_t n, int K) {
  AdjLayout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    size_t r = o;
    o += align_up(std::max<size_t>(b, 1));
    return r;
  };
  const size_t N = (size_t)c->M.Ntot;
  const size_t lb = c->p.precision == LBM_FP64 ? 8 : 4;
  L.lamA = take(c->Q * N * lb);
  L.lamB = take(c->Q * N * lb);
  L.lamF = take((size_t)c->d * N * 8);
  L.side_fwd = take(c->M.out_elem.size() * lb);
  L.lam_side = take(c->M.out_elem.size() * lb);
  L.partial_rows = kAdjBlocks;
  for (int li = 0; li < c->nlev; ++li)
    L.partial_rows = std::max<int>(L.partial_rows, (int)((c->M.lv[li].nB + LBM_BRICKS_PER_BLOCK - 1) / LBM_BRICKS_PER_BLOCK));
  // the neighbour-list reverse runs concurrently with the brick reverse, so
  // its blocks add to rows of their own
  L.side_row0 = LBM_ADJ_CONCURRENT ? L.partial_rows : 0;
  if (LBM_ADJ_CONCURRENT) L.partial_rows += kAdjBlocks;
  L.partial = take((size_t)L.partial_rows * kAccCols * 8);
  L.acc = take(32 * 8);
  int64_t max_contrib = 0;
  for (int li = 0; li < c->nlev; ++li) {
    const HostLevel& H = c->M.lv[li];
    const int64_t nsrc = (int64_t)H.src_elem.size();
    L.lam_recA.push_back(take((size_t)nsrc * mom_stride(c->Q) * lb));
    L.lam_recB.push_back(take((size_t)nsrc * mom_stride(c->Q) * lb));
    L.recA.push_back(take((size_t)nsrc * mom_stride(c->Q) * lb));
    L.recB.push_back(take((size_t)nsrc * mom_stride(c->Q) * lb));
    L.csr_off.push_back(take((size_t)(nsrc + 1) * 4));
    const int64_t nfine = li + 1 < c->nlev ? c->M.lv[li + 1].nC : 0;
    L.csr_item.push_back(take((size_t)4 * nfine * 4));
    max_contrib = std::max(max_contrib, nfine);
  }
  L.contrib = take((size_t)max_contrib * 4 * mom_stride(c->Q) * lb);
  L.state_bytes = align_up((size_t)c->Q * N * c->ops->storage_bytes);
  L.n_ck = (int)((n + K - 1) / K);
  L.n_steps = K;
  L.n_snaps = count_snapshots(c);
  // workspace rule: record the whole segment when that needs at most twice the
  // states of the step-by-step scheme, or at most 8 GiB of states
  const size_t per_step_old = (size_t)K + (size_t)L.n_snaps;
  const size_t per_step_new = (size_t)K * (size_t)(L.n_snaps + 2);
  if (c->p.adjoint_tape == 1) L.tape_all = true;
  else if (c->p.adjoint_tape == 2) L.tape_all = false;
  else L.tape_all = per_step_new <= 2 * per_step_old || per_step_new * L.state_bytes <= ((size_t)8 << 30);
  L.ck = o;
  o += (size_t)L.n_ck * L.state_bytes;
  L.steps = o;
  if (!L.tape_all) o += (size_t)L.n_steps * L.state_bytes;
  L.snaps = o;
  o += (size_t)L.n_snaps * L.state_bytes * (L.tape_all ? (size_t)K : 1);
  L.ends = o;
  if (L.tape_all) o += (size_t)2 * (size_t)(K - 1) * L.state_bytes;
  L.fin = o;
  o += L.state_bytes;
  L.total = o;
  return L;
}

const AdjOps* adj_ops_for(int precision) {
  if (precision == LBM_FP64) return adj_ops_fp64();
  if (precision == LBM_FP32DEV) return adj_ops_fp32dev();
  return adj_ops_bf16dev();
}

// side stream and fork/join events of the concurrent reverse kernels (ok
// false: not available, everything runs on the bound stream); released when
// the adjoint returns (the driver releases pending resources when done)
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ok = false;
  SideStream() {
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  ~SideStream() {
    if (s) cudaStreamDestroy(s);
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
};

}  // namespace

extern "C" {

lbm_status lbm_set_params(lbm_ctx* c, double omega_coarse, const double* u_in) {
  if (!c || !(omega_coarse > 0.0 && omega_coarse < 2.0)) return LBM_ERR_ARG;
  std::vector<double> om(c->nlev);
  om[0] = omega_coarse;
  for (int li = 1; li < c->nlev; ++li) om[li] = finer_omega(om[li - 1], c->p.time_mode);
  for (int li = 0; li < c->nlev; ++li)
    if (std::fabs(1.0 - om[li]) < 1e-3) return c->fail(LBM_ERR_ARG, "omega too close to 1 on some level");
  c->drop_graphs();  // captured steps carry the old omega and inlet values
  c->recs_valid = false;  // the source records depend on omega
  for (int li = 0; li < c->nlev; ++li) c->M.lv[li].omega = om[li];
  c->p.omega_coarse = omega_coarse;
  if (u_in) {
    for (int a = 0; a < 3; ++a) c->p.u_in[a] = u_in[a];
    int cc[kQmax][3];
    double w[kQmax];
    host_lattice(c->Q, cc, w);
    for (int i = 0; i < c->Q; ++i) {
      double cu = 0;
      for (int a = 0; a < c->d; ++a) cu += cc[i][a] * u_in[a];
      c->inlet[i] = 6.0 * w[i] * c->p.rho0 * cu;
    }
  }
  return LBM_OK;
}

lbm_status lbm_adjoint_bytes(lbm_ctx* c, int64_t n_coarse, int32_t K, uint64_t* bytes) {
  if (!c || !bytes || n_coarse < 1 || K < 1) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_adjoint_bytes before lbm_bind");
  if (c->p.time_mode == LBM_TIME_DIFFUSIVE) return c->fail(LBM_ERR_STATE, "no adjoint in LBM_TIME_DIFFUSIVE");
  *bytes = adj_layout(c, n_coarse, K).total;
  return LBM_OK;
}

lbm_status lbm_adjoint(lbm_ctx* c, int64_t n, int32_t K, int32_t objective, void* adj_ws, uint64_t bytes,
                       double* J, double* dJ_dF, double* dJ_domega, double* dJ_duin, double* dJ_df0) {
  if (!c || !adj_ws || n < 1 || K < 1 || objective < 0 || objective > 3) return LBM_ERR_ARG;
  if (!c->bound) return c->fail(LBM_ERR_STATE, "lbm_adjoint before lbm_bind");
  if (c->p.time_mode == LBM_TIME_DIFFUSIVE) return c->fail(LBM_ERR_STATE, "no adjoint in LBM_TIME_DIFFUSIVE");
  if (objective > c->d) return c->fail(LBM_ERR_ARG, "force component beyond the dimension");
  const AdjLayout L = adj_layout(c, n, K);
  if (bytes < L.total) return c->fail(LBM_ERR_ARG, "adjoint workspace too small");
  if (reinterpret_cast<uintptr_t>(adj_ws) % kAlign) return c->fail(LBM_ERR_ARG, "adjoint workspace not aligned");
  char* W = static_cast<char*>(adj_ws);
  cudaStream_t st = c->st;
  SideStream side;
  const AdjOps* aops = adj_ops_for(c->p.precision);
  const bool fp64 = c->p.precision == LBM_FP64;
  const size_t N = (size_t)c->M.Ntot;
  auto chk = [&](cudaError_t e, const char* w) { return c->cuda_check(e, w); };
  // ---- clear adjoint state, build the transposed GFC source lists
  lbm_status s = chk(cudaMemsetAsync(W, 0, L.ck, st), "adjoint clear");
  if (s != LBM_OK) return s;
  for (int li = 0; li + 1 < c->nlev; ++li) {
    const HostLevel& Hc = c->M.lv[li];
    const HostLevel& Hf = c->M.lv[li + 1];
    const int64_t nsrc = (int64_t)Hc.src_elem.size();
    std::vector<int32_t> off(nsrc + 1, 0), item(4 * Hf.nC);
    for (int64_t k = 0; k < Hf.nC; ++k)
      for (int q = 0; q < 4; ++q) off[Hf.gfc_src[(size_t)q * Hf.nC + k] + 1]++;
    for (int64_t k = 0; k < nsrc; ++k) off[k + 1] += off[k];
    std::vector<int32_t> fill(off.begin(), off.end() - 1);
    for (int64_t k = 0; k < Hf.nC; ++k)  // ghost order, then source slot: fixed summation order
      for (int q = 0; q < 4; ++q) item[fill[Hf.gfc_src[(size_t)q * Hf.nC + k]]++] = (int32_t)(4 * k + q);
    s = chk(cudaMemcpyAsync(W + L.csr_off[li], off.data(), off.size() * 4, cudaMemcpyHostToDevice, st), "csr");
    if (s == LBM_OK && !item.empty())
      s = chk(cudaMemcpyAsync(W + L.csr_item[li], item.data(), item.size() * 4, cudaMemcpyHostToDevice, st), "csr");
    if (s == LBM_OK) s = chk(cudaStreamSynchronize(st), "csr sync");
    if (s != LBM_OK) return s;
  }
  auto save_state = [&](char* dst) {
    for (int li = 0; li < c->nlev; ++li) copy_level(c, c->cur(li), dst, li);
  };
  auto restore_state = [&](const char* src, const std::vector<int>& par) {
    for (int li = 0; li < c->nlev; ++li) {
      c->parity[li] = par[li];
      copy_level(c, src, c->cur(li), li);
    }
    c->recs_valid = false;
  };
  // ---- forward with checkpoints: the parities of every step from a dry walk,
  // then each segment through lbm_step's path (graph replay of step pairs)
  std::vector<std::vector<int>> parity_at(n + 1);
  {
    const std::vector<int> p0 = c->parity;
    c->dry = true;
    for (int64_t t = 0; t < n; ++t) {
      parity_at[t] = c->parity;
      c->advance(0);
    }
    c->dry = false;
    parity_at[n] = c->parity;
    c->parity = p0;
  }
  for (int64_t t = 0; t < n && s == LBM_OK; t += K) {
    save_state(W + L.ck + (size_t)(t / K) * L.state_bytes);
    s = c->run_steps(std::min<int64_t>(K, n - t));
  }
  if (s == LBM_OK && c->parity != parity_at[n]) s = c->fail(LBM_ERR_INTERNAL, "adjoint forward parities differ");
  if (s != LBM_OK) return s;
  save_state(W + L.fin);
  s = c->launched("adjoint forward");
  if (s != LBM_OK) return s;
  // ---- objective and seed
  double red[8];
  s = lbm_reduce(c, red);
  if (s != LBM_OK) return s;
  if (J) *J = objective == 0 ? red[7] : red[3 + objective];
  char* lamA = W + L.lamA;
  char* lamB = W + L.lamB;
  auto lam_for = [&](int par) { return par ? lamB : lamA; };
  // the body-force adjoint is accumulated only when it is asked for
  double* lamF = dJ_dF ? reinterpret_cast<double*>(W + L.lamF) : nullptr;
  double* partial = reinterpret_cast<double*>(W + L.partial);
  double* acc = reinterpret_cast<double*>(W + L.acc);
  const void* force = c->force_ptr();
  auto common = [&](const void* fsrc, void* la, void* lbuf, int acc_la = 0, int acc_lb = -1) {
    AdjCommon cm{};
    cm.la = acc_la;
    cm.lb = acc_lb;
    cm.fsrc = fsrc;
    cm.force = force;
    cm.lam_a = la;
    cm.lam_b = lbuf;
    cm.lam_force = lamF;
    cm.partial = partial;
    cm.Ntot = (int64_t)N;
    cm.rho_off = c->rho_off;
    cm.rho0 = c->p.rho0;
    return cm;
  };
  for (int li = 0; li < c->nlev; ++li) {
    const HostLevel& H = c->M.lv[li];
    AdjSeedArgs a{};
    a.c = common(c->cur(li), nullptr, lam_for(c->parity[li]));
    a.objective = objective;
    a.begin = H.base + H.oF;
    a.end = H.base + H.oF + H.nF;
    a.vol = std::ldexp(1.0, -c->d * li);
    a.obs_elem = c->at<int32_t>(c->oObsElem) + H.obs_begin;
    a.obs_dir = c->at<int8_t>(c->oObsDir) + H.obs_begin;
    a.obs_a = c->at<int32_t>(c->oObsA) + H.obs_begin;
    a.obs_q = c->at<double>(c->oObsQ) + H.obs_begin;
    a.obs_n = H.obs_end - H.obs_begin;
    a.fscale = std::ldexp(1.0, (c->d - 1) * (c->nlev - 1 - li));
    if (objective == 0) {
      if (a.end > a.begin) aops->seed(c->Q, a, st);
    } else if (a.obs_n > 0) {
      // the own slot, then (interpolated bounce-back only) the second node and
      // the opposite slot, one pass each so that no two links share a slot
      for (int which = 0; which < (c->p.bouzidi ? 3 : 1); ++which) {
        a.which = which;
        aops->seed(c->Q, a, st);
      }
    }
  }
  // ---- reverse sweep
  const int nseg = L.n_ck;
  // records one coarse step's tape while running it (copies into snap_base)
  auto record_step = [&](Recorder& r, char* snap_base) -> lbm_status {
    r.counting = false;
    r.need_copy = plan_snapshots(c);
    r.snap_base = snap_base;
    r.state_bytes = L.state_bytes;
    r.max_snaps = L.n_snaps;
    c->ensure_records();  // before the hook: the tape holds the step's own ops only
    c->hook = [&](int op, int li) { r.on(op, li); };
    c->advance(0);
    c->hook = nullptr;
    if (r.overflow) return c->fail(LBM_ERR_INTERNAL, "adjoint tape needs more snapshots than counted");
    if (r.clobbered != r.need_copy) return c->fail(LBM_ERR_INTERNAL, "adjoint tape differs from its plan");
    return LBM_OK;
  };
  // runs one recorded step backwards
  auto reverse_step = [&](Recorder& r) {
    auto snap = [&](int id) { return r.where[id]; };
    // forward records of an interface, recomputed from the snapshots
    auto records = [&](int lc, int sa, int sb) {
      const HostLevel& Hc = c->M.lv[lc];
      MomentsArgs m{};
      m.force = force;
      m.elem = c->at<int32_t>(c->ld[lc].src_elem);
      m.Ntot = (int64_t)N;
      m.nsrc = c->ld[lc].nsrc;
      m.omega = Hc.omega;
      m.rho_off = c->rho_off;
      m.src = snap(sa);
      m.mom = W + L.recA[lc];
      m.prev = nullptr;
      c->ops->source_moments(c->Q, m, st);
      if (sb < 0) return static_cast<const void*>(W + L.recA[lc]);
      m.src = snap(sb);
      m.mom = W + L.recB[lc];
      m.prev = W + L.recA[lc];
      c->ops->source_moments(c->Q, m, st);
      return static_cast<const void*>(W + L.recB[lc]);
    };
    for (int k = (int)r.tape.size() - 1; k >= 0; --k) {
      const TapeOp& t = r.tape[k];
      const int li = t.level;
      const HostLevel& H = c->M.lv[li];
      if (t.op == OP_SC) {
        const int p = t.parity[li];
        const bool outlet = H.out_end > H.out_begin;
        if (outlet) {
          OutletArgs o{};
          o.src = snap(t.snap);
          o.side = W + L.side_fwd;
          o.elem = c->at<int32_t>(c->oOutElem);
          o.a = c->at<int32_t>(c->oOutA);
          o.b = c->at<int32_t>(c->oOutB);
          o.dir = c->at<int8_t>(c->oOutDir);
          o.kind = c->at<int8_t>(c->oOutKind);
          o.force = force;
          o.Ntot = (int64_t)N;
          o.begin = H.out_begin;
          o.end = H.out_end;
          o.omega = H.omega;
          o.rho_off = c->rho_off;
          o.rho0 = c->p.rho0;
          o.zero_gradient = c->p.outlet == LBM_OUTLET_ZERO_GRADIENT;
          o.q = c->at<double>(c->oOutQ);
          c->ops->outlet(c->Q, o, st);
        }
        AdjSCArgs a{};
        a.c = common(snap(t.snap), lam_for(!p), lam_for(p), li);
        a.nbr = c->at<uint32_t>(c->oNbr);
        a.side_fwd = W + L.side_fwd;
        a.lam_side = W + L.lam_side;
        a.omega = H.omega;
        std::memcpy(a.inlet, c->inlet, sizeof(a.inlet));
        a.inlet_s = c->at<double>(c->oInletS);
        // interior bricks (the first 64 nB fluid elements) through the brick
        // tables, everything else through the neighbour list
        const int64_t nbrick = 64 * H.nB;
        AdjSCArgs ab = a;
        ab.begin = H.base + H.oF;
        ab.nB = H.nB;
        ab.brick_nb = c->at<int32_t>(c->oBrickNb) + (size_t)H.brick_first * 27;
        ab.brick_tab = c->at<uint16_t>(c->oBrickTab);
        // the neighbour-list reverse on the side stream, beside the brick reverse
        const bool fork = LBM_ADJ_CONCURRENT && side.ok;
        if (fork) {
          cudaEventRecord(side.fork, st);
          cudaStreamWaitEvent(side.s, side.fork, 0);
        }
        aops->sc_brick(c->Q, ab, st);
        if (c->p.time_mode == LBM_TIME_TWO_LAYER) {
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
        a.c.partial = partial + (size_t)L.side_row0 * kAccCols;
        aops->sc(c->Q, a, fork ? side.s : st);
        if (fork) {
          cudaEventRecord(side.join, side.s);
          cudaStreamWaitEvent(st, side.join, 0);
        }
        if (outlet) {
          for (int which = 0; which < (c->p.bouzidi ? 6 : 3); ++which) {
            AdjOutletArgs o{};
            o.c = common(snap(t.snap), nullptr, lam_for(p), li);
            o.elem = c->at<int32_t>(c->oOutElem);
            o.a = c->at<int32_t>(c->oOutA);
            o.b = c->at<int32_t>(c->oOutB);
            o.dir = c->at<int8_t>(c->oOutDir);
            o.kind = c->at<int8_t>(c->oOutKind);
            o.lam_side = W + L.lam_side;
            o.begin = H.out_begin;
            o.end = H.out_end;
            o.which = which;
            o.omega = H.omega;
            o.zero_gradient = c->p.outlet == LBM_OUTLET_ZERO_GRADIENT;
            o.q = c->at<double>(c->oOutQ);
            aops->outlet(c->Q, o, st);  // pass 0 also adds d/d omega through the normal links' f^neq
          }
        }
      } else if (t.op == OP_MOM_A || t.op == OP_MOM_B) {
        if (c->ld[li].nsrc == 0) continue;
        AdjMomArgs a{};
        a.c = common(snap(t.snap), nullptr, lam_for(t.parity[li]), li);
        a.elem = c->at<int32_t>(c->ld[li].src_elem);
        a.lam_rec = W + (t.op == OP_MOM_A ? L.lam_recA[li] : L.lam_recB[li]);
        a.lam_rec_prev = t.op == OP_MOM_B ? W + L.lam_recA[li] : nullptr;
        a.nsrc = c->ld[li].nsrc;
        a.omega = H.omega;
        aops->moments(c->Q, a, st);
      } else if (t.op == OP_GFC_A || t.op == OP_GFC_B) {
        if (H.nC == 0) continue;
        const int lc = li - 1;
        const void* rec = records(lc, t.snap_a, t.op == OP_GFC_B ? t.snap_b : -1);
        AdjGfcArgs a{};
        a.c = common(nullptr, lam_for(t.parity[li]), nullptr, lc, li);
        a.rec = rec;
        a.gsrc = c->at<int32_t>(c->ld[li].gfc_src);
        a.oct = c->at<uint8_t>(c->ld[li].gfc_oct);
        a.contrib = W + L.contrib;
        a.ng = H.nC;
        a.dest0 = H.base + H.oC;
        a.omega_c = c->M.lv[lc].omega;
        a.omega_f = H.omega;
        aops->gfc(c->Q, a, st);
        AdjGatherArgs g{W + L.contrib, reinterpret_cast<const int32_t*>(W + L.csr_off[lc]),
                        reinterpret_cast<const int32_t*>(W + L.csr_item[lc]),
                        W + (t.op == OP_GFC_A ? L.lam_recA[lc] : L.lam_recB[lc]), c->ld[lc].nsrc,
                        mom_stride(c->Q)};
        launch_adj_gather(fp64, g, st);
      } else if (t.op == OP_GFF) {
        if (H.nG1 + H.nG2 == 0) continue;
        AdjGffArgs a{};
        a.c = common(snap(t.snap), lam_for(t.parity[li]), lam_for(t.parity[li + 1]), li, li + 1);
        a.child0 = c->at<int32_t>(c->ld[li].gff_child0);
        a.ng = H.nG1 + H.nG2;
        a.n_inner = H.nG1;
        a.dest0 = H.base + H.oG1;
        a.dest_outer = H.base + H.oG2;
        a.omega_c = H.omega;
        a.omega_f = c->M.lv[li + 1].omega;
        aops->gff(c->Q, a, st);
      }
    }
    return c->launched("adjoint sweep");
  };
  for (int seg = nseg - 1; seg >= 0 && s == LBM_OK; --seg) {
    const int64_t s0 = (int64_t)seg * K, s1 = std::min<int64_t>(s0 + K, n);
    restore_state(W + L.ck + (size_t)seg * L.state_bytes, parity_at[s0]);
    if (L.tape_all) {
      // record every step of the segment in one recompute; what a step's
      // reverse would read in place is copied before the next step overwrites
      // it (both buffers of a level can hold such a state)
      std::vector<Recorder> recs;
      recs.reserve((size_t)(s1 - s0));
      for (int64_t t = s0; t < s1 && s == LBM_OK; ++t) {
        recs.emplace_back(c);
        Recorder& r = recs.back();
        s = record_step(r, W + L.snaps + (size_t)(t - s0) * L.n_snaps * L.state_bytes);
        if (s != LBM_OK || t + 1 == s1) continue;
        char* ends = W + L.ends + (size_t)(t - s0) * 2 * L.state_bytes;
        for (size_t id = 0; id < r.snap_key.size(); ++id) {
          if (r.need_copy[id]) continue;
          const int li = r.snap_key[id].first;
          const int buf = r.snap_buf[id];
          char* dst = ends + (size_t)buf * L.state_bytes;
          copy_level(c, buf ? c->at(c->oB) : c->at(c->oA), dst, li);
          r.where[id] = dst;
        }
      }
      for (int64_t t = s1 - 1; t >= s0 && s == LBM_OK; --t) s = reverse_step(recs[t - s0]);
    } else {
      // recompute the segment keeping each step's start state; the last step's
      // is the live state, which its tape pass starts from directly
      for (int64_t t = s0; t + 1 < s1; ++t) {
        save_state(W + L.steps + (size_t)(t - s0) * L.state_bytes);
        c->coarse_step();
      }
      for (int64_t t = s1 - 1; t >= s0 && s == LBM_OK; --t) {
        if (t + 1 < s1) restore_state(W + L.steps + (size_t)(t - s0) * L.state_bytes, parity_at[t]);
        Recorder r(c);
        s = record_step(r, W + L.snaps);
        if (s == LBM_OK) s = reverse_step(r);
      }
    }
  }
  if (s != LBM_OK) return s;
  // ---- parameter gradients
  launch_accum(AccumArgs{partial, L.partial_rows, acc}, st);
  double hacc[kAccCols];
  s = chk(cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st), "adjoint acc");
  if (s == LBM_OK) s = chk(cudaStreamSynchronize(st), "adjoint sync");
  if (s != LBM_OK) return s;
  if (dJ_domega) {
    // omega_L = 1 / (1/2 + 2^L (1/omega_c - 1/2)): d omega_L / d omega_c = 2^L omega_L^2 / omega_c^2
    const double wc = c->M.lv[0].omega;
    double g = 0.0;
    for (int li = 0; li < c->nlev; ++li) {
      const double wl = c->M.lv[li].omega;
      g += hacc[li] * std::ldexp(1.0, li) * wl * wl / (wc * wc);
    }
    *dJ_domega = g;
  }
  if (dJ_duin)
    for (int a = 0; a < 3; ++a) dJ_duin[a] = a < c->d ? hacc[16 + a] : 0.0;
  if (dJ_dF) {
    double* stage = c->at<double>(c->oStage);
    for (int64_t first = 0; first < c->M.n_user; first += c->chunk) {
      const int64_t cnt = std::min<int64_t>(c->chunk, c->M.n_user - first);
      launch_gather_force_user(lamF, c->at<int32_t>(c->oUslot), stage, first, cnt, (int64_t)N, c->d, st);
      s = chk(cudaMemcpyAsync(dJ_dF + first * c->d, stage, cnt * c->d * 8, cudaMemcpyDeviceToHost, st), "dJdF");
      if (s == LBM_OK) s = chk(cudaStreamSynchronize(st), "dJdF sync");
      if (s != LBM_OK) return s;
    }
  }
  if (dJ_df0) {
    // the adjoint now holds dJ / d(initial pdfs), in the buffers of the parities at t0
    uint32_t pm = 0;
    for (int li = 0; li < c->nlev; ++li) pm |= (uint32_t)(parity_at[0][li] & 1) << li;
    double* stage = c->at<double>(c->oStage);
    for (int64_t first = 0; first < c->M.n_user; first += c->chunk) {
      const int64_t cnt = std::min<int64_t>(c->chunk, c->M.n_user - first);
      launch_gather_lam_user(fp64, lamA, lamB, pm, c->at<int32_t>(c->oUslot), c->at<uint8_t>(c->oUlev), stage,
                             first, cnt, (int64_t)N, c->Q, st);
      s = chk(cudaMemcpyAsync(dJ_df0 + first * c->Q, stage, cnt * c->Q * 8, cudaMemcpyDeviceToHost, st), "dJdf0");
      if (s == LBM_OK) s = chk(cudaStreamSynchronize(st), "dJdf0 sync");
      if (s != LBM_OK) return s;
    }
  }
  // ---- leave the simulation at the final state
  restore_state(W + L.fin, parity_at[n]);
  s = c->launched("adjoint restore");
  if (s == LBM_OK) s = chk(cudaStreamSynchronize(st), "adjoint end");
  return s;
}

}  // extern "C"
