// The library context (opaque at the ABI): host mesh, workspace layout, bound
// device state and the driver.  Shared by api.cpp and adjoint.cpp.
#pragma once

#include <cuda_runtime_api.h>

#include <functional>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
// Ops of the recursive level step, in the order lbm_ctx::advance issues them.
enum StepOp { OP_GFF = 0, OP_MOM_A = 1, OP_GFC_A = 2, OP_SC = 3, OP_MOM_B = 4, OP_GFC_B = 5 };
// Kernel kinds of the per-launch timing (lbm_timing_read row kTimedKinds * L + kind)
enum TimedKind { TK_INTERIOR = 0, TK_LIST = 1, TK_BOUNDARY = 2, TK_GFF = 3, TK_MOM = 4, TK_GFC = 5, TK_OUTLET = 6,
                 TK_SC_SPAN = 7 };
constexpr int kTimedKinds = 8;

struct LevelDev {
  size_t gff_child0 = 0, gfc_src = 0, gfc_oct = 0, src_elem = 0, gsrc_elem = 0, gsrc_rec = 0;
  // source records of the two pdf buffers: momA[parity] those of the current
  // state (a stream-collide writes those of its new state into the other one
  // while the GhostFromCoarser fill may still read these)
  size_t momA[2] = {0, 0};
  int64_t nsrc = 0, n_gsrc = 0, n_gsrc_inner = 0;
};

}  // namespace lbm

struct lbm_ctx {
  lbm_params p{};
  lbm::HostMesh M;
  const lbm::Ops* ops = nullptr;
  std::string err;
  int d = 2, Q = 9, nS = 3, nlev = 1;
  double rho_off = 0.0;
  double inlet[lbm::kQmax] = {};
  // layout (byte offsets into the workspace)
  size_t oA = 0, oB = 0, oNbr = 0, oBrickNb = 0, oBrickTab = 0, oInletS = 0, oOutQ = 0, oObsA = 0, oObsQ = 0, oF = 0, oOutElem = 0, oOutA = 0, oOutB = 0, oOutDir = 0, oOutKind = 0,
         oSide = 0, oObsElem = 0, oObsDir = 0, oUslot = 0, oUlev = 0, oSlotUser = 0, oStage = 0, oPartial = 0, oRed = 0,
         oSrcMask = 0, oSrcFirst = 0;
  std::vector<lbm::LevelDev> ld;
  size_t bytes = 0;
  int64_t chunk = 0;
  // bound state
  bool bound = false;
  char* ws = nullptr;
  cudaStream_t st = nullptr;
  std::vector<int> parity;
  int64_t launches = 0;
  // optional mass check (params.check_every): coarse steps since the last
  // check, and the reference mass (taken at the first lbm_step after bind,
  // init or set_state)
  int64_t steps_since_check = 0;
  bool mass_ref_valid = false;
  double mass_ref = 0.0;
  int64_t steps_done = 0;  // coarse steps since bind / init / set_state (for messages)
  void reset_check() {
    steps_since_check = 0;
    mass_ref_valid = false;
    steps_done = 0;
    recs_valid = false;
  }
  // the source records momA[parity] of every level hold the moments of the
  // current state (kept by the stream-collide epilogue from one step to the
  // next); cleared by anything else that changes the state, the force or the
  // relaxation rates, and restored by ensure_records()
  bool recs_valid = false;
  void ensure_records();
  // observer called before every op of advance() (records the adjoint tape);
  // with dry set, advance() only walks the op sequence and flips parities
  std::function<void(int op, int level)> hook;
  bool dry = false;
  // per-launch timing: 0 off; 1 every kernel of the step, launched kernel by
  // kernel; 2 steps keep replaying the captured graphs, which then record
  // events around the finest level's stream-collide launches
  int timing = 0;
  bool capturing = false;
  struct Timed {
    int li, kernel;  // lbm::TimedKind
    cudaEvent_t a, b;
  };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // runs launch(), bracketed by events on stream s (default: the bound
  // stream) when the timing mode asks for this launch
  template <class F>
  void timed_launch(int li, int kind, F&& launch, cudaStream_t s = nullptr) {
    const bool finest_sc = li == nlev - 1 && (kind <= lbm::TK_BOUNDARY || kind == lbm::TK_SC_SPAN);
    const bool rec = (timing == 1 && kind != lbm::TK_SC_SPAN) || (timing == 2 && capturing && finest_sc);
    if (!rec) {
      launch();
      return;
    }
    if (!s) s = st;
    Timed t{li, kind, get_event(), get_event()};
    // inside a capture, only an external record becomes an event-record node
    // of the graph (a plain record would just order the captured work)
    const unsigned flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaEventRecordWithFlags(t.a, s, flags);
    launch();
    cudaEventRecordWithFlags(t.b, s, flags);
    timed.push_back(t);
  }
  void recycle_timed() {
    for (auto& t : timed) {
      event_pool.push_back(t.a);
      event_pool.push_back(t.b);
    }
    timed.clear();
  }
  // CUDA graphs of two coarse steps (every level's A/B parity is back where it
  // started after two coarse steps) or of one, per starting parity state;
  // kernel arguments are baked in, so any change of them drops the graphs
  struct StepGraph {
    std::vector<int> parity;  // at the start
    std::vector<int> end;     // after the replay
    int steps;
    cudaGraphExec_t exec;
    int64_t launches;
    std::vector<Timed> timed;  // event pairs recorded by the graph (timing mode 2)
  };
  std::vector<StepGraph> graphs;
  cudaStream_t cap_stream = nullptr;
  // branch streams and fork/join events of the captured graphs, per level:
  // the level's stream-collide runs on branch `sc` (forked after its
  // GhostFromFiner, joined before the ops that read its result), and its three
  // kernels (disjoint elements, same source buffer) on `sc` and the two `side`
  // streams
  struct LevelStreams {
    cudaStream_t sc = nullptr, side[2] = {nullptr, nullptr};
    cudaEvent_t fork_sc = nullptr, done_sc = nullptr, fork = nullptr, join[2] = {nullptr, nullptr};
  };
  std::vector<LevelStreams> lvs;
  bool make_level_streams();
  // copy stream of lbm_init's double-buffered host uploads: copy_ev[0..1]
  // mark each staging half free again, [2] the bound stream's earlier work,
  // [3] a half-chunk's copies done (made on first use; false if unavailable)
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool copy_tried = false;
  bool copy_stream_ready() {
    if (!copy_tried) {
      copy_tried = true;
      bool ok = cudaStreamCreateWithFlags(&copy_st, cudaStreamNonBlocking) == cudaSuccess;
      for (cudaEvent_t& e : copy_ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        if (copy_st) cudaStreamDestroy(copy_st);
        for (cudaEvent_t& e : copy_ev)
          if (e) cudaEventDestroy(e);
        copy_st = nullptr;
        for (cudaEvent_t& e : copy_ev) e = nullptr;
      }
    }
    return copy_st != nullptr;
  }
#ifndef LBM_CONCURRENT_SC
#define LBM_CONCURRENT_SC 1
#endif
  bool concurrent_sc = LBM_CONCURRENT_SC != 0;
  // the finer level's GhostFromCoarser fill at t + 1/2 on the coarse level's
  // stream-collide branch, beside the finer level's first substep (off:
  // measured 35.5 against 32.8 ms per sphere step, the finest stream-collide
  // slowed by its neighbour)
#ifndef LBM_GFC_B_BRANCH
#define LBM_GFC_B_BRANCH 0
#endif
  bool gfc_b_branch = LBM_GFC_B_BRANCH != 0;
  // a level's stream-collide as a graph branch of its own (on: 33.06 against
  // 33.14 ms per sphere step with the level's three kernels forked either way)
#ifndef LBM_LEVEL_BRANCH
#define LBM_LEVEL_BRANCH 1
#endif
  bool level_branch = LBM_LEVEL_BRANCH != 0;
  bool graphs_on = true;
  int last_graph = -1;        // graph of the most recent replay
  bool graph_unread = false;  // its events hold a replay not yet read
  void drop_graphs() {
    for (auto& g : graphs) {
      cudaGraphExecDestroy(g.exec);
      for (auto& t : g.timed) {
        event_pool.push_back(t.a);
        event_pool.push_back(t.b);
      }
    }
    graphs.clear();
    last_graph = -1;
    graph_unread = false;
  }
  ~lbm_ctx() {
    drop_graphs();
    recycle_timed();
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (copy_st) cudaStreamDestroy(copy_st);
    for (cudaEvent_t e : copy_ev)
      if (e) cudaEventDestroy(e);
    for (auto& L : lvs) {
      for (cudaStream_t s : {L.sc, L.side[0], L.side[1]})
        if (s) cudaStreamDestroy(s);
      for (cudaEvent_t e : {L.fork_sc, L.done_sc, L.fork, L.join[0], L.join[1]})
        if (e) cudaEventDestroy(e);
    }
  }

  template <class T = void>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(ws + off);
  }
  void* cur(int li) const { return parity[li] ? at(oB) : at(oA); }
  void* nxt(int li) const { return parity[li] ? at(oA) : at(oB); }
  uint32_t parity_mask() const {
    uint32_t m = 0;
    for (int li = 0; li < nlev; ++li) m |= (uint32_t)(parity[li] & 1) << li;
    return m;
  }
  const void* force_ptr() const { return p.use_force ? at(oF) : nullptr; }

  lbm_status fail(lbm_status s, const std::string& m) {
    err = m;
    return s;
  }
  lbm_status cuda_check(cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LBM_OK;
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return LBM_ERR_CUDA;
  }
  lbm_status launched(const char* where) { return cuda_check(cudaGetLastError(), where); }

  void layout();
  // driver pieces
  void fill_gff(int li);
  // records of the level's sources into mom_off: subset SRC_ALL every
  // source, SRC_GFF the GhostFromFiner ones, SRC_GFF_OUTER those of the outer
  // GhostFromFiner layer
  void source_moments(int li, size_t mom_off, size_t prev_off = 0, cudaStream_t s = nullptr, int subset = 0);
  enum { SRC_ALL = 0, SRC_GFF = 1, SRC_GFF_OUTER = 2 };
  // all_layers false: in LINEAR mode the outer ghost layer, which no
  // stream-collide reads, is left unwritten
  // next_buffer: write the ghosts into the fine level's other buffer (the
  // one its next stream-collide writes, issued before that stream-collide)
  void fill_gfc(int li_fine, bool two_times, bool all_layers = false, cudaStream_t s = nullptr,
                bool next_buffer = false);
  // launches on stream s (default: the bound stream)
  void stream_collide(int li, cudaStream_t s = nullptr);
  void advance(int li);
  // one coarse step from the top: ensure_records(), then advance(0)
  void coarse_step() {
    ensure_records();
    advance(0);
  }
  // graph of nsteps (1 or 2) coarse steps from the current parity state,
  // captured on first use; null when capture is unavailable (the caller
  // steps eagerly)
  const StepGraph* step_graph(int nsteps);
  // n coarse steps as lbm_step issues them (graph replay unless timing mode 1)
  lbm_status run_steps(int64_t n_coarse);
};

