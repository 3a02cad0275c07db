// lbm_reduce_noalloc: the FP64 reductions of lbm_reduce without any caller-
// provided scratch memory.
//
// Who needs it: callers that may not obtain device memory at the moment they
// want the diagnostics.  Examples are a host framework whose memory manager
// owns every device allocation and forbids raw cudaMalloc, a code path running
// under a fixed device-memory budget that must not grow while a simulation is
// being monitored, or a workspace that was sized for the state alone.  They
// still own the simulation state (bound workspace); this call needs nothing
// more than that state and a host array of eight doubles for the result.
//
// The block partial sums and the final eight values live in a file-scope
// static device array compiled into the library (kRows x 8 + 8 doubles,
// about 256 KiB), which every GPU that loads the library holds until the
// process exits.  The same reduction kernels run as in lbm_reduce, with the
// same fixed grid, so the result is identical.  Limits and sharing rules are
// stated in include/lbm.h next to the declaration.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace {

constexpr int64_t kRows = 4096;  // partial rows: kReduceBlocks per level -> at most 8 levels
constexpr int kMaxDevices = 128;

static __device__ __align__(256) double g_reduce_scratch[kRows * 8 + 8];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_reduce_scratch on the device that holds the workspace.
// Looked up once per device, with that device current; host code may not use
// the symbol itself as a device address.
lbm_status scratch_on(const void* workspace, double** out, std::string* err) {
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, workspace);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    *err = "lbm_reduce_noalloc: bound workspace is not device memory";
    return e != cudaSuccess ? LBM_ERR_CUDA : LBM_ERR_STATE;
  }
  const int dev = attr.device;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = "lbm_reduce_noalloc: device ordinal out of range";
    return LBM_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    int cur = -1;
    e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != dev) e = cudaSetDevice(dev);
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_reduce_scratch);
    if (cur >= 0 && cur != dev) {
      cudaError_t e2 = cudaSetDevice(cur);
      if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess || !p) {
      *err = std::string("lbm_reduce_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return LBM_ERR_CUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_reduce_noalloc(lbm_ctx* ctx, double out[8]) {
  if (!ctx || !out) return LBM_ERR_ARG;
  lbm::ReducePlan plan;
  lbm_status s = lbm::reduce_plan(ctx, &plan);
  if (s != LBM_OK) return s;
  const int64_t rows = (int64_t)plan.levels.size() * lbm::kReduceBlocks;
  if (rows > kRows)
    return lbm::set_error(ctx, LBM_ERR_ARG,
                          "lbm_reduce_noalloc: mesh has " + std::to_string(plan.levels.size()) +
                              " levels; the static scratch holds at most " +
                              std::to_string(kRows / lbm::kReduceBlocks) + " (use lbm_reduce)");
  double* scratch = nullptr;
  std::string err;
  s = scratch_on(plan.workspace, &scratch, &err);
  if (s != LBM_OK) return lbm::set_error(ctx, s, err);
  // Every partial row read by the final sum is written by this call's level
  // kernels first, and the final kernel overwrites the result slot, so nothing
  // has to be cleared between calls.
  for (size_t li = 0; li < plan.levels.size(); ++li) {
    lbm::ReduceArgs a = plan.levels[li];
    a.partial = scratch + li * lbm::kReduceBlocks * 8;
    plan.ops->reduce(plan.Q, a, plan.stream);
  }
  double* result = scratch + kRows * 8;
  lbm::FinalArgs fa{scratch, rows, result};
  lbm::launch_final_reduce(fa, plan.stream);
  lbm::count_launches(ctx, (int64_t)plan.levels.size() + 1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, result, 8 * sizeof(double), cudaMemcpyDeviceToHost, plan.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan.stream);
  if (e != cudaSuccess)
    return lbm::set_error(ctx, LBM_ERR_CUDA, std::string("lbm_reduce_noalloc: ") + cudaGetErrorString(e));
  return LBM_OK;
}
