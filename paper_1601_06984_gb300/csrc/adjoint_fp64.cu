// FP64 instantiation of the adjoint kernels, plus the precision-independent
// adjoint helpers (partial accumulation, force gather, record gather).
#include "adjoint.cuh"

namespace lbm {

const AdjOps* adj_ops_fp64() { return dev::make_adj_ops<double>(); }

namespace dev {

// Adds one launch's per-block partial sums, in block order, to the running
// derivative accumulators (one block: deterministic).
__global__ void __launch_bounds__(256) k_accum(const AccumArgs a) {
  double acc[kPartCols];
#pragma unroll
  for (int c = 0; c < kPartCols; ++c) acc[c] = 0.0;
  for (int r = threadIdx.x; r < a.rows; r += blockDim.x)
#pragma unroll
    for (int c = 0; c < kPartCols; ++c) acc[c] += a.partial[(size_t)r * kPartCols + c];
  __shared__ double tot[kPartCols];
  block_sum_store<kPartCols>(acc, tot);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.acc_omega[a.la] += tot[0];
    if (a.lb >= 0) a.acc_omega[a.lb] += tot[1];
    for (int b = 0; b < 3; ++b) a.acc_uin[b] += tot[2 + b];
  }
}

__global__ void k_gather_force_user(const double* lam_force, const int32_t* uslot, double* stage, int64_t first,
                                    int64_t cnt, int64_t Ntot, int d) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t e = uslot[first + t];
  for (int b = 0; b < d; ++b) stage[t * d + b] = lam_force[(size_t)b * Ntot + e];
}

template <class R>
__global__ void k_gather_lam_user(const void* lamA, const void* lamB, uint32_t parity, const int32_t* uslot,
                                  const uint8_t* ulev, double* stage, int64_t first, int64_t cnt, int64_t Ntot,
                                  int Q) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int li = ulev[first + t];
  const R* lam = static_cast<const R*>(((parity >> li) & 1) ? lamB : lamA);
  const int64_t e = uslot[first + t];
  for (int q = 0; q < Q; ++q) stage[t * Q + q] = (double)lam[(size_t)q * Ntot + e];
}

}  // namespace dev

void launch_gather_lam_user(bool fp64, const void* lamA, const void* lamB, uint32_t parity, const int32_t* uslot,
                            const uint8_t* ulev, double* stage, int64_t first, int64_t cnt, int64_t Ntot, int Q,
                            cudaStream_t st) {
  if (cnt <= 0) return;
  const unsigned g = dev::blocks_for(cnt, 256);
  if (fp64) dev::k_gather_lam_user<double><<<g, 256, 0, st>>>(lamA, lamB, parity, uslot, ulev, stage, first, cnt, Ntot, Q);
  else dev::k_gather_lam_user<float><<<g, 256, 0, st>>>(lamA, lamB, parity, uslot, ulev, stage, first, cnt, Ntot, Q);
}

void launch_accum(const AccumArgs& a, cudaStream_t st) { dev::k_accum<<<1, 256, 0, st>>>(a); }

void launch_adj_gather(bool fp64, const AdjGatherArgs& a, cudaStream_t st) {
  if (a.nsrc <= 0) return;
  const unsigned g = dev::blocks_for(a.nsrc, 128);
  if (a.stride == 32) {
    if (fp64) dev::k_adj_gather<double, 32><<<g, 128, 0, st>>>(a);
    else dev::k_adj_gather<float, 32><<<g, 128, 0, st>>>(a);
  } else {
    if (fp64) dev::k_adj_gather<double, 40><<<g, 128, 0, st>>>(a);
    else dev::k_adj_gather<float, 40><<<g, 128, 0, st>>>(a);
  }
}

void launch_gather_force_user(const double* lam_force, const int32_t* uslot, double* stage, int64_t first,
                              int64_t cnt, int64_t Ntot, int d, cudaStream_t st) {
  if (cnt <= 0) return;
  dev::k_gather_force_user<<<dev::blocks_for(cnt, 256), 256, 0, st>>>(lam_force, uslot, stage, first, cnt, Ntot, d);
}

}  // namespace lbm
