// FP64 instantiation of the hot-path kernels, plus the precision-independent
// helpers (force scatter, final reduction).
#include "kernels.cuh"

namespace lbm {

const Ops* ops_fp64() { return dev::make_ops<double>(); }

namespace dev {

template <class R>
__global__ void k_scatter_force(const ForceArgs a) {
  const int D = a.dim;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.cnt) return;
  const int64_t e = a.uslot[a.first + t];
  R* F = static_cast<R*>(a.force);
  for (int b = 0; b < D; ++b) F[(size_t)b * a.Ntot + e] = R(a.stage[t * D + b]);
}

// Sum of the partial rows in a fixed order (one block): deterministic.
__global__ void __launch_bounds__(256) k_final_reduce(const FinalArgs a) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t r = threadIdx.x; r < a.n; r += blockDim.x)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += a.partial[r * 8 + c];
  block_sum_store<8>(acc, a.out);
}

}  // namespace dev

void launch_scatter_force(bool fp64, const ForceArgs& a, cudaStream_t st) {
  if (a.cnt <= 0) return;
  const unsigned g = dev::blocks_for(a.cnt, 256);
  if (fp64) dev::k_scatter_force<double><<<g, 256, 0, st>>>(a);
  else dev::k_scatter_force<float><<<g, 256, 0, st>>>(a);
}

void launch_final_reduce(const FinalArgs& a, cudaStream_t st) { dev::k_final_reduce<<<1, 256, 0, st>>>(a); }

}  // namespace lbm
