// FP64 instantiation of the adjoint kernels, plus the precision-independent
// adjoint helpers (partial accumulation, force gather, record gather).
#include <algorithm>

#include "adjoint.cuh"

namespace lbm {

const AdjOps* adj_ops_fp64() { return dev::make_adj_ops<double>(); }

namespace dev {

// Column sums of the per-block running rows, in block order (one block of
// kAccCols threads per column group: deterministic).
__global__ void __launch_bounds__(256) k_accum(const AccumArgs a) {
  const int col = threadIdx.x % kAccCols, part = threadIdx.x / kAccCols, np = blockDim.x / kAccCols;
  double s = 0.0;
  for (int r = part; r < a.rows; r += np) s += a.partial[(size_t)r * kAccCols + col];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  if (part == 0) {
    for (int k = 1; k < np; ++k) s += sh[k * kAccCols + col];
    a.acc[col] = s;
  }
}

// Row-segment copy: blockIdx.y is the row, x a grid-stride over the segment.
template <class T>
__global__ void __launch_bounds__(256) k_copy_rows(const T* __restrict__ src, T* __restrict__ dst, int64_t pitch,
                                                   int64_t off, int64_t len) {
  const int64_t base = (int64_t)blockIdx.y * pitch + off;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x)
    dst[base + k] = src[base + k];
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

void launch_copy_rows(const void* src, void* dst, size_t pitch, size_t off, size_t len, int rows, size_t elem,
                      cudaStream_t st) {
  if (len == 0 || rows <= 0) return;
  const uintptr_t s0 = reinterpret_cast<uintptr_t>(src) + off, d0 = reinterpret_cast<uintptr_t>(dst) + off;
  size_t w = 16;  // widest access every row start, length and pitch are multiples of
  while (w > elem && ((s0 | d0 | pitch | len) % w)) w /= 2;
  if ((s0 | d0 | pitch | len) % w) w = 1;
  const int64_t n = (int64_t)(len / w);
  // about 8 blocks of 256 per SM over all rows
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)152 * 8 / rows + 1));
  const dim3 grid((unsigned)want, (unsigned)rows);
  const int64_t P = (int64_t)(pitch / w), O = (int64_t)(off / w);
  switch (w) {
    case 16: dev::k_copy_rows<uint4><<<grid, 256, 0, st>>>((const uint4*)src, (uint4*)dst, P, O, n); break;
    case 8: dev::k_copy_rows<uint2><<<grid, 256, 0, st>>>((const uint2*)src, (uint2*)dst, P, O, n); break;
    case 4: dev::k_copy_rows<uint32_t><<<grid, 256, 0, st>>>((const uint32_t*)src, (uint32_t*)dst, P, O, n); break;
    case 2: dev::k_copy_rows<uint16_t><<<grid, 256, 0, st>>>((const uint16_t*)src, (uint16_t*)dst, P, O, n); break;
    default: dev::k_copy_rows<uint8_t><<<grid, 256, 0, st>>>((const uint8_t*)src, (uint8_t*)dst, P, O, n); break;
  }
}

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
