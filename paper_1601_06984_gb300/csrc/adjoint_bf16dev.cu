// BF16 deviation-storage instantiation of the adjoint kernels (FP32 adjoint).
#include "adjoint.cuh"

namespace lbm {
const AdjOps* adj_ops_bf16dev() { return dev::make_adj_ops<__nv_bfloat16>(); }
}  // namespace lbm
