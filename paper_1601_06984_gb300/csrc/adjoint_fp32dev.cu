// FP32 deviation-storage instantiation of the adjoint kernels.
#include "adjoint.cuh"

namespace lbm {
const AdjOps* adj_ops_fp32dev() { return dev::make_adj_ops<float>(); }
}  // namespace lbm
