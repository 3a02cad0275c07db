// BF16 deviation-storage (FP32 arithmetic) instantiation of the hot-path kernels.
#include "kernels.cuh"

namespace lbm {
const Ops* ops_bf16dev() { return dev::make_ops<__nv_bfloat16>(); }
}  // namespace lbm
