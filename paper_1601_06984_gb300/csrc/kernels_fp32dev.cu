// FP32 deviation-storage instantiation of the hot-path kernels.
#include "kernels.cuh"

namespace lbm {
const Ops* ops_fp32dev() { return dev::make_ops<float>(); }
}  // namespace lbm
