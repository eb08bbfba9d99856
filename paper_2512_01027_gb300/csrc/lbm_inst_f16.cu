// 16-bit population storage (scaled deviations, FP32 arithmetic).
#include "lbm_impl.cuh"

namespace lbm {

const Ops *ops_f16(int) { return nullptr; }
const Ops *ops_bf16(int) { return nullptr; }

}  // namespace lbm
