// 16-bit population storage (FP16 / BF16 scaled deviations from the lattice
// weights), FP32 arithmetic, FP32 P and u.  Compiled once per lattice
// (LBM_LAT = 0 D2Q9, 1 D3Q19, 2 D3Q27) and 16-bit type (LBM_BF16 = 0 FP16,
// 1 BF16).
#include "lbm_impl.cuh"

namespace lbm {

#if LBM_BF16
using Half16 = __nv_bfloat16;
#define LBM_OPS_NAME(l) ops_bf16_lat##l
#else
using Half16 = __half;
#define LBM_OPS_NAME(l) ops_f16_lat##l
#endif

#if LBM_LAT == 0
const Ops *LBM_OPS_NAME(0)() { return Impl<D2Q9, float, CodecDev<D2Q9, Half16>>::ops(); }
#elif LBM_LAT == 1
const Ops *LBM_OPS_NAME(1)() { return Impl<D3Q19, float, CodecDev<D3Q19, Half16>>::ops(); }
#else
const Ops *LBM_OPS_NAME(2)() { return Impl<D3Q27, float, CodecDev<D3Q27, Half16>>::ops(); }
#endif

}  // namespace lbm
