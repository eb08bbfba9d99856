// FP32 storage and arithmetic (FMA contraction allowed).
// Compiled once per lattice (LBM_LAT = 0 D2Q9, 1 D3Q19, 2 D3Q27).
#include "lbm_impl.cuh"

namespace lbm {

#if LBM_LAT == 0
const Ops *ops_f32_lat0() { return Impl<D2Q9, float, CodecId<float, true>>::ops(); }
#elif LBM_LAT == 1
const Ops *ops_f32_lat1() { return Impl<D3Q19, float, CodecId<float, true>>::ops(); }
#else
const Ops *ops_f32_lat2() { return Impl<D3Q27, float, CodecId<float, true>>::ops(); }
#endif

}  // namespace lbm
