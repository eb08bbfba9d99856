// FP64 storage and arithmetic.  Compiled with --fmad=false: every product and
// sum is rounded on its own, in the evaluation order of lbm_site.cuh.
// Compiled once per lattice (LBM_LAT = 0 D2Q9, 1 D3Q19, 2 D3Q27).
#include "lbm_impl.cuh"

namespace lbm {

#if LBM_LAT == 0
const Ops *ops_f64_lat0() { return Impl<D2Q9, double, CodecId<double, false>>::ops(); }
#elif LBM_LAT == 1
const Ops *ops_f64_lat1() { return Impl<D3Q19, double, CodecId<double, false>>::ops(); }
#else
const Ops *ops_f64_lat2() { return Impl<D3Q27, double, CodecId<double, false>>::ops(); }
#endif

}  // namespace lbm
