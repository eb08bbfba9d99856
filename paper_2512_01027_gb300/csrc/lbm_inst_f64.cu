// FP64 storage and arithmetic.  Compiled with --fmad=false: every product and
// sum is rounded on its own, in the evaluation order of lbm_site.cuh.
#include "lbm_impl.cuh"

namespace lbm {

const Ops *ops_f64(int lattice)
{
    switch (lattice) {
    case LBM_D2Q9: return Impl<D2Q9, double, CodecId<double, false>>::ops();
    case LBM_D3Q19: return Impl<D3Q19, double, CodecId<double, false>>::ops();
    case LBM_D3Q27: return Impl<D3Q27, double, CodecId<double, false>>::ops();
    default: return nullptr;
    }
}

}  // namespace lbm
