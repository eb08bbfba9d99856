// FP32 storage and arithmetic (FMA contraction allowed).
#include "lbm_impl.cuh"

namespace lbm {

const Ops *ops_f32(int lattice)
{
    switch (lattice) {
    case LBM_D2Q9: return Impl<D2Q9, float, CodecId<float, true>>::ops();
    case LBM_D3Q19: return Impl<D3Q19, float, CodecId<float, true>>::ops();
    case LBM_D3Q27: return Impl<D3Q27, float, CodecId<float, true>>::ops();
    default: return nullptr;
    }
}

}  // namespace lbm
