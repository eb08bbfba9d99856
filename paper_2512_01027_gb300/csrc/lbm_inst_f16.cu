// 16-bit population storage (FP16 / BF16 scaled deviations from the lattice
// weights), FP32 arithmetic, FP32 P and u.
#include "lbm_impl.cuh"

namespace lbm {

const Ops *ops_f16(int lattice)
{
    switch (lattice) {
    case LBM_D2Q9: return Impl<D2Q9, float, CodecDev<D2Q9, __half>>::ops();
    case LBM_D3Q19: return Impl<D3Q19, float, CodecDev<D3Q19, __half>>::ops();
    case LBM_D3Q27: return Impl<D3Q27, float, CodecDev<D3Q27, __half>>::ops();
    default: return nullptr;
    }
}

const Ops *ops_bf16(int lattice)
{
    switch (lattice) {
    case LBM_D2Q9: return Impl<D2Q9, float, CodecDev<D2Q9, __nv_bfloat16>>::ops();
    case LBM_D3Q19: return Impl<D3Q19, float, CodecDev<D3Q19, __nv_bfloat16>>::ops();
    case LBM_D3Q27: return Impl<D3Q27, float, CodecDev<D3Q27, __nv_bfloat16>>::ops();
    default: return nullptr;
    }
}

}  // namespace lbm
