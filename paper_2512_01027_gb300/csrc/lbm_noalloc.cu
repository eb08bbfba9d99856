// Allocation-free variant of the FP64 field reduction (lbm_reduce_fields_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// reduction: real-time loops that must not block in an allocator (cudaMalloc
// and cudaFree can synchronise the device), and hosts whose device memory
// comes from a pool they do not own, where a library allocating on its own
// would break the host's accounting.  This entry point takes its inputs and
// its output from the caller and keeps the per-block partial sums in a fixed
// array in device global memory instead of allocating them.
//
// The array below is a file-scope __device__ variable: every GPU that loads
// this library holds it (40 KB) until the process exits.  In host code its name
// is only a host-side stand-in, not a device address; the device address is
// obtained per device with cudaGetSymbolAddress on the first call made with
// that device current, and cached for as long as the device's context lives:
// after a cudaDeviceReset the library has to be loaded again.
#include <mutex>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {
namespace {

// Partial sums of at most kStaticBlocks blocks, kRedVals values each.
constexpr int kStaticBlocks = 1024;
constexpr long long kStaticMaxSites = (1LL << 31) - 1;

__device__ __align__(256) double g_static_partials[kStaticBlocks * kRedVals];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_dev_ptr[kMaxDevices] = {};

// Device address of g_static_partials on the current device (set up once per device).
cudaError_t static_partials(double **out, std::string *why)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *why = "cudaGetDevice failed"; return e; }
    if (dev < 0 || dev >= kMaxDevices) { *why = "device index beyond 64"; return cudaErrorInvalidDevice; }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) { *why = "cudaGetSymbolAddress(static partials) failed"; return e; }
        g_dev_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

// Same sums as the handle's reduction: phi, rho(phi) u_x, u_y, u_z, fluid sites.
__global__ void __launch_bounds__(kRedThreads) field_sums_kernel(const double *phi, const double *u,
                                                                  const uint8_t *solid, long long n, double rho_a,
                                                                  double drho, int clamp, double *partials)
{
    __shared__ double sh[kRedVals * kRedThreads];
    double v[kRedVals] = {0, 0, 0, 0, 0};
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        if (solid && solid[idx]) continue;
        const double p = phi[idx];
        const double ph = clamp ? fmin(1.0, fmax(0.0, p)) : p;
        const double rho = rho_a + ph * drho;
        v[0] += p;
        v[1] += rho * u[idx];
        v[2] += rho * u[n + idx];
        v[3] += rho * u[2 * n + idx];
        v[4] += 1.0;
    }
    block_sum<kRedVals>(v, sh);
    if (threadIdx.x == 0)
        for (int j = 0; j < kRedVals; ++j) partials[(long long)blockIdx.x * kRedVals + j] = v[j];
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_reduce_fields_noalloc(const double *d_phi, const double *d_u, const uint8_t *d_solid, int64_t n,
                                         double rho_w, double rho_a, int32_t clamp_phi_props, double *d_out,
                                         void *stream)
{
    using namespace lbm;
    if (!d_phi || !d_u || !d_out) return LBM_ERR_INVALID_ARG;
    if (n <= 0 || n > kStaticMaxSites) return LBM_ERR_INVALID_ARG;   // 1 <= n <= 2^31 - 1 sites
    if (!(rho_w > rho_a) || !(rho_a > 0)) return LBM_ERR_INVALID_ARG;
    double *partials = nullptr;
    std::string why;
    if (static_partials(&partials, &why) != cudaSuccess) return LBM_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int blocks = (int)std::min<long long>(kStaticBlocks, (n + kRedThreads - 1) / kRedThreads);
    // every block writes its own partial vector before the second pass reads
    // exactly `blocks` of them, so nothing in the array needs clearing
    // Launch errors are read with cudaPeekAtLastError, which leaves the
    // thread's error state as it is: an error already pending from earlier
    // work also makes this call return LBM_ERR_CUDA, and stays pending for
    // the caller's own checks.
    field_sums_kernel<<<blocks, kRedThreads, 0, s>>>(d_phi, d_u, d_solid, (long long)n, rho_a, rho_w - rho_a,
                                                     clamp_phi_props ? 1 : 0, partials);
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ERR_CUDA;
    finish_kernel<kRedVals><<<1, kRedThreads, 0, s>>>(partials, blocks, d_out);
    return cudaPeekAtLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
