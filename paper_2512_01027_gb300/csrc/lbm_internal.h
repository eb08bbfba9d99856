// Host-side internals shared by the API translation unit and the
// per-precision kernel instantiation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lbm.h"

namespace lbm {

struct Ops;

// Run constants in double, from which the kernels' SiteConsts<R> are made.
struct HostConsts {
    double rho_a, drho, om1, rhoref_T, cP, tau_a, dtau, inv_tau_phi, lambda_b, M3, W, eps, phi_n, phi_m, D,
        dt_pref, A_mu, B_mu, g[3];
    int clamp, full_trace;
};

HostConsts make_consts(const lbm_params &p);

struct Allocator {
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn free_fn = nullptr;
    void *ctx = nullptr;
};

}  // namespace lbm

struct lbm_ctx {
    int lattice = 0, D = 0, Q = 0, storage = 0;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    int periodic[3] = {1, 1, 1};
    lbm_params params{};
    lbm::HostConsts consts{};
    bool has_mask = false;
    int device = 0;
    // device state: ping-pong population sets and fields
    void *h[2] = {nullptr, nullptr};
    void *g[2] = {nullptr, nullptr};
    void *P[2] = {nullptr, nullptr};
    void *u[2] = {nullptr, nullptr};
    void *phi = nullptr;           // phi^{n+1} of the split form [N]
    bool inplace = false;          // one population store, AA streaming
    uint32_t *mask = nullptr;
    int *d_err = nullptr;
    double *d_scratch = nullptr;   // reduction partials + results
    size_t pop_bytes = 0;          // one population set (Q x N)
    size_t field_bytes = 0;        // one scalar field (N)
    int cur = 0;
    int zchunk = 64;
    int zchunk_auto = 64;
    int variant = 0;
    cudaStream_t stream = nullptr;
    int64_t steps = 0;
    std::string err;
    const lbm::Ops *ops = nullptr;
    lbm::Allocator allocator;
    std::vector<void *> owned;
};

namespace lbm {

// Per (lattice, storage) operations, implemented in the instantiation units.
struct Ops {
    int (*init)(lbm_ctx *c, const double *d_phi, const double *d_P, const double *d_u);
    int (*step)(lbm_ctx *c, int64_t n);
    int (*read)(lbm_ctx *c, double *d_phi, double *d_P, double *d_u, double *d_hpop, double *d_gpop);
    int (*reduce)(lbm_ctx *c, double *d_out5);
    int (*pjump)(lbm_ctx *c, const double center[3], double r_in, double r_out, double *d_out4);
    int (*probe)(lbm_ctx *c, const long long *d_sites, int n, double *d_h, double *d_g, double *d_P, double *d_u);
    size_t (*step_smem)();
    bool (*has_v2)();
};

const Ops *ops_f64(int lattice);
const Ops *ops_f32(int lattice);
const Ops *ops_f16(int lattice);
const Ops *ops_bf16(int lattice);

// Device memory through the handle's allocator.
void *dev_alloc(lbm_ctx *c, size_t bytes);
void dev_free(lbm_ctx *c, void *p);

inline int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return LBM_OK;
    if (c) c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

constexpr int kScratchDoubles = 1024 * 8 + 64;

}  // namespace lbm
