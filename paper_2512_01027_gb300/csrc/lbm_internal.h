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
    int clamp, full_trace, coupling;
};

HostConsts make_consts(const lbm_params &p);

struct Allocator {
    lbm_alloc_fn alloc = nullptr;
    lbm_free_fn free_fn = nullptr;
    void *ctx = nullptr;
};

// Head of a batch's device table (lbm_batch_*): the member count and, per
// launch k of a chunk, the number of work items it covers.
constexpr int kBatchMaxChunk = 64;

struct BatchHeader {
    long long nmem;
    long long span;                       // consecutive 128-site blocks per work item
    long long active[kBatchMaxChunk];
};

constexpr int kBatchMaxSpan = 16;

constexpr size_t batch_header_bytes() { return (sizeof(BatchHeader) + 255) / 256 * 256; }

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
    // FP32 arithmetic: during split stepping the state P, u lives in packed
    // (u, P) words fa[cur]; fb holds (u, phi) of the step being taken and pig
    // the second moments sum_i c_ia c_ib g_i of the pulled g (6 planes in 3D,
    // 3 in 2D).  P[cur], u[cur] are rebuilt from fa[cur] when read.
    void *fa[2] = {nullptr, nullptr};
    void *fb = nullptr;
    void *pig = nullptr;
    int *pctl = nullptr;           // counters of the persistent split step [2 + nz]
    int persist_stall = -1;        // testing aid of the persistent step (lbm_debug_stall)
    void *fg[2] = {nullptr, nullptr};   // BF16 storage: odd part V_g of g* per site (float4), follows cur
    bool g_deferred = false;       // the g store holds g* without its odd part, fg[cur] holds V_g
    bool fa_valid = false;         // fa[cur] holds the state
    bool soa_valid = true;         // P[cur], u[cur] hold the state
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
    int cluster_rows = 0;          // CTAs (rows) per cluster of the cluster step (0: automatic)
    int cluster_zchunk = 0;        // planes per CTA of the cluster step (0: automatic)
    int cluster_stage = 0;         // cluster step with FP32 arithmetic: rows staged by bulk copies (1: on)
    cudaStream_t stream = nullptr;
    int64_t steps = 0;
    std::string err;
    const lbm::Ops *ops = nullptr;
    lbm::Allocator allocator;
    std::vector<void *> owned;
    lbm_batch_ctx *batch = nullptr;   // the batch this handle belongs to, if any
};

// A set of handles stepped together by the batched kernels.
struct lbm_batch_ctx {
    int lattice = 0, storage = 0, device = 0;
    const lbm::Ops *ops = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<lbm_ctx *> members;
    std::vector<int64_t> remaining;   // steps each member still has to take
    std::vector<char> paused;         // members that take no steps for now
    int chunk = 16;                   // steps per chunk (one graph launch)
    bool use_graph = true;
    size_t table_bytes = 0;           // header + capacity members
    size_t cap_members = 0;
    void *d_table = nullptr;
    void *h_table = nullptr;          // pinned staging copy
    std::vector<std::pair<int, cudaGraphExec_t>> graphs;   // per (chunk length, coupled, pp): key 4 K + 2 pp + coupled
    bool coupled = false;             // the current table has a member with the u^{n+1} coupling
    bool pp = false;                  // every member of the current table uses the ping-pong store
    int grid[2] = {0, 0};
    int span = 1;                     // 128-site blocks per work item
    int blocks_per_sm = 0;            // persistent blocks per SM (0: the kernels' occupancy)
    int64_t launches = 0;             // kernels launched so far
    std::string err;
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
    int (*pack)(lbm_ctx *c);       // fa[cur] from P[cur], u[cur] when stale (no-op without packed words)
    int (*sync_soa)(lbm_ctx *c);   // P[cur], u[cur] from fa[cur] when stale (no-op without packed words)
    bool (*persist_ok)(const lbm_ctx *c);   // the persistent split step is available
    int (*split_prepare)(lbm_ctx *c);       // packed words and deferred-g state before split steps
    int (*fold)(lbm_ctx *c);                // g* complete in the store again (BF16 storage)
    // batched persistent launch (lbm_batch_*)
    size_t (*batch_member_bytes)();
    long long (*batch_items)(const lbm_ctx *c, int span);
    void (*batch_fill)(const lbm_ctx *c, int take, long long first_item, void *dst);
    int (*batch_grid)(int phase, int blocks_per_sm);
    // coupled: some member takes the u^{n+1} coupling (a third launch per step)
    // pp: every member uses the ping-pong store
    cudaError_t (*batch_launch)(cudaStream_t s, const void *d_table, int K, int grid0, int grid1, bool coupled,
                                bool pp);
    // cluster step (variant 5) with `rows` CTAs per cluster
    bool (*cluster_ok)(const lbm_ctx *c, int rows);
};

// One instantiation per (storage, lattice); lattice 0 D2Q9, 1 D3Q19, 2 D3Q27.
const Ops *ops_f64_lat0();
const Ops *ops_f64_lat1();
const Ops *ops_f64_lat2();
const Ops *ops_f32_lat0();
const Ops *ops_f32_lat1();
const Ops *ops_f32_lat2();
const Ops *ops_f16_lat0();
const Ops *ops_f16_lat1();
const Ops *ops_f16_lat2();
const Ops *ops_bf16_lat0();
const Ops *ops_bf16_lat1();
const Ops *ops_bf16_lat2();

inline const Ops *ops_for(int lattice, int storage)
{
    static const Ops *(*const table[4][3])() = {
        {ops_f64_lat0, ops_f64_lat1, ops_f64_lat2},
        {ops_f32_lat0, ops_f32_lat1, ops_f32_lat2},
        {ops_f16_lat0, ops_f16_lat1, ops_f16_lat2},
        {ops_bf16_lat0, ops_bf16_lat1, ops_bf16_lat2},
    };
    if (storage < 0 || storage > 3 || lattice < 0 || lattice > 2) return nullptr;
    return table[storage][lattice]();
}

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
