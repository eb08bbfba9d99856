// extern "C" API of the coupled LB step library (see include/lbm.h).
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_lattice.cuh"

namespace lbm {

namespace {
std::mutex g_alloc_mu;
Allocator g_alloc;                       // hooks for later lbm_create calls
thread_local std::string g_create_err;   // last lbm_create failure on this thread
}  // namespace

HostConsts make_consts(const lbm_params &p)
{
    HostConsts h;
    h.rho_a = p.rho_a;
    h.drho = p.rho_w - p.rho_a;
    h.om1 = p.rho_w / p.rho_a - 1.0;            // omega_max - 1, omega_max = rho_w / rho_a
    h.rhoref_T = p.rho_a * (1.0 / 3.0);         // rho_ref T
    h.cP = 3.0 / p.rho_a;                       // 1 / (rho_ref T)
    const double tau_w = p.nu_w * 3.0 + 0.5;    // nu / T + 1/2
    const double tau_a = p.nu_a * 3.0 + 0.5;
    h.tau_a = tau_a;
    h.dtau = tau_w - tau_a;
    h.inv_tau_phi = 1.0 / (p.M * 3.0 + 0.5);    // 1 / (M / T + 1/2)
    h.lambda_b = p.lambda_b;
    h.M3 = p.M * 3.0;
    h.W = p.W;
    h.eps = p.eps;
    h.phi_n = p.phi_n;
    h.phi_m = p.phi_m;
    h.D = p.D;
    h.dt_pref = p.gamma * p.M * 3.0 / p.W;      // gamma M / (T W)
    h.A_mu = 48.0 * p.sigma / p.W;
    h.B_mu = 1.5 * p.sigma * p.W;
    h.g[0] = p.g_ext[0];
    h.g[1] = p.g_ext[1];
    h.g[2] = p.g_ext[2];
    h.clamp = p.clamp_phi_props ? 1 : 0;
    h.full_trace = p.filter_full_trace ? 1 : 0;
    h.coupling = p.coupling_unew ? 1 : 0;
    return h;
}

void *dev_alloc(lbm_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    void *p = nullptr;
    if (c->allocator.alloc) {
        p = c->allocator.alloc(bytes, c->allocator.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void dev_free(lbm_ctx *c, void *p)
{
    if (!p) return;
    if (c->allocator.free_fn) c->allocator.free_fn(p, c->allocator.ctx);
    else cudaFree(p);
}

// Neighbour mask: bit i set when x - c_i is solid or outside a non-periodic
// edge; bit 31 set when x itself is solid.
template <class L>
__global__ void mask_kernel(const uint8_t *solid, uint32_t *mask, int nx, int ny, int nz, int px, int py, int pz,
                            long long N)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((long long)nx * ny));
    uint32_t m = (solid && solid[idx]) ? kSolidBit : 0u;
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        int xx = x - L::c(i, 0), yy = y - L::c(i, 1), zz = z - L::c(i, 2);
        bool out = false;
        if (xx < 0 || xx >= nx) { if (px) xx = wrapc(xx, nx); else out = true; }
        if (yy < 0 || yy >= ny) { if (py) yy = wrapc(yy, ny); else out = true; }
        if (zz < 0 || zz >= nz) { if (pz) zz = wrapc(zz, nz); else out = true; }
        if (!out && solid) out = solid[((long long)zz * ny + yy) * nx + xx] != 0;
        if (out) m |= (1u << i);
    });
    mask[idx] = m;
}

}  // namespace lbm

using namespace lbm;

namespace {

int fail(lbm_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

int lattice_dims(int lattice, int *D, int *Q)
{
    switch (lattice) {
    case LBM_D2Q9: *D = 2; *Q = 9; return 0;
    case LBM_D3Q19: *D = 3; *Q = 19; return 0;
    case LBM_D3Q27: *D = 3; *Q = 27; return 0;
    default: return -1;
    }
}

size_t storage_bytes(int storage)
{
    switch (storage) {
    case LBM_STORE_F64: return 8;
    case LBM_STORE_F32: return 4;
    case LBM_STORE_F16DEV:
    case LBM_STORE_BF16DEV: return 2;
    default: return 0;
    }
}

size_t compute_bytes(int storage) { return storage == LBM_STORE_F64 ? 8 : 4; }

// Device bytes of a handle: population sets, P and u (two each), phi,
// reduction scratch, error flag, and the neighbour mask when there is one.
size_t footprint_bytes(int Q, int D, long long N, int nz, int storage, bool inplace, bool has_mask)
{
    const size_t pop = (size_t)Q * (size_t)N * storage_bytes(storage);
    const size_t field = (size_t)N * compute_bytes(storage);
    size_t s = (inplace ? 2 : 4) * pop + (3 + 2 * (size_t)D) * field + sizeof(double) * kScratchDoubles + 256;
    // FP32 arithmetic: packed (u, P) ping-pong, packed (u, phi), second moments of g
    if (storage != LBM_STORE_F64) s += (2 * 16 + 16 + 4 * (D == 3 ? 6 : 3)) * (size_t)N + 4 * (2 + (size_t)nz);
    // BF16 storage: odd part of g per site, ping-pong
    if (storage == LBM_STORE_BF16DEV) s += 2 * 16 * (size_t)N;
    if (has_mask) s += sizeof(uint32_t) * (size_t)N;
    return s;
}

void release(lbm_ctx *c)
{
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    for (void *p : c->owned) dev_free(c, p);
    c->owned.clear();
}

void *own(lbm_ctx *c, size_t bytes)
{
    void *p = dev_alloc(c, bytes);
    if (p) c->owned.push_back(p);
    return p;
}

int sync_and_check(lbm_ctx *c)
{
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy(err flag)");
    if (flag & 2)
        return fail(c, LBM_ERR_TIMEOUT, "a bounded wait of the persistent or cluster step ran out (results invalid)");
    if (flag) return fail(c, LBM_ERR_NONFINITE, "a step produced a non-finite phi, P or u");
    return LBM_OK;
}

// Staging memory of the host-field calls: one stream-ordered pool per device
// that keeps what it has allocated (release threshold unbounded), so a call
// reuses the previous call's memory instead of paying a cudaMalloc and a
// synchronising cudaFree of the fields' size.  Held: the largest staging area
// used so far on the device (40 B per site of the largest lattice).
cudaMemPool_t staging_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
    }
    return pools[dev];
}

// Temporary device buffer of one call: from the staging pool, freed in
// stream order at scope exit; with an allocator hook set, from the hook,
// released after the stream drains.
struct Temp {
    lbm_ctx *c;
    void *p = nullptr;
    bool pooled = false;
    Temp(lbm_ctx *ctx, size_t bytes) : c(ctx)
    {
        if (!c->allocator.alloc) {
            cudaMemPool_t pool = staging_pool(c->device);
            if (pool && cudaMallocFromPoolAsync(&p, bytes, pool, c->stream) == cudaSuccess) {
                pooled = true;
                return;
            }
            cudaGetLastError();
            p = nullptr;
        }
        p = dev_alloc(c, bytes);
    }
    ~Temp()
    {
        if (!p) return;
        if (pooled) {
            cudaFreeAsync(p, c->stream);
        } else {
            cudaStreamSynchronize(c->stream);
            dev_free(c, p);
        }
    }
    double *d() const { return static_cast<double *>(p); }
};

}  // namespace

extern "C" {

int lbm_default_params(lbm_params *p)
{
    if (!p) return LBM_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(lbm_params);
    p->rho_w = 1.0;
    p->rho_a = 1e-3;
    p->nu_w = 0.0167;
    p->nu_a = 0.167;
    p->sigma = 1e-3;
    p->M = 0.166;
    p->W = 4.0;
    p->lambda_b = 1.0 / 6.0;
    p->gamma = -22.5;
    p->phi_n = 0.8;
    p->phi_m = 0.2;
    p->D = 1e-4;
    p->eps = 1e-10;
    p->clamp_phi_props = 1;
    p->filter_full_trace = 0;
    p->storage = LBM_STORE_F32;
    return LBM_OK;
}

int lbm_lattice_info(int lattice, int *d, int *Q, int *c, double *w)
{
    int D = 0, q = 0;
    if (lattice_dims(lattice, &D, &q) != 0) return LBM_ERR_INVALID_ARG;
    if (d) *d = D;
    if (Q) *Q = q;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) {
            const int v = (lattice == LBM_D2Q9) ? D2Q9::c(i, a) : detail::c3(i, a);
            if (c) c[3 * i + a] = v;
        }
        if (w) w[i] = (lattice == LBM_D2Q9) ? D2Q9::w(i) : (lattice == LBM_D3Q19 ? D3Q19::w(i) : D3Q27::w(i));
    }
    return LBM_OK;
}

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return LBM_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_fn = free_fn;
    g_alloc.ctx = ctx;
    return LBM_OK;
}

int lbm_create(const lbm_grid *grid, int lattice, const lbm_params *params, lbm_handle *out)
{
    if (!out) return fail(nullptr, LBM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !params) return fail(nullptr, LBM_ERR_INVALID_ARG, "grid or params is NULL");
    if (params->struct_size != sizeof(lbm_params))
        return fail(nullptr, LBM_ERR_INVALID_ARG, "params->struct_size != sizeof(lbm_params)");
    int D = 0, Q = 0;
    if (lattice_dims(lattice, &D, &Q) != 0) return fail(nullptr, LBM_ERR_INVALID_ARG, "unknown lattice");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (D == 2 && grid->nz != 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "2D lattice needs nz == 1");
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 31) - 1) return fail(nullptr, LBM_ERR_INVALID_ARG, "grid too large (N >= 2^31)");
    const lbm_params &p = *params;
    if (!(p.rho_a > 0) || !(p.rho_w > p.rho_a) || !(p.nu_w > 0) || !(p.nu_a > 0) || !(p.M > 0) || !(p.W > 0) ||
        !(p.D > 0) || !(p.eps >= 0) || !std::isfinite(p.sigma))
        return fail(nullptr, LBM_ERR_INVALID_ARG,
                    "invalid parameters (need rho_w > rho_a > 0, nu > 0, M > 0, W > 0, D > 0)");
    const int storage = p.storage;
    if (storage_bytes(storage) == 0 || (p.inplace != 0 && p.inplace != 1) ||
        (p.coupling_unew != 0 && p.coupling_unew != 1))
        return fail(nullptr, LBM_ERR_INVALID_ARG, "unknown storage, or inplace / coupling_unew not 0/1");
    const Ops *ops = ops_for(lattice, storage);
    if (!ops) return fail(nullptr, LBM_ERR_UNSUPPORTED, "lattice/storage combination not built");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(nullptr, LBM_ERR_CUDA, std::string("no usable CUDA device: ") +
                                               (e == cudaSuccess ? "0 devices" : cudaGetErrorString(e)));
    }

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    cudaGetDevice(&c->device);
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->allocator = g_alloc;
    }
    c->lattice = lattice; c->D = D; c->Q = Q; c->storage = storage;
    c->nx = grid->nx; c->ny = grid->ny; c->nz = grid->nz; c->N = N;
    for (int a = 0; a < 3; ++a) c->periodic[a] = grid->periodic[a] ? 1 : 0;
    if (D == 2) c->periodic[2] = 1;
    c->params = p;
    c->consts = make_consts(p);
    c->ops = ops;
    bool any_solid = false;
    if (grid->solid)
        for (long long i = 0; i < N && !any_solid; ++i) any_solid = grid->solid[i] != 0;
    c->has_mask = any_solid || !c->periodic[0] || !c->periodic[1] || !c->periodic[2];
    // z chunk of the fused step: enough CTAs for several waves on the device
    if (D == 3) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const long long tiles = (long long)((c->nx + 29) / 30) * ((c->ny + 5) / 6);
        const long long want = 8LL * sms;
        long long chunks = (want + tiles - 1) / tiles;
        if (chunks < 1) chunks = 1;
        long long zc = (c->nz + chunks - 1) / chunks;
        if (zc < 8) zc = 8;
        if (zc > c->nz) zc = c->nz;
        c->zchunk = (int)zc;
    } else {
        c->zchunk = 1;
    }
    c->zchunk_auto = c->zchunk;

    const size_t sb = storage_bytes(storage), cb = compute_bytes(storage);
    c->pop_bytes = (size_t)Q * (size_t)N * sb;
    c->field_bytes = (size_t)N * cb;
    c->inplace = p.inplace == 1;
    for (int b = 0; b < 2; ++b) {
        if (b == 1 && c->inplace) {
            c->h[1] = c->h[0];
            c->g[1] = c->g[0];
        } else {
            c->h[b] = own(c, c->pop_bytes);
            c->g[b] = own(c, c->pop_bytes);
        }
        c->P[b] = own(c, c->field_bytes);
        c->u[b] = own(c, c->field_bytes * D);
        if (!c->h[b] || !c->g[b] || !c->P[b] || !c->u[b]) {
            g_create_err = "device allocation of the population store failed";
            release(c);
            delete c;
            return LBM_ERR_OOM;
        }
    }
    c->phi = own(c, c->field_bytes);
    if (storage != LBM_STORE_F64 && c->phi) {
        c->fa[0] = own(c, 16 * (size_t)N);
        c->fa[1] = own(c, 16 * (size_t)N);
        c->fb = own(c, 16 * (size_t)N);
        c->pig = own(c, 4 * (size_t)(D == 3 ? 6 : 3) * (size_t)N);
        c->pctl = static_cast<int *>(own(c, sizeof(int) * (2 + (size_t)c->nz)));
        if (storage == LBM_STORE_BF16DEV) {
            c->fg[0] = own(c, 16 * (size_t)N);
            c->fg[1] = own(c, 16 * (size_t)N);
            if (!c->fg[0] || !c->fg[1]) c->phi = nullptr;
        }
        if (!c->fa[0] || !c->fa[1] || !c->fb || !c->pig || !c->pctl) c->phi = nullptr;
    }
    if (!c->phi) {
        g_create_err = "device allocation of the phi field or the packed words failed";
        release(c);
        delete c;
        return LBM_ERR_OOM;
    }
    c->d_err = static_cast<int *>(own(c, 256));
    c->d_scratch = static_cast<double *>(own(c, sizeof(double) * kScratchDoubles));
    if (!c->d_err || !c->d_scratch) {
        g_create_err = "device allocation failed";
        release(c);
        delete c;
        return LBM_ERR_OOM;
    }
    int rc = LBM_OK;
    for (int b = 0; b < 2 && rc == LBM_OK; ++b) {
        if (!(b == 1 && c->inplace)) {
            rc = cuda_fail(c, cudaMemset(c->h[b], 0, c->pop_bytes), "cudaMemset");
            if (rc == LBM_OK) rc = cuda_fail(c, cudaMemset(c->g[b], 0, c->pop_bytes), "cudaMemset");
        }
        if (rc == LBM_OK) rc = cuda_fail(c, cudaMemset(c->P[b], 0, c->field_bytes), "cudaMemset");
        if (rc == LBM_OK) rc = cuda_fail(c, cudaMemset(c->u[b], 0, c->field_bytes * D), "cudaMemset");
    }
    if (rc == LBM_OK) rc = cuda_fail(c, cudaMemset(c->d_err, 0, sizeof(int)), "cudaMemset");
    if (rc == LBM_OK && c->has_mask) {
        c->mask = static_cast<uint32_t *>(own(c, sizeof(uint32_t) * (size_t)N));
        void *dsolid = nullptr;
        if (!c->mask) rc = LBM_ERR_OOM;
        if (rc == LBM_OK && grid->solid) {
            dsolid = dev_alloc(c, (size_t)N);
            if (!dsolid) rc = LBM_ERR_OOM;
            else rc = cuda_fail(c, cudaMemcpy(dsolid, grid->solid, (size_t)N, cudaMemcpyHostToDevice), "cudaMemcpy(solid)");
        }
        if (rc == LBM_OK) {
            const int t = 256;
            const unsigned blocks = (unsigned)((N + t - 1) / t);
            const uint8_t *s = static_cast<const uint8_t *>(dsolid);
            const int px = c->periodic[0], py = c->periodic[1], pz = c->periodic[2];
            if (lattice == LBM_D2Q9) mask_kernel<D2Q9><<<blocks, t>>>(s, c->mask, c->nx, c->ny, c->nz, px, py, pz, N);
            else if (lattice == LBM_D3Q19) mask_kernel<D3Q19><<<blocks, t>>>(s, c->mask, c->nx, c->ny, c->nz, px, py, pz, N);
            else mask_kernel<D3Q27><<<blocks, t>>>(s, c->mask, c->nx, c->ny, c->nz, px, py, pz, N);
            rc = cuda_fail(c, cudaGetLastError(), "mask_kernel launch");
            if (rc == LBM_OK) rc = cuda_fail(c, cudaDeviceSynchronize(), "mask_kernel");
        }
        if (dsolid) dev_free(c, dsolid);
    }
    if (rc != LBM_OK) {
        g_create_err = c->err.empty() ? "device setup failed" : c->err;
        release(c);
        delete c;
        return rc;
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (h->batch) lbm_batch_remove(h->batch, h);
    release(h);
    delete h;
    return LBM_OK;
}

int lbm_set_stream(lbm_handle h, void *cuda_stream)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return LBM_OK;
}

int lbm_init_fields_device(lbm_handle h, const double *d_phi, const double *d_P, const double *d_u)
{
    if (!h || !d_phi || !d_P || !d_u) return h ? fail(h, LBM_ERR_INVALID_ARG, "NULL field") : LBM_ERR_INVALID_ARG;
    int rc = cuda_fail(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "cudaMemsetAsync(err)");
    if (rc != LBM_OK) return rc;
    return h->ops->init(h, d_phi, d_P, d_u);
}

int lbm_init_fields(lbm_handle h, const double *phi, const double *P, const double *u)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (!phi || !P || !u) return fail(h, LBM_ERR_INVALID_ARG, "NULL field");
    const size_t n = (size_t)h->N;
    Temp t(h, sizeof(double) * 5 * n);
    if (!t.p) return fail(h, LBM_ERR_OOM, "temporary device buffer");
    double *d = t.d();
    int rc = cuda_fail(h, cudaMemcpyAsync(d, phi, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "H2D phi");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(d + n, P, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "H2D P");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(d + 2 * n, u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream), "H2D u");
    if (rc == LBM_OK) rc = lbm_init_fields_device(h, d, d + n, d + 2 * n);
    // the caller may reuse phi, P, u as soon as this returns
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_step(lbm_handle h, int64_t n)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (n < 0) return fail(h, LBM_ERR_INVALID_ARG, "n < 0");
    if (h->batch) return fail(h, LBM_ERR_INVALID_ARG, "the handle is stepped by its batch (lbm_batch_step)");
    return h->ops->step(h, n);
}

int lbm_read_fields_device(lbm_handle h, double *d_phi, double *d_P, double *d_u)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    return h->ops->read(h, d_phi, d_P, d_u, nullptr, nullptr);
}

int lbm_read_fields(lbm_handle h, double *phi, double *P, double *u)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)h->N;
    Temp t(h, sizeof(double) * 5 * n);
    if (!t.p) return fail(h, LBM_ERR_OOM, "temporary device buffer");
    double *d = t.d();
    int rc = h->ops->read(h, phi ? d : nullptr, P ? d + n : nullptr, u ? d + 2 * n : nullptr, nullptr, nullptr);
    if (rc == LBM_OK && phi) rc = cuda_fail(h, cudaMemcpyAsync(phi, d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream), "D2H phi");
    if (rc == LBM_OK && P) rc = cuda_fail(h, cudaMemcpyAsync(P, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream), "D2H P");
    if (rc == LBM_OK && u) rc = cuda_fail(h, cudaMemcpyAsync(u, d + 2 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream), "D2H u");
    if (rc != LBM_OK) return rc;
    return sync_and_check(h);
}

int lbm_steps_done(lbm_handle h, int64_t *steps)
{
    if (!h || !steps) return LBM_ERR_INVALID_ARG;
    *steps = h->steps;
    return LBM_OK;
}

int lbm_check(lbm_handle h)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    return sync_and_check(h);
}

int lbm_reduce(lbm_handle h, double out[5])
{
    if (!h || !out) return LBM_ERR_INVALID_ARG;
    double *d_out = h->d_scratch + (kScratchDoubles - 16);
    int rc = h->ops->reduce(h, d_out);
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(out, d_out, sizeof(double) * 5, cudaMemcpyDeviceToHost, h->stream), "D2H reduce");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_pressure_jump(lbm_handle h, const double center[3], double r_in, double r_out, double *dP)
{
    if (!h || !center || !dP) return LBM_ERR_INVALID_ARG;
    if (!(r_in > 0) || !(r_out >= r_in)) return fail(h, LBM_ERR_INVALID_ARG, "need 0 < r_in <= r_out");
    double *d_out = h->d_scratch + (kScratchDoubles - 16);
    double v[4];
    int rc = h->ops->pjump(h, center, r_in, r_out, d_out);
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(v, d_out, sizeof(v), cudaMemcpyDeviceToHost, h->stream), "D2H pjump");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc != LBM_OK) return rc;
    if (v[1] <= 0 || v[3] <= 0) return fail(h, LBM_ERR_INVALID_ARG, "no fluid site inside r_in or outside r_out");
    *dP = v[0] / v[1] - v[2] / v[3];
    return LBM_OK;
}

int lbm_get_state(lbm_handle h, double *h_pop, double *g_pop, double *P, double *u)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    const size_t n = (size_t)h->N, q = (size_t)h->Q;
    Temp t(h, sizeof(double) * (2 * q + 4) * n);
    if (!t.p) return fail(h, LBM_ERR_OOM, "temporary device buffer");
    double *d = t.d();
    double *dh = d, *dg = d + q * n, *dP = d + 2 * q * n, *du = d + (2 * q + 1) * n;
    int rc = h->ops->read(h, nullptr, dP, du, dh, dg);
    if (rc == LBM_OK && h_pop) rc = cuda_fail(h, cudaMemcpyAsync(h_pop, dh, sizeof(double) * q * n, cudaMemcpyDeviceToHost, h->stream), "D2H h");
    if (rc == LBM_OK && g_pop) rc = cuda_fail(h, cudaMemcpyAsync(g_pop, dg, sizeof(double) * q * n, cudaMemcpyDeviceToHost, h->stream), "D2H g");
    if (rc == LBM_OK && P) rc = cuda_fail(h, cudaMemcpyAsync(P, dP, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream), "D2H P");
    if (rc == LBM_OK && u) rc = cuda_fail(h, cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream), "D2H u");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int lbm_probe(lbm_handle h, int64_t n, const int64_t *sites, double *h_pop, double *g_pop, double *P, double *u)
{
    if (!h || !sites || n < 0) return LBM_ERR_INVALID_ARG;
    if (n == 0) return LBM_OK;
    if (n > (1LL << 30)) return fail(h, LBM_ERR_INVALID_ARG, "too many probe sites");
    for (int64_t j = 0; j < n; ++j)
        if (sites[j] < 0 || sites[j] >= h->N) return fail(h, LBM_ERR_INVALID_ARG, "probe site out of range");
    const size_t q = (size_t)h->Q, m = (size_t)n;
    Temp t(h, sizeof(double) * (2 * q + 4) * m + sizeof(long long) * m);
    if (!t.p) return fail(h, LBM_ERR_OOM, "temporary device buffer");
    double *d = t.d();
    double *dh = d, *dg = d + q * m, *dP = d + 2 * q * m, *du = d + (2 * q + 1) * m;
    long long *ds = reinterpret_cast<long long *>(d + (2 * q + 4) * m);
    int rc = cuda_fail(h, cudaMemcpyAsync(ds, sites, sizeof(long long) * m, cudaMemcpyHostToDevice, h->stream), "H2D sites");
    if (rc == LBM_OK) rc = h->ops->probe(h, ds, (int)n, dh, dg, dP, du);
    if (rc == LBM_OK && h_pop) rc = cuda_fail(h, cudaMemcpyAsync(h_pop, dh, sizeof(double) * q * m, cudaMemcpyDeviceToHost, h->stream), "D2H probe");
    if (rc == LBM_OK && g_pop) rc = cuda_fail(h, cudaMemcpyAsync(g_pop, dg, sizeof(double) * q * m, cudaMemcpyDeviceToHost, h->stream), "D2H probe");
    if (rc == LBM_OK && P) rc = cuda_fail(h, cudaMemcpyAsync(P, dP, sizeof(double) * m, cudaMemcpyDeviceToHost, h->stream), "D2H probe");
    if (rc == LBM_OK && u) rc = cuda_fail(h, cudaMemcpyAsync(u, du, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, h->stream), "D2H probe");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

// Checkpoint header: identifies the layout the raw bytes after it are in.
struct StateHeader {
    char magic[8];                 // "LBMSTATE"
    int32_t version, lattice, storage, inplace;
    int32_t nx, ny, nz, reserved;
};
static_assert(sizeof(StateHeader) == 40, "state header layout");

static StateHeader state_header(lbm_handle h)
{
    StateHeader s{};
    std::memcpy(s.magic, "LBMSTATE", 8);
    s.version = 1;
    s.lattice = h->lattice;
    s.storage = h->storage;
    s.inplace = h->inplace ? 1 : 0;
    s.nx = h->nx;
    s.ny = h->ny;
    s.nz = h->nz;
    return s;
}

int lbm_state_bytes(lbm_handle h, size_t *bytes)
{
    if (!h || !bytes) return LBM_ERR_INVALID_ARG;
    *bytes = sizeof(StateHeader) + 2 * h->pop_bytes + (size_t)(1 + h->D) * h->field_bytes + sizeof(int64_t);
    return LBM_OK;
}

int lbm_save_state(lbm_handle h, void *host_buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !host_buf) return LBM_ERR_INVALID_ARG;
    lbm_state_bytes(h, &need);
    if (bytes != need) return fail(h, LBM_ERR_INVALID_ARG, "buffer size != lbm_state_bytes");
    char *p = static_cast<char *>(host_buf);
    const StateHeader hd = state_header(h);
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    if (const int rs = h->ops->sync_soa(h); rs != LBM_OK) return rs;
    if (const int rf = h->ops->fold(h); rf != LBM_OK) return rf;
    const int b = h->cur;
    int rc = cuda_fail(h, cudaMemcpyAsync(p, h->h[b], h->pop_bytes, cudaMemcpyDeviceToHost, h->stream), "D2H state");
    p += h->pop_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(p, h->g[b], h->pop_bytes, cudaMemcpyDeviceToHost, h->stream), "D2H state");
    p += h->pop_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(p, h->P[b], h->field_bytes, cudaMemcpyDeviceToHost, h->stream), "D2H state");
    p += h->field_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(p, h->u[b], h->field_bytes * h->D, cudaMemcpyDeviceToHost, h->stream), "D2H state");
    p += h->field_bytes * h->D;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc == LBM_OK) std::memcpy(p, &h->steps, sizeof(int64_t));
    return rc;
}

int lbm_load_state(lbm_handle h, const void *host_buf, size_t bytes)
{
    size_t need = 0;
    if (!h || !host_buf) return LBM_ERR_INVALID_ARG;
    lbm_state_bytes(h, &need);
    if (bytes != need) return fail(h, LBM_ERR_INVALID_ARG, "buffer size != lbm_state_bytes");
    const char *p = static_cast<const char *>(host_buf);
    const StateHeader want = state_header(h);
    if (std::memcmp(p, &want, sizeof want) != 0)
        return fail(h, LBM_ERR_INVALID_ARG, "state was saved by a handle of another lattice, grid, storage or layout");
    p += sizeof want;
    const int b = h->cur;
    int rc = cuda_fail(h, cudaMemcpyAsync(h->h[b], p, h->pop_bytes, cudaMemcpyHostToDevice, h->stream), "H2D state");
    p += h->pop_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(h->g[b], p, h->pop_bytes, cudaMemcpyHostToDevice, h->stream), "H2D state");
    p += h->pop_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(h->P[b], p, h->field_bytes, cudaMemcpyHostToDevice, h->stream), "H2D state");
    p += h->field_bytes;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemcpyAsync(h->u[b], p, h->field_bytes * h->D, cudaMemcpyHostToDevice, h->stream), "H2D state");
    p += h->field_bytes * h->D;
    if (rc == LBM_OK) rc = cuda_fail(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream), "cudaMemsetAsync(err)");
    if (rc == LBM_OK) rc = cuda_fail(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (rc == LBM_OK) std::memcpy(&h->steps, p, sizeof(int64_t));
    h->fa_valid = false;
    h->soa_valid = true;
    h->g_deferred = false;
    return rc;
}

int lbm_set_tuning(lbm_handle h, int variant, int zchunk)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (variant < 0 || variant > 5 || zchunk < 0) return fail(h, LBM_ERR_INVALID_ARG, "variant in 0..5, zchunk >= 0");
    if (variant == 5) {
        if (h->consts.coupling)
            return fail(h, LBM_ERR_UNSUPPORTED, "coupling_unew = 1 steps in the split form only");
        bool ok = false;
        if (h->cluster_rows > 0) ok = h->ops->cluster_ok(h, h->cluster_rows);
        else
            for (int r : {8, 4, 2}) ok = ok || h->ops->cluster_ok(h, r);
        if (!ok)
            return fail(h, LBM_ERR_UNSUPPORTED,
                        "the cluster step needs a 3D lattice, a ping-pong store, nx a multiple of 32 and at most "
                        "256, ny a multiple of the cluster rows, 2 nx a multiple of 32 x rows, Q * sites < 2^32 "
                        "and no BF16 storage");
        h->variant = 5;
        h->cluster_zchunk = zchunk;
        return LBM_OK;
    }
    if (variant == 4 && !h->ops->persist_ok(h))
        return fail(h, LBM_ERR_UNSUPPORTED, "the persistent step needs FP32 arithmetic and Q * sites < 2^32");
    if (variant == 2 && !h->ops->has_v2())
        return fail(h, LBM_ERR_UNSUPPORTED, "pipelined kernel needs a 3D lattice with FP32 populations");
    if (h->inplace && (variant == 1 || variant == 2))
        return fail(h, LBM_ERR_UNSUPPORTED, "an in-place store streams with the split form only");
    if (h->consts.coupling && variant != 0 && variant != 3)
        return fail(h, LBM_ERR_UNSUPPORTED, "coupling_unew = 1 steps in the split form only");
    h->variant = variant;
    if (h->D == 3) h->zchunk = zchunk > 0 ? (zchunk < h->nz ? zchunk : h->nz) : h->zchunk_auto;
    return LBM_OK;
}

int lbm_set_cluster(lbm_handle h, int rows, int staged)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (rows != 0 && rows != 2 && rows != 4 && rows != 8 && rows != 16)
        return fail(h, LBM_ERR_INVALID_ARG, "rows in {0, 2, 4, 8, 16}");
    if (staged < -1 || staged > 1) return fail(h, LBM_ERR_INVALID_ARG, "staged in {-1, 0, 1}");
    if (rows != 0 && !h->ops->cluster_ok(h, rows))
        return fail(h, LBM_ERR_UNSUPPORTED, "the cluster step cannot use clusters of that many rows here");
    h->cluster_rows = rows;
    h->cluster_stage = staged == 1 ? 1 : 0;
    return LBM_OK;
}

int lbm_debug_stall(lbm_handle h, int plane)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (plane >= h->nz) return fail(h, LBM_ERR_INVALID_ARG, "plane >= nz");
    h->persist_stall = plane < 0 ? -1 : plane;
    return LBM_OK;
}

int lbm_footprint(lbm_handle h, size_t *device_bytes, size_t *step_bytes)
{
    if (!h) return LBM_ERR_INVALID_ARG;
    if (device_bytes) *device_bytes = footprint_bytes(h->Q, h->D, h->N, h->nz, h->storage, h->inplace, h->mask != nullptr);
    if (step_bytes) *step_bytes = 2 * (2 * h->pop_bytes) + 2 * (size_t)(1 + h->D) * h->field_bytes;
    return LBM_OK;
}

int lbm_estimate_footprint(const lbm_grid *grid, int lattice, const lbm_params *params, size_t *device_bytes)
{
    if (!grid || !params || !device_bytes || params->struct_size != sizeof(lbm_params)) return LBM_ERR_INVALID_ARG;
    int D = 0, Q = 0;
    if (lattice_dims(lattice, &D, &Q) != 0 || storage_bytes(params->storage) == 0) return LBM_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || (D == 2 && grid->nz != 1)) return LBM_ERR_INVALID_ARG;
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 31) - 1) return LBM_ERR_INVALID_ARG;
    bool mask = !grid->periodic[0] || !grid->periodic[1] || (D == 3 && !grid->periodic[2]);
    if (grid->solid)
        for (long long i = 0; i < N && !mask; ++i) mask = grid->solid[i] != 0;
    *device_bytes = footprint_bytes(Q, D, N, grid->nz, params->storage, params->inplace == 1, mask);
    return LBM_OK;
}

const char *lbm_last_error(lbm_handle h)
{
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

}  // extern "C"
