// Template implementation of the per-(lattice, storage) operations; included
// by one instantiation unit per precision.
#pragma once

#include <algorithm>
#include <cstring>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_step_v2.cuh"
#include "lbm_split.cuh"
#include "lbm_batch.cuh"
#include "lbm_persist.cuh"
#include "lbm_cluster.cuh"

#include <type_traits>

namespace lbm {

template <class R>
inline SiteConsts<R> site_consts(const HostConsts &h)
{
    SiteConsts<R> k;
    k.rho_a = R(h.rho_a); k.drho = R(h.drho); k.om1 = R(h.om1); k.rhoref_T = R(h.rhoref_T);
    k.cP = R(h.cP); k.tau_a = R(h.tau_a); k.dtau = R(h.dtau); k.inv_tau_phi = R(h.inv_tau_phi);
    k.lambda_b = R(h.lambda_b); k.M3 = R(h.M3); k.W = R(h.W); k.eps = R(h.eps);
    k.phi_n = R(h.phi_n); k.phi_m = R(h.phi_m); k.D = R(h.D); k.dt_pref = R(h.dt_pref);
    k.invW = R(1.0 / h.W); k.invD = R(1.0 / h.D);
    k.A_mu = R(h.A_mu); k.B_mu = R(h.B_mu);
    k.g[0] = R(h.g[0]); k.g[1] = R(h.g[1]); k.g[2] = R(h.g[2]);
    k.clamp = h.clamp; k.full_trace = h.full_trace; k.coupling = h.coupling;
    return k;
}

template <class L, class R, class C>
struct Impl {
    using S = typename C::S;

    static size_t step_smem() { return step_smem_bytes<L, R>(); }

    static constexpr bool kV2 = (L::D == 3) && sizeof(S) == 4 && std::is_same<R, float>::value;
    static bool has_v2() { return kV2; }

    template <bool M>
    static int launch_step_v2(lbm_ctx *c, const StepArgs<R, S> &a)
    {
        if constexpr (kV2) {
            using Tl = TileV2<L>;
            const size_t smem = step_v2_smem_bytes<L, R, S>();
            static bool attr_set = false;
            if (!attr_set) {
                cudaError_t e = cudaFuncSetAttribute(step_kernel_v2<L, R, C, M>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return cuda_fail(c, e, "cudaFuncSetAttribute(step v2)");
                attr_set = true;
            }
            dim3 block(Tl::SX, Tl::SY, 1);
            dim3 grid((c->nx + Tl::TX - 1) / Tl::TX, (c->ny + Tl::TY - 1) / Tl::TY,
                      (c->nz + c->zchunk - 1) / c->zchunk);
            step_kernel_v2<L, R, C, M><<<grid, block, smem, c->stream>>>(a);
            return cuda_fail(c, cudaGetLastError(), "step_kernel_v2 launch");
        } else {
            (void)a;
            c->err = "pipelined step kernel not available for this lattice/storage";
            return LBM_ERR_UNSUPPORTED;
        }
    }

    template <bool M>
    static int launch_step(lbm_ctx *c, const StepArgs<R, S> &a)
    {
        using Tl = Tile<L>;
        const size_t smem = step_smem_bytes<L, R>();
        static bool attr_set = false;
        if (!attr_set) {
            cudaError_t e = cudaFuncSetAttribute(step_kernel<L, R, C, M>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaFuncSetAttribute(step)");
            attr_set = true;
        }
        dim3 block(Tl::SX, Tl::SY, 1);
        dim3 grid((c->nx + Tl::TX - 1) / Tl::TX, (c->ny + Tl::TY - 1) / Tl::TY,
                  (L::D == 3) ? (c->nz + c->zchunk - 1) / c->zchunk : 1);
        step_kernel<L, R, C, M><<<grid, block, smem, c->stream>>>(a);
        return cuda_fail(c, cudaGetLastError(), "step_kernel launch");
    }

    template <int MODE, class IX>
    static void launch_split_ix(lbm_ctx *c, const SplitArgs<R, S> &a)
    {
        const unsigned blocks = (unsigned)((c->N + kSplitThreads - 1) / kSplitThreads);
        // with the u^{n+1} coupling, the omega-term of P^{n+1} between the two
        if (c->has_mask) {
            moments_kernel<L, R, C, true, MODE, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
            if (c->consts.coupling) coupling_kernel<L, R, C, true, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
            collide_kernel<L, R, C, true, MODE, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
        } else {
            moments_kernel<L, R, C, false, MODE, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
            if (c->consts.coupling) coupling_kernel<L, R, C, false, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
            collide_kernel<L, R, C, false, MODE, IX><<<blocks, kSplitThreads, 0, c->stream>>>(a);
        }
    }

    template <int MODE>
    static int launch_split(lbm_ctx *c, const SplitArgs<R, S> &a)
    {
        if (split_idx32(L::Q, c->N)) launch_split_ix<MODE, uint32_t>(c, a);
        else launch_split_ix<MODE, long long>(c, a);
        return cuda_fail(c, cudaGetLastError(), "split step launch");
    }

    // Arguments of the split step taken with the ping-pong index cur ^ flip.
    static SplitArgs<R, S> split_args(const lbm_ctx *c, int flip)
    {
        SplitArgs<R, S> a;
        a.mask = c->mask;
        a.err = c->d_err;
        a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
        a.N = c->N;
        // one thread a site from site 0 (split launches, batch items of whole
        // 128-site blocks): whole warps when N is a multiple of 32
        a.vote = (c->N & 31) == 0;
        a.k = site_consts<R>(c->consts);
        a.phi = static_cast<R *>(c->phi);
        const int src = c->cur ^ flip, dst = 1 - src;
        a.seed = (unsigned)(c->steps + flip);
        a.F_old = static_cast<const float4 *>(c->fa[src]);
        a.F_new = static_cast<float4 *>(c->fa[dst]);
        a.FB = static_cast<float4 *>(c->fb);
        a.PiG = static_cast<float *>(c->pig);
        a.G_old = static_cast<const float4 *>(c->fg[src]);
        a.G_new = static_cast<float4 *>(c->fg[dst]);
        a.src_h = static_cast<const S *>(c->h[src]);
        a.src_g = static_cast<const S *>(c->g[src]);
        a.dst_h = static_cast<S *>(c->h[dst]);
        a.dst_g = static_cast<S *>(c->g[dst]);
        a.P_old = static_cast<const R *>(c->P[src]);
        a.P_new = static_cast<R *>(c->P[dst]);
        a.u_old = static_cast<const R *>(c->u[src]);
        a.u_new = static_cast<R *>(c->u[dst]);
        return a;
    }

    // Stream mode of the step that follows `steps` completed steps.
    static int split_mode(const lbm_ctx *c, int64_t steps)
    {
        if (!c->inplace) return kPingPong;
        return steps % 2 == 0 ? kAAOdd : kAAEven;
    }

    // Packed (u, P) words of the current state, when they are stale.
    static int pack(lbm_ctx *c)
    {
        if constexpr (kPacked<R>) {
            if (c->fa_valid || !c->fa[c->cur]) return LBM_OK;
            const unsigned blocks = (unsigned)((c->N + 255) / 256);
            pack_kernel<L::D><<<blocks, 256, 0, c->stream>>>(static_cast<const float *>(c->P[c->cur]),
                                                             static_cast<const float *>(c->u[c->cur]),
                                                             static_cast<float4 *>(c->fa[c->cur]), c->N);
            const int rc = cuda_fail(c, cudaGetLastError(), "pack_kernel launch");
            if (rc == LBM_OK) c->fa_valid = true;
            return rc;
        } else {
            return LBM_OK;
        }
    }

    // Before split steps: packed (u, P) words; with BF16 storage V_g = 0
    // when the store holds complete g* (the first pull adds nothing).
    static int split_prepare(lbm_ctx *c)
    {
        int rc = pack(c);
        if constexpr (kPacked<R> && C::kGodd) {
            if (rc == LBM_OK && !c->g_deferred && c->fg[c->cur])
                rc = cuda_fail(c, cudaMemsetAsync(c->fg[c->cur], 0, 16 * (size_t)c->N, c->stream),
                               "cudaMemsetAsync(V_g)");
        }
        return rc;
    }

    // Complete g* in the store (BF16 storage, odd part deferred).
    static int fold(lbm_ctx *c)
    {
        if constexpr (kPacked<R> && C::kGodd) {
            if (!c->g_deferred) return LBM_OK;
            const unsigned blocks = (unsigned)((c->N + 127) / 128);
            fold_g_kernel<L, C><<<blocks, 128, 0, c->stream>>>(read_args(c), static_cast<S *>(c->g[c->cur]),
                                                              static_cast<const float4 *>(c->fg[c->cur]));
            const int rc = cuda_fail(c, cudaGetLastError(), "fold_g_kernel launch");
            if (rc == LBM_OK) c->g_deferred = false;
            return rc;
        } else {
            return LBM_OK;
        }
    }

    // The planes P[cur], u[cur] from the packed words, when they are stale.
    static int sync_soa(lbm_ctx *c)
    {
        if constexpr (kPacked<R>) {
            if (c->soa_valid) return LBM_OK;
            const unsigned blocks = (unsigned)((c->N + 255) / 256);
            unpack_kernel<L::D><<<blocks, 256, 0, c->stream>>>(static_cast<const float4 *>(c->fa[c->cur]), c->mask,
                                                               static_cast<float *>(c->P[c->cur]),
                                                               static_cast<float *>(c->u[c->cur]), c->N);
            const int rc = cuda_fail(c, cudaGetLastError(), "unpack_kernel launch");
            if (rc == LBM_OK) c->soa_valid = true;
            return rc;
        } else {
            return LBM_OK;
        }
    }

    static int step_split(lbm_ctx *c, int64_t n)
    {
        if (n > 0) {
            const int rc = split_prepare(c);
            if (rc != LBM_OK) return rc;
        }
        for (int64_t s = 0; s < n; ++s) {
            const SplitArgs<R, S> a = split_args(c, 0);
            int rc;
            const int mode = split_mode(c, c->steps);
            if (mode == kPingPong) rc = launch_split<kPingPong>(c, a);
            else if (mode == kAAOdd) rc = launch_split<kAAOdd>(c, a);
            else rc = launch_split<kAAEven>(c, a);
            if (rc != LBM_OK) return rc;
            c->cur = 1 - c->cur;
            c->steps += 1;
            if constexpr (kPacked<R>) {
                c->soa_valid = false;                      // the state is in fa[cur]
                if constexpr (C::kGodd) c->g_deferred = true;   // fg[cur] holds V_g
            }
        }
        return LBM_OK;
    }

    // --- batched persistent launch (lbm_batch_*) ---------------------------
    static size_t batch_member_bytes() { return sizeof(BatchMember<R, S>); }

    // Work items of a member: `span` consecutive blocks of kSplitThreads sites.
    static long long batch_items(const lbm_ctx *c, int span)
    {
        const long long per = (long long)kSplitThreads * span;
        return (c->N + per - 1) / per;
    }

    static void batch_fill(const lbm_ctx *c, int take, long long first_item, void *dst)
    {
        BatchMember<R, S> m;
        std::memset(&m, 0, sizeof m);
        m.a[0] = split_args(c, 0);
        m.a[1] = split_args(c, 1);
        m.mode[0] = split_mode(c, c->steps);
        m.mode[1] = split_mode(c, c->steps + 1);
        m.first_item = first_item;
        m.items = batch_items(c, 1);
        m.take = take;
        m.has_mask = c->has_mask ? 1 : 0;
        std::memcpy(dst, &m, sizeof m);
    }

    // Persistent grid of a batch launch: blocks_per_sm per SM (0: as many as
    // fit, the kernel's occupancy), never more than fit.
    static int batch_grid(int phase, int blocks_per_sm)
    {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (phase == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<L, R, C, 0>, kSplitThreads, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<L, R, C, 1>, kSplitThreads, 0);
        if (per_sm < 1) per_sm = 1;
        if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
        return per_sm * (sms > 0 ? sms : 1);
    }

    static cudaError_t batch_launch(cudaStream_t s, const void *d_table, int K, int grid0, int grid1, bool coupled,
                                    bool pp)
    {
        const BatchHeader *hdr = static_cast<const BatchHeader *>(d_table);
        const BatchMember<R, S> *mem = reinterpret_cast<const BatchMember<R, S> *>(
            static_cast<const char *>(d_table) + batch_header_bytes());
        // pp: every member uses the ping-pong store (kernels with that mode only);
        // the grids sized for the general kernels fit these as well
        for (int k = 0; k < K; ++k) {
            if (pp) batch_kernel<L, R, C, 0, true><<<grid0, kSplitThreads, 0, s>>>(hdr, mem, k);
            else batch_kernel<L, R, C, 0><<<grid0, kSplitThreads, 0, s>>>(hdr, mem, k);
            if (coupled) batch_kernel<L, R, C, 2><<<grid1, kSplitThreads, 0, s>>>(hdr, mem, k);
            if (pp) batch_kernel<L, R, C, 1, true><<<grid1, kSplitThreads, 0, s>>>(hdr, mem, k);
            else batch_kernel<L, R, C, 1><<<grid1, kSplitThreads, 0, s>>>(hdr, mem, k);
        }
        return cudaGetLastError();
    }

    // --- persistent split step (one launch per step) ------------------------
    static bool persist_ok(const lbm_ctx *c)
    {
        return kPacked<R> && c->pctl != nullptr && split_idx32(L::Q, c->N);
    }

    template <bool M, int MODE>
    static int launch_persist(lbm_ctx *c, const SplitArgs<R, S> &a)
    {
        if constexpr (kPacked<R>) {
            static int grid = 0;
            if (grid == 0) {
                int sms = 0, per_sm = 0;
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, split_persistent_kernel<L, C, M, MODE>,
                                                              kSplitThreads, 0);
                grid = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
            }
            PersistArgs p;
            p.ctl = c->pctl;
            p.nz = L::D == 3 ? c->nz : 1;
            p.nxy = (int)(c->N / p.nz);
            p.bpp = (p.nxy + kSplitThreads * kPersistSpan - 1) / (kSplitThreads * kPersistSpan);
            p.zper = L::D == 3 ? c->periodic[2] : 1;
            p.lag = kPersistLag;
            p.stall = c->persist_stall;
            p.err = c->d_err;
            const long long items = 2LL * p.nz * p.bpp;
            const int g = (int)std::min<long long>(grid, items);
            int rc = cuda_fail(c, cudaMemsetAsync(c->pctl, 0, sizeof(int) * (2 + (size_t)p.nz), c->stream),
                               "cudaMemsetAsync(persistent counters)");
            if (rc != LBM_OK) return rc;
            SplitArgs<R, S> ap = a;
            ap.vote = (p.nxy & 31) == 0;   // items are blocks of one plane
            split_persistent_kernel<L, C, M, MODE><<<g, kSplitThreads, 0, c->stream>>>(ap, p);
            return cuda_fail(c, cudaGetLastError(), "split_persistent_kernel launch");
        } else {
            return LBM_ERR_UNSUPPORTED;
        }
    }

    static int step_persist(lbm_ctx *c, int64_t n)
    {
        if (n > 0) {
            const int rc = split_prepare(c);
            if (rc != LBM_OK) return rc;
        }
        for (int64_t s = 0; s < n; ++s) {
            const SplitArgs<R, S> a = split_args(c, 0);
            const int mode = split_mode(c, c->steps);
            int rc;
            if (c->has_mask) {
                if (mode == kPingPong) rc = launch_persist<true, kPingPong>(c, a);
                else if (mode == kAAOdd) rc = launch_persist<true, kAAOdd>(c, a);
                else rc = launch_persist<true, kAAEven>(c, a);
            } else {
                if (mode == kPingPong) rc = launch_persist<false, kPingPong>(c, a);
                else if (mode == kAAOdd) rc = launch_persist<false, kAAOdd>(c, a);
                else rc = launch_persist<false, kAAEven>(c, a);
            }
            if (rc != LBM_OK) return rc;
            c->cur = 1 - c->cur;
            c->steps += 1;
            c->soa_valid = false;
            if constexpr (C::kGodd) c->g_deferred = true;
        }
        return LBM_OK;
    }

    // --- cluster step (one launch per step, variant 5) -------------------------
    static bool cluster_ok_rows(const lbm_ctx *c, int cy)
    {
        if constexpr (L::D == 3 && !C::kGodd) return cluster_ok(L::D, L::Q, c->nx, c->ny, c->N, cy, c->inplace, false);
        else return false;
    }

    // Rows per cluster: the handle's choice, else the largest of 16 (where
    // the device allows that non-portable size), 8, 4, 2 the lattice fits.
    static int cluster_rows(const lbm_ctx *c)
    {
        if (c->cluster_rows > 0) return c->cluster_rows;
        if (cluster_ok_rows(c, 16) && cluster16_allowed(c)) return 16;
        for (int r : {8, 4, 2})
            if (cluster_ok_rows(c, r)) return r;
        return 8;
    }

    static bool cluster16_allowed(const lbm_ctx *c)
    {
        if constexpr (L::D == 3 && !C::kGodd) {
            static int ok = -1;
            if (ok < 0) {
                ok = 1;
                for_each_cluster_kernel([&](auto kernel) {
                    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
                        ok = 0;
                });
                cudaGetLastError();
            }
            (void)c;
            return ok == 1;
        } else {
            (void)c;
            return false;
        }
    }

    // Every instantiation of the cluster kernel this (lattice, storage) has.
    template <class F>
    static void for_each_cluster_kernel(F &&f)
    {
        if constexpr (L::D == 3 && !C::kGodd) {
            f(cluster_step_kernel<L, R, C, true, false>);
            f(cluster_step_kernel<L, R, C, false, false>);
            if constexpr (kPacked<R>) {
                f(cluster_step_kernel<L, R, C, true, true>);
                f(cluster_step_kernel<L, R, C, false, true>);
            }
        }
    }

    // Rows staged by bulk copies: FP32 arithmetic, unless the handle says no.
    static bool cluster_staged(const lbm_ctx *c) { return kPacked<R> && c->cluster_stage != 0; }

    static bool cluster_ok_h(const lbm_ctx *c) { return cluster_ok_rows(c, cluster_rows(c)); }

    // Planes per CTA: the handle's zchunk when set, else about six waves of
    // CTAs (two resident per SM).
    static int cluster_zchunk(const lbm_ctx *c)
    {
        if (c->cluster_zchunk > 0) return c->cluster_zchunk < c->nz ? c->cluster_zchunk : c->nz;
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const long long want = 6LL * 2 * sms;
        long long chunks = (want + c->ny - 1) / c->ny;
        if (chunks < 1) chunks = 1;
        long long zc = (c->nz + chunks - 1) / chunks;
        if (zc < 8) zc = 8;
        if (zc > c->nz) zc = c->nz;
        return (int)zc;
    }

    template <bool M, bool STAGE>
    static int launch_cluster(lbm_ctx *c, const SplitArgs<R, S> &a)
    {
        if constexpr (L::D == 3 && !C::kGodd && (!STAGE || kPacked<R>)) {
            const int cy = cluster_rows(c);
            const size_t smem = cluster_smem_bytes<R, S>(c->nx, L::Q, STAGE);
            static bool attr_set = false;
            if (!attr_set) {
                // the largest any lattice needs (nx = 256), set once
                cudaError_t e = cudaFuncSetAttribute(
                    cluster_step_kernel<L, R, C, M, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                    (int)cluster_smem_bytes<R, S>(kClusterMaxThreads, L::Q, STAGE));
                if (e != cudaSuccess) return cuda_fail(c, e, "cudaFuncSetAttribute(cluster step)");
                attr_set = true;
            }
            if (cy > 8) cluster16_allowed(c);
            ClusterArgs g;
            g.zchunk = cluster_zchunk(c);
            g.cy = cy;
            g.zper = c->periodic[2];
            g.yper = c->periodic[1];
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(1, (unsigned)c->ny, (unsigned)((c->nz + g.zchunk - 1) / g.zchunk));
            cfg.blockDim = dim3((unsigned)c->nx, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = c->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 1;
            attr[0].val.clusterDim.y = (unsigned)cy;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            return cuda_fail(c, cudaLaunchKernelEx(&cfg, cluster_step_kernel<L, R, C, M, STAGE>, a, g),
                             "cluster_step_kernel launch");
        } else {
            (void)a;
            c->err = "cluster step not available for this lattice/storage";
            return LBM_ERR_UNSUPPORTED;
        }
    }

    static int step_cluster(lbm_ctx *c, int64_t n)
    {
        if (n > 0) {
            const int rc = split_prepare(c);
            if (rc != LBM_OK) return rc;
        }
        for (int64_t s = 0; s < n; ++s) {
            const SplitArgs<R, S> a = split_args(c, 0);
            const bool st = cluster_staged(c);
            const int rc = c->has_mask ? (st ? launch_cluster<true, true>(c, a) : launch_cluster<true, false>(c, a))
                                       : (st ? launch_cluster<false, true>(c, a) : launch_cluster<false, false>(c, a));
            if (rc != LBM_OK) return rc;
            c->cur = 1 - c->cur;
            c->steps += 1;
            if constexpr (kPacked<R>) c->soa_valid = false;
        }
        return LBM_OK;
    }

    static int step(lbm_ctx *c, int64_t n)
    {
        if (c->variant == 5 && cluster_ok_h(c)) return step_cluster(c, n);
        if (c->variant == 4 && persist_ok(c)) return step_persist(c, n);
        if (c->inplace || c->variant == 3 || c->variant == 0 || c->variant == 4 || c->variant == 5)
            return step_split(c, n);
        if (n > 0) {
            int rc = sync_soa(c);
            if (rc == LBM_OK) rc = fold(c);
            if (rc != LBM_OK) return rc;
        }
        StepArgs<R, S> a;
        a.mask = c->mask;
        a.err = c->d_err;
        a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
        a.per_x = c->periodic[0]; a.per_y = c->periodic[1]; a.per_z = c->periodic[2];
        a.zchunk = c->zchunk;
        a.N = c->N;
        a.k = site_consts<R>(c->consts);
        for (int64_t s = 0; s < n; ++s) {
            const int src = c->cur, dst = 1 - c->cur;
            a.src_h = static_cast<const S *>(c->h[src]);
            a.src_g = static_cast<const S *>(c->g[src]);
            a.dst_h = static_cast<S *>(c->h[dst]);
            a.dst_g = static_cast<S *>(c->g[dst]);
            a.P_old = static_cast<const R *>(c->P[src]);
            a.P_new = static_cast<R *>(c->P[dst]);
            a.u_old = static_cast<const R *>(c->u[src]);
            a.u_new = static_cast<R *>(c->u[dst]);
            const bool v2 = kV2 && c->variant != 1;
            const int rc = v2 ? (c->has_mask ? launch_step_v2<true>(c, a) : launch_step_v2<false>(c, a))
                              : (c->has_mask ? launch_step<true>(c, a) : launch_step<false>(c, a));
            if (rc != LBM_OK) return rc;
            c->cur = dst;
            c->steps += 1;
            c->fa_valid = false;   // the fused kernels keep the state in P, u only
        }
        return LBM_OK;
    }

    static int init(lbm_ctx *c, const double *d_phi, const double *d_P, const double *d_u)
    {
        InitArgs<R, S> a;
        a.phi0 = d_phi; a.P0 = d_P; a.u0 = d_u;
        a.h = static_cast<S *>(c->h[0]);
        a.g = static_cast<S *>(c->g[0]);
        a.P = static_cast<R *>(c->P[0]);
        a.u = static_cast<R *>(c->u[0]);
        a.mask = c->mask;
        a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
        a.N = c->N;
        a.aa = c->inplace ? 1 : 0;
        a.k = site_consts<R>(c->consts);
        const int threads = 128;
        const unsigned blocks = (unsigned)((c->N + threads - 1) / threads);
        if (c->has_mask) init_kernel<L, R, C, true><<<blocks, threads, 0, c->stream>>>(a);
        else init_kernel<L, R, C, false><<<blocks, threads, 0, c->stream>>>(a);
        c->cur = 0;
        c->steps = 0;
        c->fa_valid = false;
        c->soa_valid = true;
        c->g_deferred = false;
        return cuda_fail(c, cudaGetLastError(), "init_kernel launch");
    }

    static ReadArgs<R, S> read_args(lbm_ctx *c)
    {
        ReadArgs<R, S> a;
        a.h = static_cast<const S *>(c->h[c->cur]);
        a.g = static_cast<const S *>(c->g[c->cur]);
        a.P = static_cast<const R *>(c->P[c->cur]);
        a.u = static_cast<const R *>(c->u[c->cur]);
        a.mask = c->mask;
        a.phi_out = a.P_out = a.u_out = a.hpop_out = a.gpop_out = nullptr;
        a.N = c->N;
        a.cP = R(c->consts.cP);
        a.aa = c->inplace ? 1 + (int)(c->steps % 2) : 0;
        a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
        a.G = nullptr;
        if constexpr (kPacked<R> && C::kGodd)
            if (c->g_deferred) a.G = static_cast<const float4 *>(c->fg[c->cur]);
        return a;
    }

    static int read(lbm_ctx *c, double *d_phi, double *d_P, double *d_u, double *d_hpop, double *d_gpop)
    {
        if (const int rs = sync_soa(c); rs != LBM_OK) return rs;
        ReadArgs<R, S> a = read_args(c);
        a.phi_out = d_phi; a.P_out = d_P; a.u_out = d_u; a.hpop_out = d_hpop; a.gpop_out = d_gpop;
        const int threads = 256;
        const unsigned blocks = (unsigned)((c->N + threads - 1) / threads);
        if (c->has_mask) read_kernel<L, R, C, true><<<blocks, threads, 0, c->stream>>>(a);
        else read_kernel<L, R, C, false><<<blocks, threads, 0, c->stream>>>(a);
        return cuda_fail(c, cudaGetLastError(), "read_kernel launch");
    }

    static int reduce(lbm_ctx *c, double *d_out5)
    {
        if (const int rs = sync_soa(c); rs != LBM_OK) return rs;
        ReadArgs<R, S> a = read_args(c);
        const int blocks = (int)std::min<long long>(kRedMaxBlocks, (c->N + kRedThreads - 1) / kRedThreads);
        double *partials = c->d_scratch;
        if (c->has_mask)
            reduce_kernel<L, R, C, true><<<blocks, kRedThreads, 0, c->stream>>>(
                a, R(c->consts.rho_a), R(c->consts.drho), c->consts.clamp, partials);
        else
            reduce_kernel<L, R, C, false><<<blocks, kRedThreads, 0, c->stream>>>(
                a, R(c->consts.rho_a), R(c->consts.drho), c->consts.clamp, partials);
        finish_kernel<kRedVals><<<1, kRedThreads, 0, c->stream>>>(partials, blocks, d_out5);
        return cuda_fail(c, cudaGetLastError(), "reduce launch");
    }

    static int pjump(lbm_ctx *c, const double center[3], double r_in, double r_out, double *d_out4)
    {
        if (const int rs = sync_soa(c); rs != LBM_OK) return rs;
        const int blocks = (int)std::min<long long>(kRedMaxBlocks, (c->N + kRedThreads - 1) / kRedThreads);
        double *partials = c->d_scratch;
        const R *P = static_cast<const R *>(c->P[c->cur]);
        if (c->has_mask)
            pjump_kernel<R, true><<<blocks, kRedThreads, 0, c->stream>>>(
                P, c->mask, c->nx, c->ny, c->nz, c->N, center[0], center[1], center[2], r_in, r_out, partials);
        else
            pjump_kernel<R, false><<<blocks, kRedThreads, 0, c->stream>>>(
                P, c->mask, c->nx, c->ny, c->nz, c->N, center[0], center[1], center[2], r_in, r_out, partials);
        finish_kernel<4><<<1, kRedThreads, 0, c->stream>>>(partials, blocks, d_out4);
        return cuda_fail(c, cudaGetLastError(), "pjump launch");
    }

    static int probe(lbm_ctx *c, const long long *d_sites, int n, double *d_h, double *d_g, double *d_P, double *d_u)
    {
        if (const int rs = sync_soa(c); rs != LBM_OK) return rs;
        ReadArgs<R, S> a = read_args(c);
        const int threads = 128;
        probe_kernel<L, R, C><<<(n + threads - 1) / threads, threads, 0, c->stream>>>(a, d_sites, n, d_h, d_g, d_P, d_u);
        return cuda_fail(c, cudaGetLastError(), "probe_kernel launch");
    }

    static const Ops *ops()
    {
        static const Ops o = {&init,      &step,       &read,         &reduce,      &pjump,
                              &probe,     &step_smem,  &has_v2,       &pack,        &sync_soa,
                              &persist_ok, &split_prepare, &fold, &batch_member_bytes,
                              &batch_items, &batch_fill, &batch_grid, &batch_launch, &cluster_ok_rows};
        return &o;
    }
};

}  // namespace lbm
