// One-launch step on thread-block clusters (variant 5).
//
// The split form hands the moments of a step (phi, u, P and the second
// moments of the pulled g) from one launch to the next through HBM and pulls
// h twice.  Here a CTA owns one row of sites (x = 0 .. nx-1 at fixed y) and
// marches in z through a chunk of planes; a cluster of CY CTAs covers CY
// consecutive rows.  For each plane q a CTA
//   - computes the moments of its own row (S0, S1) into a four-plane ring of
//     (u, phi) words in its shared memory, and keeps P^{n+1} and the second
//     moments of the pulled g for its own threads;
//   - after a cluster barrier, collides the plane q-1 (S2..S5): the stencils
//     read the (u, phi) words of planes q-2 .. q, of its own row from its own
//     ring and of the rows y-1, y+1 from the rings of the neighbouring CTAs of
//     the cluster (distributed shared memory).
// The rows just outside the cluster (y0 - 1 and y0 + CY) have no owner in it:
// their moments are recomputed, spread evenly over the CTAs of the cluster
// (2 nx / CY sites each per plane, whole warps, rotating over the warps), and
// stored into the halo ring of the first and the last CTA.  The first chunk
// plane and the one after the chunk are recomputed the same way by the
// chunks on either side.  So a step moves each population through HBM once
// (plus the halo rows and planes), and P, u once.
//
// Staged form (STAGE, FP32 arithmetic): the rows a plane's moments pull, one
// row of nx populations per direction and population set (the row of
// x - c_i at y - c_iy, z - c_iz, read whole so that the shift in x is an
// index in shared memory), arrive by bulk asynchronous copies (cp.async.bulk,
// the tensor memory accelerator) into shared memory two planes ahead, with
// completion counted on an mbarrier per buffer.  The copies of plane q+2
// stream while the CTA collides plane q, so the moments read shared memory
// and the collision takes the pulled h from the same buffer instead of a
// second read.  Buffers: h three planes deep (moments q+1, collision q, copy
// q+2), g two.  A site whose source is solid or outside (a mask bit) takes
// its bounce-back value from the population store as in the split form.
// The halo rows' moments read the store directly.
//
// Ring slots are used modulo 4: a CTA writes plane q+1 while the slowest CTA
// of its cluster may still read planes q-2 .. q (one barrier per plane), so
// four slots never overlap.  The barrier (barrier.cluster arrive.release /
// wait.acquire) orders the shared-memory writes of every CTA of the cluster
// before the reads of the next collision, and the reads of a copy buffer
// before the copy that refills it; a final barrier keeps every CTA's shared
// memory alive until the last remote read.  Every copy issued is waited
// for; a wait gives up after 1 s of the GPU's timer, sets the timeout bit
// and waits once more (bounded) before the CTA goes on without computing.
//
// Per-site arithmetic is that of the split form (moments_site_f32 /
// moments_site_canon, stencil_packed / the canonical stencils,
// collide_pairs / collide), so an FP64 lattice steps bit for bit like the
// split form and the oracle; with FP32 arithmetic the compiler may contract
// products and sums differently, so the forms agree to rounding.
//
// Requirements (else LBM_ERR_UNSUPPORTED): a 3D lattice, ping-pong store, nx
// a multiple of 32 and at most 256, ny a multiple of CY, 2 nx a multiple of
// 32 CY, Q N < 2^32, no BF16 odd-part deferral.
#pragma once

#include <cooperative_groups.h>

#include "lbm_split.cuh"
#include "lbm_persist.cuh"

namespace lbm {

namespace cg = cooperative_groups;

constexpr int kClusterRing = 4;       // plane slots of the (u, phi) ring
constexpr int kClusterMaxThreads = 256;

// (u_x, u_y, u_z, phi) of one site in the ring.
struct alignas(16) Dbl4 {
    double x, y, z, w;
};
template <class R>
struct RingWord {
    using T = float4;
};
template <>
struct RingWord<double> {
    using T = Dbl4;
};

struct ClusterArgs {
    int zchunk;   // planes per CTA
    int cy;       // CTAs (rows) per cluster
    int zper;     // periodic in z
    int yper;     // periodic in y
};

// Second moments kept per thread between the moments and the collision of a
// plane (FP32 arithmetic only).
template <class R>
inline constexpr int kClusterNS = std::is_same<R, float>::value ? 6 : 0;

constexpr int kStageH = 3, kStageG = 2;   // copy buffers of h and g (planes)

// Dynamic shared memory of one CTA: (staged) h rows [3][Q][nx] and g rows
// [2][Q][nx] in storage format, own ring [4][nx], halo ring [4][nx],
// P^{n+1} [2][nx], second moments [2][NS][nx], (staged) three mbarriers.
template <class R, class S>
__host__ __device__ constexpr size_t cluster_smem_bytes(int nx, int Q, bool stage)
{
    return (stage ? sizeof(S) * (size_t)(kStageH + kStageG) * Q * nx : 0) +
           sizeof(typename RingWord<R>::T) * 2 * kClusterRing * (size_t)nx + sizeof(R) * 2 * (size_t)nx +
           sizeof(float) * 2 * kClusterNS<R> * (size_t)nx + (stage ? 8 * kStageH : 0);
}

// --- mbarrier and bulk copy (shared::cta addresses) -----------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// One arrival that also announces `bytes` of copies completing on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Prefetch of `bytes` (a multiple of 16, 16-byte aligned) from global memory
// into L2 by the bulk copy engine; no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `bar` with the given parity, at most 1 s of the
// GPU's timer (and a poll count as backstop).  False when it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < kPersistMaxSpin; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (global_ns() - t0 > kPersistWaitNs) break;
    }
    return false;
}

// Pulled populations of the own row from the staged rows: slot i of the
// site x comes from element x - c_ix (wrapped) of the row staged for i; a
// solid or outside source reads the site's own post-collision -i from the
// store (halfway bounce-back, as read_idx in the ping-pong mode).
template <class L, bool HAS_MASK, class S>
struct StagedPull {
    const S *h, *g;     // population store (bounce-back)
    const S *sh, *sg;   // staged rows [Q][nx]
    int x, nx;
    template <int i>
    __device__ __forceinline__ void get(uint32_t N, const Nbr32 &, int idx, uint32_t m, S &hr, S &gr) const
    {
        if constexpr (i != 0 && HAS_MASK) {
            if ((m >> i) & 1u) {
                const uint32_t e = (uint32_t)opp(i) * N + (uint32_t)idx;
                hr = h[e];
                gr = g[e];
                return;
            }
        }
        constexpr int cx = L::c(i, 0);
        int xs = x - cx;
        if constexpr (cx > 0) xs = xs < 0 ? xs + nx : xs;
        if constexpr (cx < 0) xs = xs >= nx ? xs - nx : xs;
        hr = sh[i * nx + xs];
        gr = sg[i * nx + xs];
    }
};

// c_ia of direction i (a runtime index) from the lattice's constexpr table.
template <class L>
__device__ __forceinline__ int lattice_c(int i, int a)
{
    int v = 0;
    static_for<0, L::Q>([&](auto I) {
        constexpr int k = decltype(I)::value;
        if (k == i) v = a == 0 ? L::c(k, 0) : (a == 1 ? L::c(k, 1) : L::c(k, 2));
    });
    return v;
}

template <class L, class R, class C, bool HAS_MASK, bool STAGE>
__global__ void __launch_bounds__(kClusterMaxThreads, STAGE ? 1 : 2)
    cluster_step_kernel(const SplitArgs<R, typename C::S> a, const ClusterArgs g)
{
    using V4 = typename RingWord<R>::T;
    using S = typename C::S;
    static_assert(L::D == 3, "cluster step: 3D lattices");
    static_assert(!STAGE || kPacked<R>, "staged cluster step: FP32 arithmetic");
    constexpr int Q = L::Q;
    constexpr int NS = kClusterNS<R>;
    cg::cluster_group cl = cg::this_cluster();
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const uint32_t N = (uint32_t)a.N;
    const int CY = g.cy;
    const int rank = (int)cl.block_index().y;
    const int x = (int)threadIdx.x;
    const int y = (int)blockIdx.y;
    const int y0 = y - rank;                          // first row of the cluster
    const int zb = (int)blockIdx.z * g.zchunk;
    const int ze = min(nz, zb + g.zchunk);
    const int warp = x >> 5, lane = x & 31;
    const int nw = nx >> 5;
    const int HS = 2 * nx / CY;                       // halo sites recomputed per CTA and plane
    const int hw = HS >> 5;                           // ... in whole warps

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sp = smem_raw;
    S *hbuf = reinterpret_cast<S *>(sp);                             // [3][Q][nx] (staged)
    S *gbuf = hbuf + (STAGE ? kStageH * Q * nx : 0);                 // [2][Q][nx] (staged)
    sp = reinterpret_cast<unsigned char *>(gbuf + (STAGE ? kStageG * Q * nx : 0));
    V4 *ring = reinterpret_cast<V4 *>(sp);                           // [4][nx]
    V4 *ringh = ring + kClusterRing * nx;                            // [4][nx]
    R *stP = reinterpret_cast<R *>(ringh + kClusterRing * nx);       // [2][nx]
    float *stM = reinterpret_cast<float *>(stP + 2 * nx);            // [2][NS][nx]
    uint64_t *bars = reinterpret_cast<uint64_t *>(stM + 2 * NS * nx);   // [3] (staged)

    if constexpr (STAGE) {
        if (x == 0)
            for (int b = 0; b < kStageH; ++b) mbar_init(bars + b, 1);
        mbar_init_fence();
    }
    // barrier initialisation visible to the copies, and every CTA of the
    // cluster started before any remote access
    cl.sync();

    // rows y - 1 and y + 1: the neighbouring CTA's ring, or this CTA's halo
    // ring at the edges of the cluster
    const V4 *row_m = rank > 0 ? cl.map_shared_rank(ring, rank - 1) : ringh;
    const V4 *row_p = rank < CY - 1 ? cl.map_shared_rank(ring, rank + 1) : ringh;
    V4 *halo_lo = cl.map_shared_rank(ringh, 0);
    V4 *halo_hi = cl.map_shared_rank(ringh, CY - 1);

    // plane q wrapped into the grid; false outside a closed axis
    auto plane_of = [&](int q, int &qw) -> bool {
        qw = q;
        if (q < 0 || q >= nz) {
            if (!g.zper) return false;
            qw = q < 0 ? q + nz : q - nz;
        }
        return true;
    };
    auto hslot = [](int q) { return ((q % kStageH) + kStageH) % kStageH; };

    // --- staged copies of the rows plane q pulls (thread 0 issues them)
    uint32_t parity = 0;      // bit b: parity of the next phase of mbarrier b
    bool failed = false;      // a copy wait ran out: compute nothing more
    auto issue = [&](int q) {
        if constexpr (STAGE) {
            int qw;
            if (x != 0 || !plane_of(q, qw)) return;
            const int hb = hslot(q), gb = q & 1;
            uint32_t rows = 0;
            int ys[Q], zs[Q];
            bool ok[Q];
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                int yy = y - L::c(i, 1), zz = qw - L::c(i, 2);
                bool v = true;
                if (yy < 0 || yy >= ny) {
                    if (g.yper) yy = yy < 0 ? yy + ny : yy - ny;
                    else v = false;
                }
                if (zz < 0 || zz >= nz) {
                    if (g.zper) zz = zz < 0 ? zz + nz : zz - nz;
                    else v = false;
                }
                ys[i] = yy;
                zs[i] = zz;
                ok[i] = v;
                rows += v ? 1u : 0u;
            });
            const uint32_t row_bytes = (uint32_t)(nx * sizeof(S));
            mbar_arrive_expect_tx(bars + hb, 2 * rows * row_bytes);
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                if (ok[i]) {
                    const uint32_t off = (uint32_t)i * N + (uint32_t)((zs[i] * ny + ys[i]) * nx);
                    bulk_copy_g2s(hbuf + (hb * Q + i) * nx, a.src_h + off, row_bytes, bars + hb);
                    bulk_copy_g2s(gbuf + (gb * Q + i) * nx, a.src_g + off, row_bytes, bars + hb);
                }
            });
        } else {
            // the store is read directly: bring the rows plane q pulls (one
            // row of each population set per direction, one thread each)
            // and its packed state words into L2 while the CTA collides
            int qw;
            if (!plane_of(q, qw) || x >= 2 * Q + 1) return;
            if (x == 2 * Q) {
                if constexpr (kPacked<R>) {
                    int zz = qw + 1;
                    if (zz >= nz) zz = g.zper ? zz - nz : -1;
                    if (zz >= 0) {
                        for (int dy = -1; dy <= 1; ++dy) {
                            int yy = y + dy;
                            if (yy < 0 || yy >= ny) {
                                if (!g.yper) continue;
                                yy = yy < 0 ? yy + ny : yy - ny;
                            }
                            bulk_prefetch_l2(a.F_old + (zz * ny + yy) * nx, (uint32_t)(nx * sizeof(float4)));
                        }
                    }
                }
                return;
            }
            const int i = x % Q;
            int yy = y - lattice_c<L>(i, 1), zz = qw - lattice_c<L>(i, 2);
            if (yy < 0 || yy >= ny) {
                if (!g.yper) return;
                yy = yy < 0 ? yy + ny : yy - ny;
            }
            if (zz < 0 || zz >= nz) {
                if (!g.zper) return;
                zz = zz < 0 ? zz + nz : zz - nz;
            }
            const uint32_t off = (uint32_t)i * N + (uint32_t)((zz * ny + yy) * nx);
            bulk_prefetch_l2((x < Q ? a.src_h : a.src_g) + off, (uint32_t)(nx * sizeof(S)));
        }
    };
    auto await = [&](int q) {
        if constexpr (STAGE) {
            int qw;
            if (!plane_of(q, qw)) return;
            const int hb = hslot(q);
            if (!mbar_wait_bounded(bars + hb, (parity >> hb) & 1u)) {
                if (!failed) atomicOr(a.err, 2);
                failed = true;
                mbar_wait_bounded(bars + hb, (parity >> hb) & 1u);
            }
            parity ^= 1u << hb;
        } else {
            (void)q;
        }
    };

    // --- S0 + S1 of plane q: own row, and this CTA's share of the halo rows
    auto moments = [&](int q) {
        int qw;
        if (!plane_of(q, qw) || failed) return;       // outside a closed axis: never read
        const bool in_chunk = q >= zb && q < ze;
        const int slot = q & (kClusterRing - 1), half = q & 1;
        {
            const int idx = (qw * ny + y) * nx + x;
            uint32_t m = 0;
            if constexpr (HAS_MASK) m = a.mask[idx];
            if constexpr (kPacked<R>) {
                auto sink = [&](float ux, float uy, float uz, float Pn, float phi, const float *pm) {
                    if (in_chunk) a.F_new[idx] = make_float4(ux, uy, uz, Pn);
                    ring[slot * nx + x] = make_float4(ux, uy, uz, phi);
                    stP[half * nx + x] = Pn;
                    static_for<0, NS>([&](auto J) {
                        constexpr int j = decltype(J)::value;
                        stM[(half * NS + j) * nx + x] = pm[j];
                    });
                };
                if constexpr (STAGE) {
                    const StagedPull<L, HAS_MASK, S> pull{a.src_h, a.src_g, hbuf + hslot(q) * Q * nx,
                                                          gbuf + (q & 1) * Q * nx, x, nx};
                    moments_site_f32<L, C, HAS_MASK, kPingPong, uint32_t>(a, idx, m, pull, sink);
                } else {
                    moments_site_f32<L, C, HAS_MASK, kPingPong, uint32_t>(
                        a, idx, m, global_pull<L, kPingPong, uint32_t, HAS_MASK>(a.src_h, a.src_g), sink);
                }
            } else {
                if (!(m & kSolidBit))
                    moments_site_canon<L, R, C, HAS_MASK, kPingPong, uint32_t>(
                        a, idx, m, [&](const R (&u)[3], R Pn, R phi) {
                            if (in_chunk) {
                                a.P_new[idx] = Pn;
                                static_for<0, 3>([&](auto A) {
                                    constexpr int ax = decltype(A)::value;
                                    a.u_new[(uint32_t)ax * N + (uint32_t)idx] = u[ax];
                                });
                            }
                            ring[slot * nx + x] = V4{u[0], u[1], u[2], phi};
                            stP[half * nx + x] = Pn;
                        });
            }
        }
        // halo piece j of this CTA: warps rotate over the planes
        const int j = ((warp - q * hw) % nw + nw) % nw;
        if (j < hw) {
            const int s = rank * HS + j * 32 + lane;   // 0 .. 2 nx - 1: lower row, then upper row
            const bool lower = s < nx;
            const int xh = lower ? s : s - nx;
            int yh = lower ? y0 - 1 : y0 + CY;
            if (yh < 0 || yh >= ny) {
                if (!g.yper) return;                  // outside a closed axis: never read
                yh = yh < 0 ? yh + ny : yh - ny;
            }
            V4 *dst = (lower ? halo_lo : halo_hi) + slot * nx + xh;
            const int idx = (qw * ny + yh) * nx + xh;
            uint32_t m = 0;
            if constexpr (HAS_MASK) m = a.mask[idx];
            if constexpr (kPacked<R>) {
                moments_site_f32<L, C, HAS_MASK, kPingPong, uint32_t>(
                    a, idx, m, global_pull<L, kPingPong, uint32_t, HAS_MASK>(a.src_h, a.src_g),
                    [&](float ux, float uy, float uz, float, float phi, const float *) {
                        *dst = make_float4(ux, uy, uz, phi);
                    });
            } else {
                if (!(m & kSolidBit))
                    moments_site_canon<L, R, C, HAS_MASK, kPingPong, uint32_t>(
                        a, idx, m, [&](const R (&u)[3], R, R phi) { *dst = V4{u[0], u[1], u[2], phi}; });
            }
        }
    };

    // --- S0 + S2..S5 of plane p (zb <= p < ze), own row
    auto collide_plane = [&](int p) {
        if (failed) return;
        const int idx = (p * ny + y) * nx + x;
        uint32_t m = 0;
        if constexpr (HAS_MASK) m = a.mask[idx];
        if (m & kSolidBit) return;
        const Nbr32 nb(idx, nx, ny, nz);
        const int sl[3] = {(p - 1) & (kClusterRing - 1), p & (kClusterRing - 1), (p + 1) & (kClusterRing - 1)};
        const V4 *rows[3] = {row_m, ring, row_p};
        const int xo[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        // (u, phi) at x + s c_i
        auto at = [&](auto I, int s) -> V4 {
            constexpr int i = decltype(I)::value;
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            return rows[1 + s * cy][sl[1 + s * cz] * nx + xo[1 + s * cx]];
        };
        const int half = p & 1;
        R hp[Q], hs[Q], gs[Q];
        if constexpr (kPacked<R>) {
            S hraw[Q];
            if constexpr (STAGE) {
                const StagedPull<L, HAS_MASK, S> pull{a.src_h, a.src_g, hbuf + hslot(p) * Q * nx, gbuf, x, nx};
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    if constexpr (i != 0 && HAS_MASK) {
                        if ((m >> i) & 1u) {
                            hraw[i] = a.src_h[(uint32_t)opp(i) * N + (uint32_t)idx];
                            return;
                        }
                    }
                    constexpr int cx = L::c(i, 0);
                    int xs = x - cx;
                    if constexpr (cx > 0) xs = xs < 0 ? xs + nx : xs;
                    if constexpr (cx < 0) xs = xs >= nx ? xs - nx : xs;
                    hraw[i] = pull.sh[i * nx + xs];
                });
            } else {
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    hraw[i] = a.src_h[read_idx<L, kPingPong, i, uint32_t>(N, nb, idx, m, HAS_MASK)];
                });
            }
            float pm[6];
            static_for<0, NS>([&](auto J) {
                constexpr int j = decltype(J)::value;
                pm[j] = stM[(half * NS + j) * nx + x];
            });
            const float4 f0 = ring[sl[1] * nx + x];
            const float u[3] = {f0.x, f0.y, f0.z};
            const float phi = f0.w;
            const float P = stP[half * nx + x];
            float gphi[3], lphi, gu[3][3];
            if (m == 0u) stencil_packed<L, false>(at, m, phi, gphi, lphi, gu);
            else stencil_packed<L, true>(at, m, phi, gphi, lphi, gu);
            const float phihat = a.k.clamp ? clamp01(phi) : phi;
            const float rho = a.k.rho_a + phihat * a.k.drho;
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                hp[i] = C::template dec_h<i>(hraw[i]);
            });
            collide_pairs<L, false, C::kPdev, true, false>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, nullptr,
                                                           hs, gs, pm, nullptr);
            if (!(isfinite(phi) && isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2])))
                atomicOr(a.err, 1);
        } else {
            const V4 f0 = ring[sl[1] * nx + x];
            const R phi = f0.w;
            R gphi[3], lphi;
            stencil<L, R>([&](auto I, int s) { return at(I, s).w; }, m, phi, phi, gphi, lphi);
            R u[3] = {f0.x, f0.y, f0.z}, gu[3][3], lap_unused;
            stencil<L, R>([&](auto I, int s) { return at(I, s).x; }, m, u[0], R(0), gu[0], lap_unused);
            stencil<L, R>([&](auto I, int s) { return at(I, s).y; }, m, u[1], R(0), gu[1], lap_unused);
            stencil<L, R>([&](auto I, int s) { return at(I, s).z; }, m, u[2], R(0), gu[2], lap_unused);
            const R P = stP[half * nx + x];
            const R phihat = a.k.clamp ? clamp01(phi) : phi;
            const R rho = a.k.rho_a + phihat * a.k.drho;
            R gp[Q];
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const uint32_t e = read_idx<L, kPingPong, i, uint32_t>(N, nb, idx, m, HAS_MASK);
                hp[i] = C::template dec_h<i>(a.src_h[e]);
                gp[i] = C::template dec_g<i>(a.src_g[e]);
            });
            collide<L, R, false, C::kPdev>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, gp, hs, gs);
            if (!(isfinite(phi) && isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2])))
                atomicOr(a.err, 1);
        }
        compensate_h<L, C>(hs);
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const uint32_t e = eidx<uint32_t>(i, N, idx);
            if constexpr (i == 0 && C::kRound16) {
                a.dst_h[e] = C::template enc_h_sr<0>(hs[0], mix32((uint32_t)idx * 0x9e3779b9u ^ mix32(a.seed)));
            } else {
                a.dst_h[e] = C::template enc_h<i>(hs[i]);
            }
            a.dst_g[e] = C::template enc_g<i>(gs[i]);
        });
    };

    // Order: copies of plane q are issued two planes ahead, after the
    // barrier that ends the last reads of their buffers (g: moments of q-2,
    // h: collision of q-3).
    issue(zb - 1);
    issue(zb);
    await(zb - 1);
    moments(zb - 1);
    await(zb);
    moments(zb);
    cl.sync();
    if (zb + 1 <= ze) issue(zb + 1);
    for (int p = zb; p < ze; ++p) {
        await(p + 1);
        moments(p + 1);
        cl.sync();
        if (p + 2 <= ze) issue(p + 2);
        collide_plane(p);
    }
    cl.sync();
}

// True when the cluster step can run this lattice (see the file header).
inline bool cluster_ok(int D, int Q, int nx, int ny, long long N, int cy, bool inplace, bool godd)
{
    return D == 3 && !inplace && !godd && nx % 32 == 0 && nx <= kClusterMaxThreads && cy >= 2 && ny % cy == 0 &&
           (2 * nx) % (32 * cy) == 0 && split_idx32(Q, N);
}

}  // namespace lbm
