// Split form of the coupled step: two launches per time step, one thread per
// site, no shared memory and no block-wide synchronisation.
//
//   moments_kernel  (S0, S1): pull both populations, phi = sum h_i, K_i,
//                   u^{n+1}, P^{n+1}; write phi, u^{n+1}, P^{n+1} (FP32
//                   arithmetic: as packed words, with the second moments of
//                   the pulled g, see below).
//   collide_kernel  (S0, S2..S5): stencils of phi and u^{n+1} read from what
//                   the first launch wrote (L1/L2 hits), pull the populations
//                   again (FP32 arithmetic: h only), both collisions, store.
//
// The grid-wide dependency between the moments and their stencils is the
// launch boundary, so no halo is recomputed; the price is a second read of
// populations and the hand-over between the launches (measured 633 instead
// of 464 B per FP32 D3Q27 site update).  The
// split form also admits in-place streaming: with the AA pattern a site
// reads and writes one and the same set of population slots in every step,
// so both launches can work on a single population store.
//
// Population addressing (slot i of site x is pop[i * N + x]):
//   ping-pong   read  f_i(x) = src[i][x - c_i]                write dst[i][x]
//   AA, even    read  f_i(x) = pop[i][x]                      write pop[-i][x]
//   AA, odd     read  f_i(x) = pop[-i][x - c_i]               write pop[i][x + c_i]
// with halfway bounce-back: a solid source x - c_i reads the site's own
// post-collision value of -i (ping-pong: src[-i][x]; AA odd: pop[i][x]); a
// solid destination x + c_i in an odd step stores to pop[-i][x].  After an
// even step (and after initialisation) the post-collision f*_i(x) sits in
// pop[-i][x]; after an odd step in pop[i][x + c_i] (pop[-i][x] next to a
// solid).
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

// Site coordinates and wrapped neighbour offsets in 32 bits (N < 2^31 sites):
// the site x + s c is xo[1 + s c_x] + yo[1 + s c_y] + zo[1 + s c_z].  Slot i
// of a population set is its own plane base + (size_t)i * N, a value uniform
// across the grid, so an access costs one 32-bit offset and one wide
// multiply-add on top of the load.
struct Nbr32 {
    int xo[3], yo[3], zo[3];
    __device__ __forceinline__ Nbr32(int idx, int nx, int ny, int nz)
    {
        const int x = idx % nx;
        const int y = (idx / nx) % ny;
        const int z = idx / (nx * ny);
        const int nxy = nx * ny;
        xo[0] = wrapc(x - 1, nx); xo[1] = x; xo[2] = wrapc(x + 1, nx);
        yo[0] = wrapc(y - 1, ny) * nx; yo[1] = y * nx; yo[2] = wrapc(y + 1, ny) * nx;
        zo[0] = wrapc(z - 1, nz) * nxy; zo[1] = z * nxy; zo[2] = wrapc(z + 1, nz) * nxy;
    }
    template <class L, int i>
    __device__ __forceinline__ int at(int s) const
    {
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        if (s > 0) return xo[1 + cx] + yo[1 + cy] + zo[1 + cz];
        return xo[1 - cx] + yo[1 - cy] + zo[1 - cz];
    }
};

// Element index slot * N + off in the index type IX: 32-bit unsigned when
// Q N < 2^32 (one multiply-add per access, no 64-bit arithmetic), else
// 64-bit.
template <class IX>
__device__ __forceinline__ IX eidx(int slot, IX N, int off)
{
    return (IX)slot * N + (IX)off;
}

// Index at which f_i(x) is read, for the stream mode.
template <class L, int MODE, int i, class IX>
__device__ __forceinline__ IX read_idx(IX N, const Nbr32 &nb, int idx, uint32_t m, bool has_mask)
{
    if constexpr (i == 0) {
        return (IX)idx;                               // rest population never moves
    } else {
        const bool bb = has_mask && ((m >> i) & 1u);  // x - c_i solid/outside
        if constexpr (MODE == kPingPong)
            return bb ? eidx<IX>(opp(i), N, idx) : eidx<IX>(i, N, nb.at<L, i>(-1));
        else if constexpr (MODE == kAAEven)
            return eidx<IX>(i, N, idx);
        else
            return bb ? eidx<IX>(i, N, idx) : eidx<IX>(opp(i), N, nb.at<L, i>(-1));
    }
}

// Index to which f*_i(x) is written, for the stream mode.
template <class L, int MODE, int i, class IX>
__device__ __forceinline__ IX write_idx(IX N, const Nbr32 &nb, int idx, uint32_t m, bool has_mask)
{
    if constexpr (i == 0) {
        return (IX)idx;
    } else if constexpr (MODE == kPingPong) {
        return eidx<IX>(i, N, idx);
    } else if constexpr (MODE == kAAEven) {
        return eidx<IX>(opp(i), N, idx);
    } else {
        const bool bb = has_mask && ((m >> opp(i)) & 1u);   // x + c_i solid/outside
        return bb ? eidx<IX>(opp(i), N, idx) : eidx<IX>(i, N, nb.at<L, i>(1));
    }
}

// FP32 arithmetic keeps the state (u, P) of each site as one packed 16-byte
// word while it steps in the split form: the moments launch reads a
// neighbour's velocity and pressure with one load.  It also leaves for the
// collision launch the packed (u, phi) words of the new step and the second
// moments sum_i c_ia c_ib g_i of the pulled g, which is all the filter
// collision needs of g, so the collision launch pulls h only.
//
// BF16 storage: in the light phase the odd part of g*, w_i c_i . V_g with
// V_g = u/T + F/(rho T) + sigma grad rho/(rho^2 T), is hundreds of times the
// velocity it leaves after the pull (F/rho and grad P/rho nearly cancel), so
// rounding g* to 8 significant bits would swamp u.  The collision launch stores g*
// without that part, in 16 bits, and V_g per site in FP32; the next pull adds
// w_i c_i . V_g of the site the population left back.
template <class R>
inline constexpr bool kPacked = std::is_same<R, float>::value;

constexpr int kSplitThreads = 128;
constexpr int kSplitMinBlocks = 4;   // <= 128 registers a thread: 16 warps an SM

// S0 + S1 at site idx (0 <= idx < a.N).
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__device__ __forceinline__ void moments_site(const SplitArgs<R, typename C::S> &a, const int idx)
{
    constexpr int D = L::D, Q = L::Q;
    uint32_t m = 0;
    if constexpr (HAS_MASK) m = a.mask[idx];
    if (m & kSolidBit) return;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    R hp[Q], gp[Q], Pn[Q], K[Q];
    R P0;
    if constexpr (kPacked<R>) P0 = a.F_old[idx].w;
    else P0 = a.P_old[idx];
    R sum_wcu = R(0);
    [[maybe_unused]] float vgown[3];
    if constexpr (kPacked<R> && C::kGodd) {
        const float4 v4 = a.G_old[idx];
        vgown[0] = v4.x; vgown[1] = v4.y; vgown[2] = v4.z;
    }
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const IX e = read_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK);
        hp[i] = C::template dec_h<i>(a.src_h[e]);
        gp[i] = C::template dec_g<i>(a.src_g[e]);
        if constexpr (i == 0) {
            Pn[0] = P0;
        } else {
            const bool bb = HAS_MASK && ((m >> i) & 1u);
            const int src = nb.at<L, i>(-1);
            R un[3];
            if constexpr (kPacked<R>) {
                const float4 f = a.F_old[src];
                Pn[i] = bb ? P0 : f.w;
                un[0] = f.x; un[1] = f.y; un[2] = f.z;
                if constexpr (C::kGodd) {
                    // add back the odd part w_i c_i . V_g of the site the population
                    // left (bounce-back: g*_{-i}(x), whose part is - w_i c_i . V_g(x))
                    const float4 v4 = a.G_old[src];
                    const float vs[3] = {v4.x, v4.y, v4.z};
                    const float corr = bb ? -dot_c<L, i>(vgown) : dot_c<L, i>(vs);
                    gp[i] = gp[i] + float(L::w(i)) * corr;
                }
            } else {
                Pn[i] = bb ? P0 : a.P_old[src];
                static_for<0, 3>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    if constexpr (ax < D && L::c(i, ax) != 0) {
                        if (!bb) un[ax] = a.u_old[eidx<IX>(ax, N, src)];
                    } else {
                        un[ax] = R(0);
                    }
                });
            }
            if (!bb) sum_wcu = sum_wcu + R(L::w(i)) * dot_c<L, i>(un);
        }
    });
    R phi, phihat, rho, u[3], sumg, sumK;
    R Pnew;
    if constexpr (kPairForms<R>) {
        s1_pairs<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, sumg, sumK);
        Pnew = s1_pressure_pairs<R, C::kPdev>(a.k, rho, sumg, sumK, sum_wcu, P0);
    } else {
        s1_moments<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, K);
        Pnew = s1_pressure<L, R, C::kPdev>(a.k, gp, K, rho, sum_wcu, P0);
    }
    if constexpr (kPacked<R>) {
        const float uz = D == 3 ? u[2] : 0.f;
        a.F_new[idx] = make_float4(u[0], u[1], uz, Pnew);
        a.FB[idx] = make_float4(u[0], u[1], uz, phi);
        // sum_i c_ia c_ib g_i, per pair (c_ia c_ib is even in c)
        constexpr int NS = D == 3 ? 6 : 3;
        float pm[NS];
        static_for<0, NS>([&](auto J) { pm[decltype(J)::value] = 0.f; });
        static_for<0, (Q - 1) / 2>([&](auto Pp) {
            constexpr int i = 2 * decltype(Pp)::value + 1;
            const float gsum = gp[i] + gp[i + 1];
            static_for<0, D>([&](auto A) {
                constexpr int a0 = decltype(A)::value;
                static_for<a0, D>([&](auto Bb) {
                    constexpr int b0 = decltype(Bb)::value;
                    constexpr int cc = L::c(i, a0) * L::c(i, b0);
                    if constexpr (cc != 0) acc_c<cc>(pm[pig_slot<D>(a0, b0)], gsum);
                });
            });
        });
        static_for<0, NS>([&](auto J) {
            constexpr int j = decltype(J)::value;
            a.PiG[eidx<IX>(j, N, idx)] = pm[j];
        });
    } else {
        a.P_new[idx] = Pnew;
        static_for<0, D>([&](auto A) {
            constexpr int ax = decltype(A)::value;
            a.u_new[eidx<IX>(ax, N, idx)] = u[ax];
        });
        a.phi[idx] = phi;
    }
}

// Load that bypasses L1 when CG: for data other blocks wrote earlier in the
// same launch (the persistent step).
template <bool CG, class T>
__device__ __forceinline__ T ld_maybe_cg(const T *p)
{
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// S0 + S2..S5 at site idx (0 <= idx < a.N).
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX, bool CG = false>
__device__ __forceinline__ void collide_site(const SplitArgs<R, typename C::S> &a, const int idx)
{
    constexpr int D = L::D, Q = L::Q;
    uint32_t m = 0;
    if constexpr (HAS_MASK) m = a.mask[idx];
    if (m & kSolidBit) return;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    // S2: stencils of phi^{n+1} and u^{n+1} from the fields of the moments launch
    R phi, gphi[3], lphi;
    R u[3], gu[3][3];
    R P;
    if constexpr (kPacked<R>) {
        const float4 f0 = ld_maybe_cg<CG>(a.FB + idx);
        u[0] = f0.x; u[1] = f0.y; u[2] = f0.z;
        phi = f0.w;
        P = ld_maybe_cg<CG>(a.F_new + idx).w;
        auto at = [&](auto I, int s) { return ld_maybe_cg<CG>(a.FB + nb.at<L, decltype(I)::value>(s)); };
        if (m == 0u) stencil_packed<L, false>(at, m, phi, gphi, lphi, gu);
        else stencil_packed<L, true>(at, m, phi, gphi, lphi, gu);
    } else {
        P = a.P_new[idx];
        phi = a.phi[idx];
        stencil_any<L, R>([&](auto I, int s) { return a.phi[nb.at<L, decltype(I)::value>(s)]; }, m, phi, phi, gphi,
                          lphi);
        u[2] = R(0);
        gu[0][2] = gu[1][2] = gu[2][0] = gu[2][1] = gu[2][2] = R(0);
        static_for<0, D>([&](auto A) {
            constexpr int ax = decltype(A)::value;
            u[ax] = a.u_new[eidx<IX>(ax, N, idx)];
            R lap_unused;
            stencil_any<L, R>(
                [&](auto I, int s) { return a.u_new[eidx<IX>(ax, N, nb.at<L, decltype(I)::value>(s))]; }, m, u[ax],
                R(0), gu[ax], lap_unused);
        });
    }
    const R phihat = a.k.clamp ? clamp01(phi) : phi;
    const R rho = a.k.rho_a + phihat * a.k.drho;
    R hp[Q], hs[Q], gs[Q];
    if constexpr (kPacked<R>) {
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            hp[i] = C::template dec_h<i>(a.src_h[read_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK)]);
        });
        constexpr int NS = D == 3 ? 6 : 3;
        float pm[NS];
        static_for<0, NS>([&](auto J) {
            constexpr int j = decltype(J)::value;
            pm[j] = ld_maybe_cg<CG>(a.PiG + eidx<IX>(j, N, idx));
        });
        float vg[3];
        collide_pairs<L, false, C::kPdev, true, C::kGodd>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, nullptr,
                                                         hs, gs, pm, vg);
        if constexpr (C::kGodd) a.G_new[idx] = make_float4(vg[0], vg[1], vg[2], 0.f);
    } else {
        R gp[Q];
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const IX e = read_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK);
            hp[i] = C::template dec_h<i>(a.src_h[e]);
            gp[i] = C::template dec_g<i>(a.src_g[e]);
        });
        collide<L, R, false, C::kPdev>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, gp, hs, gs);
    }
    compensate_h<L, C>(hs);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const IX e = write_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK);
        if constexpr (i == 0 && C::kRound16) {
            // the rest population carries the site's rounding: round it without
            // bias, so a liquid just above phi = 1 does not lose mass step by step
            a.dst_h[e] = C::template enc_h_sr<0>(hs[0], mix32((uint32_t)idx * 0x9e3779b9u ^ mix32(a.seed)));
        } else {
            a.dst_h[e] = C::template enc_h<i>(hs[i]);
        }
        a.dst_g[e] = C::template enc_g<i>(gs[i]);
    });
    if (!(isfinite(phi) && isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2])))
        atomicOr(a.err, 1);
}

template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__global__ void __launch_bounds__(kSplitThreads, kSplitMinBlocks) moments_kernel(const SplitArgs<R, typename C::S> a)
{
    const long long idx = (long long)blockIdx.x * kSplitThreads + threadIdx.x;
    if (idx < a.N) moments_site<L, R, C, HAS_MASK, MODE, IX>(a, (int)idx);
}

template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__global__ void __launch_bounds__(kSplitThreads, kSplitMinBlocks) collide_kernel(const SplitArgs<R, typename C::S> a)
{
    const long long idx = (long long)blockIdx.x * kSplitThreads + threadIdx.x;
    if (idx < a.N) collide_site<L, R, C, HAS_MASK, MODE, IX>(a, (int)idx);
}

// True when every element index of the lattice's population sets fits in 32
// bits, so the kernels can take the 32-bit index path.
inline bool split_idx32(int Q, long long N) { return (unsigned long long)Q * (unsigned long long)N < (1ULL << 32); }

}  // namespace lbm
