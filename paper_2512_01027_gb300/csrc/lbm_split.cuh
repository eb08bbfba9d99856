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

// Source of the pulled populations of the moments: GlobalPull reads them
// from the population store at read_idx (every stream mode, bounce-back
// included); the cluster step substitutes rows it staged in shared memory.
template <class L, int MODE, class IX, bool HAS_MASK, class S>
struct GlobalPull {
    const S *h, *g;
    template <int i>
    __device__ __forceinline__ void get(IX N, const Nbr32 &nb, int idx, uint32_t m, S &hr, S &gr) const
    {
        const IX e = read_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK);
        hr = h[e];
        gr = g[e];
    }
};

template <class L, int MODE, class IX, bool HAS_MASK, class S>
__device__ __forceinline__ GlobalPull<L, MODE, IX, HAS_MASK, S> global_pull(const S *h, const S *g)
{
    return GlobalPull<L, MODE, IX, HAS_MASK, S>{h, g};
}

// S0 + S1 at site idx with FP32 arithmetic.  Every pulled population and
// every neighbour word goes straight into running sums, so no per-direction
// value waits for phi: 1/(T rho) multiplies the pressure sums once, after the
// loop.  The sums are those of s1_pairs and s1_pressure_pairs (u = sum of the
// g differences + 1/(T rho) sum w_i c_i {P(x - c_i) - P(x + c_i)} per pair),
// accumulated as the loads arrive, which leaves registers for more loads in
// flight.
template <class L, class C, bool HAS_MASK, int MODE, class IX, class Pull, class Sink>
__device__ __forceinline__ void moments_site_packed(const SplitArgs<float, typename C::S> &a, const int idx,
                                                    const uint32_t m, const Pull &pull, Sink &&sink)
{
    constexpr int D = L::D, Q = L::Q;
    constexpr int NS = D == 3 ? 6 : 3;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    const float P0 = a.F_old[idx].w;
    [[maybe_unused]] float vgown[3];
    if constexpr (C::kGodd) {
        const float4 v4 = a.G_old[idx];
        vgown[0] = v4.x; vgown[1] = v4.y; vgown[2] = v4.z;
    }
    float phi = 0.f, sumg = 0.f, swP = 0.f, sum_wcu = 0.f;
    float ug[3] = {0.f, 0.f, 0.f}, up[3] = {0.f, 0.f, 0.f}, pm[NS];
    static_for<0, NS>([&](auto J) { pm[decltype(J)::value] = 0.f; });
    float gfirst = 0.f, pfirst = 0.f;   // the first member (c) of the current pair (c, -c)
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        typename C::S hr, gr;
        pull.template get<i>(N, nb, idx, m, hr, gr);
        const float hv = C::template dec_h<i>(hr);
        float gv = C::template dec_g<i>(gr);
        if constexpr (i == 0) {
            phi = hv;
            sumg = gv;
        } else {
            phi = phi + hv;
            const bool bb = HAS_MASK && ((m >> i) & 1u);
            const int src = nb.at<L, i>(-1);
            const float4 f = a.F_old[src];
            const float pn = bb ? P0 : f.w;
            if constexpr (C::kGodd) {
                // add back the odd part w_i c_i . V_g of the site the population
                // left (bounce-back: g*_{-i}(x), whose part is - w_i c_i . V_g(x))
                const float4 v4 = a.G_old[src];
                const float vs[3] = {v4.x, v4.y, v4.z};
                const float corr = bb ? -dot_c<L, i>(vgown) : dot_c<L, i>(vs);
                gv = gv + float(L::w(i)) * corr;
            }
            if (!bb) {
                const float un[3] = {f.x, f.y, f.z};
                sum_wcu = sum_wcu + float(L::w(i)) * dot_c<L, i>(un);
            }
            if constexpr (i & 1) {
                gfirst = gv;
                pfirst = pn;
            } else {
                constexpr int ic = i - 1;                    // c_i = -c_ic
                const float wi = float(L::w(ic));
                const float dg = gfirst - gv, dp = wi * (pfirst - pn);
                static_for<0, 3>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    if constexpr (L::c(ic, ax) != 0) {
                        acc_c<L::c(ic, ax)>(ug[ax], dg);
                        acc_c<L::c(ic, ax)>(up[ax], dp);
                    }
                });
                const float gsum = gfirst + gv;
                sumg = sumg + gsum;
                swP = swP + wi * (pfirst + pn);
                // sum_i c_ia c_ib g_i (c_ia c_ib is even in c)
                static_for<0, D>([&](auto A) {
                    constexpr int a0 = decltype(A)::value;
                    static_for<a0, D>([&](auto Bb) {
                        constexpr int b0 = decltype(Bb)::value;
                        constexpr int cc = L::c(ic, a0) * L::c(ic, b0);
                        if constexpr (cc != 0) acc_c<cc>(pm[pig_slot<D>(a0, b0)], gsum);
                    });
                });
            }
        }
    });
    const float phihat = a.k.clamp ? clamp01(phi) : phi;
    const float rho = a.k.rho_a + phihat * a.k.drho;
    const float kfac = 3.f / rho;                        // 1 / (T rho)
    float u[3];
    static_for<0, 3>([&](auto A) {
        constexpr int ax = decltype(A)::value;
        u[ax] = ug[ax] + kfac * up[ax];                  // u = sum_i (g_i + K_i) c_i
    });
    const float sumK = kfac * (swP - float(1.0 - L::w(0)) * P0);
    // the u^{n+1} coupling leaves the omega-term to the collision launch
    const float Pnew = s1_pressure_pairs<float, C::kPdev>(a.k, rho, sumg, sumK, a.k.coupling ? 0.f : sum_wcu, P0);
    const float uz = D == 3 ? u[2] : 0.f;
    sink(u[0], u[1], uz, Pnew, phi, pm);
}

// Separable neighbour sums (D3Q27).  Its weights factor over the axes,
// w_i = s(c_ix) s(c_iy) s(c_iz) with s(0) = 2/3 and s(+-1) = 1/6, so a
// weighted sum over the 27 neighbours is three passes of three points: a
// smoothing S = (1/6, 2/3, 1/6) or a difference D = (-1/6, 0, 1/6) along each
// axis.  A warp whose 32 sites are consecutive in x and have no solid or
// outside neighbour does the y and z passes on its own column (9 loads instead
// of 26) and the x pass across lanes with shuffles; lanes 0 and 31 also
// sum the columns just outside the warp.
constexpr float kS0 = 2.f / 3.f, kS1 = 1.f / 6.f;

__device__ __forceinline__ float sm3(float m, float c, float p) { return kS1 * (m + p) + kS0 * c; }
__device__ __forceinline__ float df3(float m, float p) { return kS1 * (p - m); }

// y and z passes over the packed (u, P) words of one column, rows r[1 + dy][1 + dz]:
// sP = S_y S_z P, dyP = D_y S_z P, dzP = S_y D_z P, sUx = S_y S_z u_x,
// e = D_y S_z u_y + S_y D_z u_z.
struct ColUP {
    float sP, dyP, dzP, sUx, e;
};

__device__ __forceinline__ ColUP col_up(const float4 (&r)[3][3])
{
    float szP[3], dzP[3], szUx[3], szUy[3], dzUz[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        szP[j] = sm3(r[j][0].w, r[j][1].w, r[j][2].w);
        dzP[j] = df3(r[j][0].w, r[j][2].w);
        szUx[j] = sm3(r[j][0].x, r[j][1].x, r[j][2].x);
        szUy[j] = sm3(r[j][0].y, r[j][1].y, r[j][2].y);
        dzUz[j] = df3(r[j][0].z, r[j][2].z);
    }
    ColUP o;
    o.sP = sm3(szP[0], szP[1], szP[2]);
    o.dyP = df3(szP[0], szP[2]);
    o.dzP = sm3(dzP[0], dzP[1], dzP[2]);
    o.sUx = sm3(szUx[0], szUx[1], szUx[2]);
    o.e = df3(szUy[0], szUy[2]) + sm3(dzUz[0], dzUz[1], dzUz[2]);
    return o;
}

__device__ __forceinline__ void load_col(const float4 *F, int xo, const Nbr32 &nb, float4 (&r)[3][3])
{
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) r[j][k] = F[xo + nb.yo[j] + nb.zo[k]];
}

// Column whose sums lane 0 (x - 1) and lane 31 (x + 1) need from outside the
// warp.  The other lanes load their own column again (L1 hits), so the loads
// go out without a branch, together with those of the own column.
__device__ __forceinline__ int halo_col(const Nbr32 &nb, int lane)
{
    return lane == 0 ? nb.xo[0] : (lane == 31 ? nb.xo[2] : nb.xo[1]);
}

// Value of the lane at x - 1 (lane 0: h, the column before the warp) and at x + 1.
__device__ __forceinline__ float lane_xm(float v, float h, int lane)
{
    const float t = __shfl_up_sync(0xffffffffu, v, 1);
    return lane == 0 ? h : t;
}
__device__ __forceinline__ float lane_xp(float v, float h, int lane)
{
    const float t = __shfl_down_sync(0xffffffffu, v, 1);
    return lane == 31 ? h : t;
}

// S0 + S1 at site idx, separable form (D3Q27, FP32 arithmetic, a warp of 32
// sites in one row, none with a solid or outside neighbour; every lane of the
// warp calls it).  With no bounce-back every sum runs over all 26 neighbours:
//   sum_i w_i P(x - c_i)         = S_x S_y S_z P
//   sum_i w_i c_ia P(x - c_i)    = - D_a S S P
//   sum_i w_i c_i . u(x - c_i)   = - sum_a D_a S S u_a
// the same quantities moments_site_packed sums direction by direction.
template <class L, class C, int MODE, class IX, class Pull, class Sink>
__device__ __forceinline__ void moments_site_sep(const SplitArgs<float, typename C::S> &a, const int idx,
                                                 const Pull &pull, Sink &&sink)
{
    static_assert(L::Q == 27 && !C::kGodd, "separable moments: D3Q27 without the odd-part deferral");
    constexpr int Q = L::Q, NS = 6;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, a.nz);
    const int lane = (int)(threadIdx.x & 31u);
    float4 r[3][3], rh[3][3];
    load_col(a.F_old, nb.xo[1], nb, r);
    load_col(a.F_old, halo_col(nb, lane), nb, rh);
    const float P0 = r[1][1].w;
    float phi = 0.f, sumg = 0.f;
    float ug[3] = {0.f, 0.f, 0.f}, pm[NS];
    static_for<0, NS>([&](auto J) { pm[decltype(J)::value] = 0.f; });
    float gfirst = 0.f;
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        typename C::S hr, gr;
        pull.template get<i>(N, nb, idx, 0u, hr, gr);
        const float hv = C::template dec_h<i>(hr);
        const float gv = C::template dec_g<i>(gr);
        if constexpr (i == 0) {
            phi = hv;
            sumg = gv;
        } else {
            phi = phi + hv;
            if constexpr (i & 1) {
                gfirst = gv;
            } else {
                constexpr int ic = i - 1;
                const float dg = gfirst - gv;
                static_for<0, 3>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    if constexpr (L::c(ic, ax) != 0) acc_c<L::c(ic, ax)>(ug[ax], dg);
                });
                const float gsum = gfirst + gv;
                sumg = sumg + gsum;
                static_for<0, 3>([&](auto A) {
                    constexpr int a0 = decltype(A)::value;
                    static_for<a0, 3>([&](auto Bb) {
                        constexpr int b0 = decltype(Bb)::value;
                        constexpr int cc = L::c(ic, a0) * L::c(ic, b0);
                        if constexpr (cc != 0) acc_c<cc>(pm[pig_slot<3>(a0, b0)], gsum);
                    });
                });
            }
        }
    });
    const ColUP own = col_up(r);
    const ColUP hal = col_up(rh);
    const float sPm = lane_xm(own.sP, hal.sP, lane), sPp = lane_xp(own.sP, hal.sP, lane);
    const float sssP = sm3(sPm, own.sP, sPp);
    float up[3];
    up[0] = -df3(sPm, sPp);
    up[1] = -sm3(lane_xm(own.dyP, hal.dyP, lane), own.dyP, lane_xp(own.dyP, hal.dyP, lane));
    up[2] = -sm3(lane_xm(own.dzP, hal.dzP, lane), own.dzP, lane_xp(own.dzP, hal.dzP, lane));
    const float divu = df3(lane_xm(own.sUx, hal.sUx, lane), lane_xp(own.sUx, hal.sUx, lane)) +
                       sm3(lane_xm(own.e, hal.e, lane), own.e, lane_xp(own.e, hal.e, lane));
    const float sum_wcu = a.k.coupling ? 0.f : -divu;   // the u^{n+1} coupling: added by the collision
    const float swP = sssP - float(L::w(0)) * P0;
    const float phihat = a.k.clamp ? clamp01(phi) : phi;
    const float rho = a.k.rho_a + phihat * a.k.drho;
    const float kfac = 3.f / rho;
    float u[3];
    static_for<0, 3>([&](auto A) {
        constexpr int ax = decltype(A)::value;
        u[ax] = ug[ax] + kfac * up[ax];
    });
    const float sumK = kfac * (swP - float(1.0 - L::w(0)) * P0);
    const float Pnew = s1_pressure_pairs<float, C::kPdev>(a.k, rho, sumg, sumK, sum_wcu, P0);
    sink(u[0], u[1], u[2], Pnew, phi, pm);
}

// True when the separable form applies to this kernel instantiation (its
// BF16 odd-part corrections are per direction).
template <class L, class R, class C>
inline constexpr bool kSepForm = kPacked<R> && L::Q == 27 && !C::kGodd;

// The split form's hand-over of the moments (FP32 arithmetic): the packed
// (u^{n+1}, P^{n+1}) state word, the packed (u^{n+1}, phi^{n+1}) word and
// the second moments of the pulled g.
template <class L, class C, class IX>
__device__ __forceinline__ auto split_sink(const SplitArgs<float, typename C::S> &a, const int idx)
{
    return [&a, idx](float ux, float uy, float uz, float Pnew, float phi, const float *pm) {
        constexpr int NS = L::D == 3 ? 6 : 3;
        a.F_new[idx] = make_float4(ux, uy, uz, Pnew);
        a.FB[idx] = make_float4(ux, uy, uz, phi);
        static_for<0, NS>([&](auto J) {
            constexpr int j = decltype(J)::value;
            a.PiG[eidx<IX>(j, (IX)a.N, idx)] = pm[j];
        });
    };
}

// S0 + S1 at site idx with FP32 arithmetic, results to sink(u_x, u_y, u_z,
// P^{n+1}, phi^{n+1}, pm).  A warp whose sites have no solid or outside
// neighbour (a warp vote, where a.vote says that all 32 lanes call this
// together) takes the code without bounce-back selections.  D3Q27 takes the
// separable sums there instead, which need the warp's 32 sites in one row
// (nx a multiple of 32); with other nx it keeps one copy of the pair code,
// so the kernel does not carry three.
template <class L, class C, bool HAS_MASK, int MODE, class IX, class Pull, class Sink>
__device__ __forceinline__ void moments_site_f32(const SplitArgs<float, typename C::S> &a, const int idx,
                                                 const uint32_t m, const Pull &pull, Sink &&sink)
{
    if constexpr (kSepForm<L, float, C>) {
        if ((a.nx & 31) == 0 && !(HAS_MASK && __any_sync(0xffffffffu, m != 0u))) {
            moments_site_sep<L, C, MODE, IX>(a, idx, pull, sink);
            return;
        }
    } else {
        if (!HAS_MASK || (a.vote && !__any_sync(0xffffffffu, m != 0u))) {
            moments_site_packed<L, C, false, MODE, IX>(a, idx, 0u, pull, sink);
            return;
        }
    }
    if (m & kSolidBit) return;
    moments_site_packed<L, C, HAS_MASK, MODE, IX>(a, idx, m, pull, sink);
}

// S0 + S1 at a fluid site idx in the canonical order of the oracle (FP64),
// results to sink(u, P^{n+1}, phi^{n+1}).
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX, class Sink>
__device__ __forceinline__ void moments_site_canon(const SplitArgs<R, typename C::S> &a, const int idx,
                                                   const uint32_t m, Sink &&sink)
{
    constexpr int D = L::D, Q = L::Q;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    R hp[Q], gp[Q], Pn[Q], K[Q];
    const R P0 = a.P_old[idx];
    R sum_wcu = R(0);
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
            Pn[i] = bb ? P0 : a.P_old[src];
            static_for<0, 3>([&](auto A) {
                constexpr int ax = decltype(A)::value;
                if constexpr (ax < D && L::c(i, ax) != 0) {
                    if (!bb) un[ax] = a.u_old[eidx<IX>(ax, N, src)];
                } else {
                    un[ax] = R(0);
                }
            });
            if (!bb) sum_wcu = sum_wcu + R(L::w(i)) * dot_c<L, i>(un);
        }
    });
    R phi, phihat, rho, u[3];
    s1_moments<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, K);
    // the u^{n+1} coupling: the collision launch adds the omega-term
    const R Pnew = s1_pressure<L, R, C::kPdev>(a.k, gp, K, rho, a.k.coupling ? R(0) : sum_wcu, P0);
    sink(u, Pnew, phi);
}

// S0 + S1 at site idx (0 <= idx < a.N).  FP64: the canonical order of the
// oracle; FP32 arithmetic: moments_site_f32 into the split form's hand-over.
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__device__ __forceinline__ void moments_site(const SplitArgs<R, typename C::S> &a, const int idx)
{
    constexpr int D = L::D;
    uint32_t m = 0;
    if constexpr (HAS_MASK) m = a.mask[idx];
    if constexpr (kPacked<R>) {
        moments_site_f32<L, C, HAS_MASK, MODE, IX>(a, idx, m, global_pull<L, MODE, IX, HAS_MASK>(a.src_h, a.src_g),
                                                   split_sink<L, C, IX>(a, idx));
    } else {
        if (m & kSolidBit) return;
        moments_site_canon<L, R, C, HAS_MASK, MODE, IX>(a, idx, m, [&](const R (&u)[3], R Pnew, R phi) {
            const IX N = (IX)a.N;
            a.P_new[idx] = Pnew;
            static_for<0, D>([&](auto A) {
                constexpr int ax = decltype(A)::value;
                a.u_new[eidx<IX>(ax, N, idx)] = u[ax];
            });
            a.phi[idx] = phi;
        });
    }
}

// S0 + S2..S5 at site idx (0 <= idx < a.N).
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__device__ __forceinline__ void collide_site_impl(const SplitArgs<R, typename C::S> &a, const int idx,
                                                  const uint32_t m)
{
    constexpr int D = L::D, Q = L::Q;
    if (m & kSolidBit) return;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    // S2: stencils of phi^{n+1} and u^{n+1} from the fields of the moments launch
    R phi, gphi[3], lphi;
    R u[3], gu[3][3];
    R P;
    constexpr int NS = D == 3 ? 6 : 3;
    [[maybe_unused]] typename C::S hraw[Q];
    [[maybe_unused]] float pm[NS];
    // 4-byte storage, ping-pong store: the pulled h and the second moments of
    // g are issued before the stencil's loads (a compiler-only fence keeps
    // that order), so that a thread has its loads in flight together.  With
    // 16-bit storage (decoding) and in the in-place store (its index
    // selections) the registers do not allow it: there they follow the stencil.
    constexpr bool kEarlyH = kPacked<R> && sizeof(typename C::S) == 4 && MODE == kPingPong;
    auto load_h_pig = [&]() {
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            hraw[i] = a.src_h[read_idx<L, MODE, i, IX>(N, nb, idx, m, HAS_MASK)];
        });
        static_for<0, NS>([&](auto J) {
            constexpr int j = decltype(J)::value;
            pm[j] = a.PiG[eidx<IX>(j, N, idx)];
        });
    };
    if constexpr (kPacked<R>) {
        if constexpr (kEarlyH) {
            load_h_pig();
            asm volatile("" ::: "memory");
        }
        const float4 f0 = a.FB[idx];
        u[0] = f0.x; u[1] = f0.y; u[2] = f0.z;
        phi = f0.w;
        P = a.F_new[idx].w;
        auto at = [&](auto I, int s) { return a.FB[nb.at<L, decltype(I)::value>(s)]; };
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
        if constexpr (!kEarlyH) load_h_pig();
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            hp[i] = C::template dec_h<i>(hraw[i]);
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

// S0 + S2..S5 at site idx.  With FP32 arithmetic and whole warps (a.vote),
// a warp whose sites have no solid or outside neighbour runs the code
// without bounce-back selections (the same arithmetic: with no mask bit set
// both give the same bits).  Not in the even step of the in-place store:
// there the two copies of the code need more registers than it has.
template <class L, class R, class C, bool HAS_MASK, int MODE, class IX>
__device__ __forceinline__ void collide_site(const SplitArgs<R, typename C::S> &a, const int idx)
{
    uint32_t m = 0;
    if constexpr (HAS_MASK) {
        m = a.mask[idx];
        if constexpr (kPacked<R> && MODE != kAAEven) {
            if (a.vote && !__any_sync(0xffffffffu, m != 0u)) {
                collide_site_impl<L, R, C, false, MODE, IX>(a, idx, 0u);
                return;
            }
        }
    }
    collide_site_impl<L, R, C, HAS_MASK, MODE, IX>(a, idx, m);
}

// The u^{n+1} reading of the pressure formula's omega-term (coupling_unew):
// omega rho_ref sum_i w_i c_i . u(x - c_i) taken with the new velocity,
// whose neighbours the moments launch does not have yet.  The moments leave
// the term out of P^{n+1}; this adds it at a fluid site before the
// collision reads P^{n+1}.  FP32 arithmetic: sum_i w_i c_i . u(x - c_i) =
// -T div u with the divergence of the collision's pair stencil over the
// packed (u, phi) words (u = 0 at a solid neighbour); FP64: the sum over the
// directions in the canonical order of the moments' own sum.
template <class L, class R, class C, bool HAS_MASK, class IX>
__device__ __forceinline__ void coupling_site(const SplitArgs<R, typename C::S> &a, const int idx)
{
    constexpr int D = L::D, Q = L::Q;
    uint32_t m = 0;
    if constexpr (HAS_MASK) m = a.mask[idx];
    if (m & kSolidBit) return;
    const IX N = (IX)a.N;
    const Nbr32 nb(idx, a.nx, a.ny, D == 3 ? a.nz : 1);
    R phi, swcu = R(0);
    if constexpr (kPacked<R>) {
        float gphi[3], lphi, gu[3][3];
        phi = a.FB[idx].w;
        auto at = [&](auto I, int s) { return a.FB[nb.at<L, decltype(I)::value>(s)]; };
        if (m == 0u) stencil_packed<L, false>(at, m, phi, gphi, lphi, gu);
        else stencil_packed<L, true>(at, m, phi, gphi, lphi, gu);
        float div = gu[0][0] + gu[1][1];
        if constexpr (D == 3) div = div + gu[2][2];
        swcu = div * float(-1.0 / 3.0);
    } else {
        phi = a.phi[idx];
        static_for<1, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (!(HAS_MASK && ((m >> i) & 1u))) {
                const int src = nb.at<L, i>(-1);
                R un[3];
                static_for<0, 3>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    if constexpr (ax < D && L::c(i, ax) != 0) un[ax] = a.u_new[eidx<IX>(ax, N, src)];
                    else un[ax] = R(0);
                });
                swcu = swcu + R(L::w(i)) * dot_c<L, i>(un);
            }
        });
    }
    const R phihat = a.k.clamp ? clamp01(phi) : phi;
    const R rho = a.k.rho_a + phihat * a.k.drho;
    const R omega = (rho - a.k.rho_a) / a.k.drho * a.k.om1;
    if constexpr (kPacked<R>) {
        float4 *w = a.F_new + idx;
        w->w = w->w + omega * a.k.rho_a * swcu;
    } else {
        a.P_new[idx] = a.P_new[idx] + omega * a.k.rho_a * swcu;
    }
}

template <class L, class R, class C, bool HAS_MASK, class IX>
__global__ void __launch_bounds__(kSplitThreads) coupling_kernel(const SplitArgs<R, typename C::S> a)
{
    const long long idx = (long long)blockIdx.x * kSplitThreads + threadIdx.x;
    if (idx < a.N) coupling_site<L, R, C, HAS_MASK, IX>(a, (int)idx);
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
