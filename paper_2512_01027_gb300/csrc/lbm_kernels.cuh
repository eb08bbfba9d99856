// Kernels of the coupled LB step: fused step, initialisation, readout,
// FP64 reductions.  Templated on lattice L, compute type R and population
// storage codec C (identity for FP64/FP32, scaled 16-bit deviations for the
// reduced-storage forms).
//
// Fused step (one launch per time step, ping-pong buffers src -> dst):
//   A CTA owns an interior tile of TX x TY sites in (x, y) and marches in z
//   over a chunk [zb, ze).  Its threads cover the tile plus a one-site halo
//   (SX = TX + 2, SY = TY + 2).  For each plane the threads pull the
//   populations of their site and compute the moments (phi, u^{n+1}, and for
//   interior sites P^{n+1}) into a three-plane ring in shared memory; the
//   interior sites also park their pulled populations in shared memory.  One
//   plane later, when the ring holds phi and u on planes z-1, z, z+1, the
//   interior threads evaluate the stencils from the ring, collide both
//   populations and store them.  The halo moments are recomputed by the
//   neighbouring CTA's threads instead of exchanged, so one launch is one
//   time step: every population is read from HBM once and written once
//   (halo re-reads hit L2).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "lbm_lattice.cuh"
#include "lbm_site.cuh"

namespace lbm {

constexpr uint32_t kSolidBit = 1u << 31;

// ---------------------------------------------------------------------------
// Storage codecs

// Identity storage (FP64 / FP32): populations stored as computed.  PD: the
// rest population of g is held as g_0 - P^n/(rho_ref T) (reduced-precision
// paths, see s1_pressure); view_g restores g_0 for callers reading the state.
template <class R, bool PD>
struct CodecId {
    using S = R;
    static constexpr bool kPdev = PD;
    static constexpr bool kGodd = false;
    static constexpr bool kRound16 = false;
    template <int i>
    __device__ __forceinline__ static R dec_h(S v) { return v; }
    template <int i>
    __device__ __forceinline__ static S enc_h(R v) { return v; }
    template <int i>
    __device__ __forceinline__ static S enc_h_sr(R v, uint32_t) { return v; }
    template <int i>
    __device__ __forceinline__ static R dec_g(S v) { return v; }
    template <int i>
    __device__ __forceinline__ static S enc_g(R v) { return v; }
    template <int i>
    __device__ __forceinline__ static R view_g(S v, R P, R cP)
    {
        if constexpr (PD && i == 0) return v + P * cP;
        else return v;
    }
};

// 16-bit storage of scaled populations, FP32 arithmetic.  h_i is held as
// t = h_i / w_i (bulk heavy phase t = 1, bulk light phase t = 0, both exact).
// Near t = 0 a 16-bit float is much finer than near 1, and that is where it
// matters: in the light phase rho = rho_a + phi (rho_w - rho_a) with rho_a
// ~ 1e-3, so an error of 1e-4 in phi there is a 10 % error in rho and in
// everything divided by it.  g_i is held as g_i S / w_i (g_i is already a
// deviation: g_eq_i = Gamma_i - w_i + ...), with S = 1024 for FP16 to keep
// small values out of the subnormal range and S = 1 for BF16; the rest
// population of g is held without its P^n / (rho_ref T) part (kPdev).
template <class H>
struct Codec16 {
    using S = H;
    static constexpr bool kPdev = true;
    static constexpr bool kHalf = std::is_same<H, __half>::value;
    static constexpr float kScale = kHalf ? 1024.0f : 1.0f;
    __device__ __forceinline__ static float to_f(H v)
    {
        if constexpr (kHalf) return __half2float(v);
        else return __bfloat162float(v);
    }
    __device__ __forceinline__ static H from_f(float v)
    {
        if constexpr (kHalf) return __float2half_rn(v);
        else return __float2bfloat16_rn(v);
    }
    // Unbiased (stochastic) rounding: v goes to the 16-bit value above with
    // probability (v - below) / (above - below), decided by r (uniform 32 bits).
    // A v within FP32 noise (2^-20 relative) of a 16-bit value is that value:
    // exact states (a fluid at rest) stay exact.
    __device__ __forceinline__ static H from_f_sr(float v, uint32_t r)
    {
        const H n = from_f(v);
        if (fabsf(v - to_f(n)) <= fabsf(v) * (1.0f / 1048576.0f)) return n;
        H lo, hi;
        if constexpr (kHalf) {
            lo = __float2half_rd(v);
            hi = __float2half_ru(v);
        } else {
            lo = __float2bfloat16_rd(v);
            hi = __float2bfloat16_ru(v);
        }
        const float flo = to_f(lo), fhi = to_f(hi);
        if (!(fhi > flo)) return lo;
        const float p = (v - flo) / (fhi - flo);
        return (float)(r >> 8) * (1.0f / 16777216.0f) < p ? hi : lo;
    }
};

// 32-bit mixer (Wellons' "lowbias32") of a counter: the random bits of the
// stochastic rounding, a function of (site, step) only.
__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <class L, class H>
struct CodecDev {
    using S = H;
    using B = Codec16<H>;
    static constexpr bool kPdev = true;
    static constexpr bool kRound16 = true;
    // BF16 (8 significant bits): g is stored without its first-order odd part
    // w_i c_i . V_g (V_g per site, kept beside the populations in FP32), so
    // what is rounded to 16 bits is the small remainder (see lbm_split.cuh).
    // FP16 meets the velocity bound without it and keeps the bandwidth.
    static constexpr bool kGodd = !B::kHalf;
    template <int i>
    __device__ __forceinline__ static float dec_h(S v)
    {
        constexpr float w = (float)L::w(i);
        return B::to_f(v) * w;
    }
    template <int i>
    __device__ __forceinline__ static S enc_h(float h)
    {
        constexpr float iw = (float)(1.0 / L::w(i));
        return B::from_f(h * iw);
    }
    template <int i>
    __device__ __forceinline__ static S enc_h_sr(float h, uint32_t r)
    {
        constexpr float iw = (float)(1.0 / L::w(i));
        return B::from_f_sr(h * iw, r);
    }
    template <int i>
    __device__ __forceinline__ static float dec_g(S v)
    {
        constexpr float ws = (float)(L::w(i) / (double)B::kScale);
        return B::to_f(v) * ws;
    }
    template <int i>
    __device__ __forceinline__ static S enc_g(float g)
    {
        constexpr float sw = (float)((double)B::kScale / L::w(i));
        return B::from_f(g * sw);
    }
    template <int i>
    __device__ __forceinline__ static float view_g(S v, float P, float cP)
    {
        if constexpr (i == 0) return dec_g<0>(v) + P * cP;
        else return dec_g<i>(v);
    }
};

// 16-bit storage: the rounding of the moving populations h_i (i != 0) is
// taken up by the rest population before it is rounded in turn, so the
// stored sum_i h_i of a site (its phi) carries one rounding instead of Q.
// Without it, a liquid slightly above phi = 1 rounds down in every
// direction at every step and the phase mass drifts.
template <class L, class C, class R>
__device__ __forceinline__ void compensate_h(R *hs)
{
    if constexpr (C::kRound16) {
        R e = R(0);
        static_for<1, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            e = e + (C::template dec_h<i>(C::template enc_h<i>(hs[i])) - hs[i]);
        });
        hs[0] = hs[0] - e;
    }
}

// cp.async helpers (LDGSTS: global -> shared without a register round trip)
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Kernel arguments

template <class R, class S>
struct StepArgs {
    const S *src_h;
    const S *src_g;
    S *dst_h;
    S *dst_g;
    const R *P_old;
    R *P_new;
    const R *u_old;      // [D][N]
    R *u_new;            // [D][N]
    const uint32_t *mask;  // [N] or nullptr
    int *err;
    int nx, ny, nz;
    int per_x, per_y, per_z;
    int zchunk;
    long long N;
    SiteConsts<R> k;
};

__device__ __forceinline__ int wrapc(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

enum StreamMode { kPingPong = 0, kAAEven = 1, kAAOdd = 2 };

template <class R, class S>
struct SplitArgs {
    const S *src_h, *src_g;   // populations read (ping-pong source, or the single AA store)
    S *dst_h, *dst_g;         // populations written (ping-pong destination, or the AA store)
    const R *P_old, *u_old;   // P^n, u^n [D][N]
    R *P_new, *u_new;         // P^{n+1}, u^{n+1} [D][N]
    R *phi;                   // phi^{n+1} [N]
    const float4 *F_old;      // packed (u^n, P^n) per site, FP32 arithmetic only (else NULL)
    float4 *F_new;            // packed (u^{n+1}, P^{n+1})
    unsigned seed;            // steps taken before this one (stream of the stochastic rounding)
    float4 *FB;               // packed (u^{n+1}, phi^{n+1})
    float *PiG;               // sum_i c_ia c_ib g_i of the pulled g, [3 or 6][N]
    const float4 *G_old;      // BF16 storage: odd part V_g of g* of the current state (see lbm_split.cuh)
    float4 *G_new;            // ... of the state being made
    const uint32_t *mask;
    int *err;
    int nx, ny, nz;
    long long N;
    int vote;                 // 1: the launch hands each warp to the per-site code with all 32 lanes,
                              // so the site code may take a warp vote
    SiteConsts<R> k;
};

// (u, P) of one site packed in a 16-byte word (z component 0 in 2D): the
// split kernels read a neighbour's velocity and pressure with one load.
template <int D>
__global__ void __launch_bounds__(256) pack_kernel(const float *__restrict__ P, const float *__restrict__ u,
                                                   float4 *__restrict__ F, long long N)
{
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    F[x] = make_float4(u[x], u[N + x], D == 3 ? u[2 * N + x] : 0.f, P[x]);
}

// The planes P, u[D] of the fluid sites from the packed words (solid sites
// hold no state and keep their values).
template <int D>
__global__ void __launch_bounds__(256) unpack_kernel(const float4 *__restrict__ F, const uint32_t *__restrict__ mask,
                                                     float *__restrict__ P, float *__restrict__ u, long long N)
{
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    if (mask && (mask[x] & kSolidBit)) return;
    const float4 f = F[x];
    P[x] = f.w;
    u[x] = f.x;
    u[N + x] = f.y;
    if (D == 3) u[2 * N + x] = f.z;
}

// Site coordinates and wrapped neighbour offsets: site of x + s c with
// s c in {-1, 0, 1} per axis is xo[1 + sc_x] + yo[1 + sc_y] + zo[1 + sc_z].
struct Nbr {
    long long xo[3], yo[3], zo[3];
    __device__ __forceinline__ Nbr(long long idx, int nx, int ny, int nz)
    {
        const int x = (int)(idx % nx);
        const int y = (int)((idx / nx) % ny);
        const int z = (int)(idx / ((long long)nx * ny));
        const long long nxy = (long long)nx * ny;
        xo[0] = wrapc(x - 1, nx); xo[1] = x; xo[2] = wrapc(x + 1, nx);
        yo[0] = (long long)wrapc(y - 1, ny) * nx; yo[1] = (long long)y * nx; yo[2] = (long long)wrapc(y + 1, ny) * nx;
        zo[0] = (long long)wrapc(z - 1, nz) * nxy; zo[1] = (long long)z * nxy; zo[2] = (long long)wrapc(z + 1, nz) * nxy;
    }
    // site x + s c_i
    template <class L, int i>
    __device__ __forceinline__ long long at(int s) const
    {
        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        if (s > 0) return xo[1 + cx] + yo[1 + cy] + zo[1 + cz];
        return xo[1 - cx] + yo[1 - cy] + zo[1 - cz];
    }
};

// Post-collision f*_i(x) location after initialisation / an even AA step
// (parity 0) or after an odd AA step (parity 1).
template <class L, int i>
__device__ __forceinline__ long long aa_state_off(const Nbr &nb, long long idx, long long N, uint32_t m, bool has_mask,
                                                  int parity)
{
    if constexpr (i == 0) {
        return idx;
    } else {
        if (parity == 0) return (long long)opp(i) * N + idx;
        const bool bb = has_mask && ((m >> opp(i)) & 1u);
        return bb ? (long long)opp(i) * N + idx : (long long)i * N + nb.at<L, i>(1);
    }
}


template <class L>
struct Tile {
    static constexpr int SX = 32;
    static constexpr int SY = 8;
    static constexpr int TX = SX - 2;
    static constexpr int TY = SY - 2;
    static constexpr int TI = TX * TY;
    static constexpr int RING = (L::D == 3) ? 3 : 1;
    static constexpr int STASH = (L::D == 3) ? 2 : 1;
    static constexpr int NT = SX * SY;
};

template <class L, class R>
__host__ __device__ constexpr size_t step_smem_bytes()
{
    using Tl = Tile<L>;
    return sizeof(R) * (size_t)(Tl::RING * Tl::SX * Tl::SY * (1 + L::D)         // ring phi, u
                                + Tl::STASH * Tl::TI * (2 * L::Q + 3))          // stash hp, gp, P, rho, phihat
           + sizeof(uint32_t) * (size_t)(Tl::STASH * Tl::TI);                  // stash mask
}

// ---------------------------------------------------------------------------
// Fused step kernel

template <class L, class R, class C, bool HAS_MASK>
__global__ void __launch_bounds__(Tile<L>::NT)
step_kernel(const StepArgs<R, typename C::S> a)
{
    using S = typename C::S;
    using Tl = Tile<L>;
    constexpr int D = L::D, Q = L::Q;
    constexpr int SX = Tl::SX, SY = Tl::SY, TX = Tl::TX, TY = Tl::TY, TI = Tl::TI;
    constexpr int PL = SX * SY;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *ring_phi = reinterpret_cast<R *>(smem_raw);
    R *ring_u = ring_phi + Tl::RING * PL;
    R *st_h = ring_u + Tl::RING * D * PL;
    R *st_g = st_h + Tl::STASH * Q * TI;
    R *st_P = st_g + Tl::STASH * Q * TI;
    R *st_rho = st_P + Tl::STASH * TI;
    R *st_ph = st_rho + Tl::STASH * TI;
    uint32_t *st_m = reinterpret_cast<uint32_t *>(st_ph + Tl::STASH * TI);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
    const int xs = X0 - 1 + tx, ys = Y0 - 1 + ty;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long N = a.N;
    const int zb = (D == 3) ? blockIdx.z * a.zchunk : 0;
    const int ze = (D == 3) ? min(nz, zb + a.zchunk) : 1;
    const bool in_tile = (tx >= 1 && tx <= TX && ty >= 1 && ty <= TY && xs < nx && ys < ny);
    const int ti = (ty - 1) * TX + (tx - 1);

    // (x, y) of this thread's S1 site, wrapped; validity in x, y
    bool xy_ok = true;
    int xw = xs, yw = ys;
    if (xs < 0 || xs >= nx) { if (a.per_x) xw = wrapc(xs, nx); else xy_ok = false; }
    if (ys < 0 || ys >= ny) { if (a.per_y) yw = wrapc(ys, ny); else xy_ok = false; }
    // source offsets x - c, c in {-1, 0, 1}: xo[1 - c]
    int xo[3], yo[3];
    xo[0] = wrapc(xw - 1, nx); xo[1] = xw; xo[2] = wrapc(xw + 1, nx);
    yo[0] = wrapc(yw - 1, ny) * nx; yo[1] = yw * nx; yo[2] = wrapc(yw + 1, ny) * nx;

    const int z_first = (D == 3) ? zb - 1 : 0;
    const int z_last = (D == 3) ? ze : 0;
    for (int zz = z_first; zz <= z_last; ++zz) {
        // ---------------- S0 + S1 on plane zz ----------------
        {
            bool ok = xy_ok;
            int zw = zz;
            if (D == 3 && (zz < 0 || zz >= nz)) { if (a.per_z) zw = wrapc(zz, nz); else ok = false; }
            const bool interior = in_tile && zz >= zb && zz < ze;
            if (ok) {
                const long long plane = (long long)zw * nx * ny;
                const long long idx = plane + yo[1] + xo[1];
                uint32_t m = 0;
                if constexpr (HAS_MASK) m = a.mask[idx];
                if (!(m & kSolidBit)) {
                    long long zo[3];
                    if constexpr (D == 3) {
                        zo[0] = (long long)wrapc(zw - 1, nz) * nx * ny;
                        zo[1] = plane;
                        zo[2] = (long long)wrapc(zw + 1, nz) * nx * ny;
                    } else {
                        zo[0] = zo[1] = zo[2] = 0;
                    }
                    R hp[Q], gp[Q], Pn[Q], K[Q];
                    const R P0 = a.P_old[idx];
                    R sum_wcu = R(0);
                    static_for<0, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                        if constexpr (i == 0) {
                            hp[0] = C::template dec_h<0>(a.src_h[idx]);
                            gp[0] = C::template dec_g<0>(a.src_g[idx]);
                            Pn[0] = P0;
                        } else {
                            const long long src = zo[1 - cz] + yo[1 - cy] + xo[1 - cx];
                            const bool solid_src = HAS_MASK && ((m >> i) & 1u);
                            if (solid_src) {
                                // halfway bounce-back: h_i(x) = h*_{-i}(x)
                                hp[i] = C::template dec_h<opp(i)>(a.src_h[(long long)opp(i) * N + idx]);
                                gp[i] = C::template dec_g<opp(i)>(a.src_g[(long long)opp(i) * N + idx]);
                                Pn[i] = P0;
                            } else {
                                hp[i] = C::template dec_h<i>(a.src_h[(long long)i * N + src]);
                                gp[i] = C::template dec_g<i>(a.src_g[(long long)i * N + src]);
                                Pn[i] = a.P_old[src];
                                if (interior) {
                                    R un[3];
                                    static_for<0, D>([&](auto A) {
                                        constexpr int ax = decltype(A)::value;
                                        if constexpr (L::c(i, ax) != 0) un[ax] = a.u_old[(long long)ax * N + src];
                                        else un[ax] = R(0);
                                    });
                                    if constexpr (D == 2) un[2] = R(0);
                                    sum_wcu = sum_wcu + R(L::w(i)) * dot_c<L, i>(un);
                                }
                            }
                        }
                    });
                    R phi, phihat, rho, u[3], sumg, sumK;
                    if constexpr (kPairForms<R>) s1_pairs<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, sumg, sumK);
                    else s1_moments<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, K);
                    const int rs = (D == 3) ? (zz + 3) % 3 : 0;
                    ring_phi[rs * PL + ty * SX + tx] = phi;
                    static_for<0, D>([&](auto A) {
                        constexpr int ax = decltype(A)::value;
                        ring_u[(rs * D + ax) * PL + ty * SX + tx] = u[ax];
                    });
                    if (interior) {
                        R Pnew;
                        if constexpr (kPairForms<R>) Pnew = s1_pressure_pairs<R, C::kPdev>(a.k, rho, sumg, sumK, sum_wcu, P0);
                        else Pnew = s1_pressure<L, R, C::kPdev>(a.k, gp, K, rho, sum_wcu, P0);
                        const int ss = (D == 3) ? (zz & 1) : 0;
                        static_for<0, Q>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            st_h[(ss * Q + i) * TI + ti] = hp[i];
                            st_g[(ss * Q + i) * TI + ti] = gp[i];
                        });
                        st_P[ss * TI + ti] = Pnew;
                        st_rho[ss * TI + ti] = rho;
                        st_ph[ss * TI + ti] = phihat;
                        st_m[ss * TI + ti] = m;
                    }
                } else if (interior) {
                    const int ss = (D == 3) ? (zz & 1) : 0;
                    st_m[ss * TI + ti] = m;
                }
            } else if (interior) {
                const int ss = (D == 3) ? (zz & 1) : 0;
                st_m[ss * TI + ti] = kSolidBit;
            }
        }
        __syncthreads();
        // ---------------- S2..S5 on plane zc ----------------
        const int zc = (D == 3) ? zz - 1 : zz;
        if (zc >= zb && in_tile) {
            const int ss = (D == 3) ? (zc & 1) : 0;
            const uint32_t m = st_m[ss * TI + ti];
            if (!(m & kSolidBit)) {
                const int r0 = (D == 3) ? (zc + 3) % 3 : 0;
                const int rm = (D == 3) ? (zc + 2) % 3 : 0;
                const int rp = (D == 3) ? (zc + 4) % 3 : 0;
                const int c0 = ty * SX + tx;
                auto ring_at = [&](const R *base, int plane_stride, auto I, int s) -> R {
                    constexpr int i = decltype(I)::value;
                    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                    const int r = (cz == 0) ? r0 : ((cz * s > 0) ? rp : rm);
                    return base[r * plane_stride + c0 + s * (cy * SX + cx)];
                };
                const R phi = ring_phi[r0 * PL + c0];
                R gphi[3], lphi;
                stencil_any<L, R>([&](auto I, int s) { return ring_at(ring_phi, PL, I, s); }, m, phi, phi, gphi, lphi);
                R u[3], gu[3][3];
                u[2] = R(0);
                gu[0][2] = gu[1][2] = gu[2][0] = gu[2][1] = gu[2][2] = R(0);
                static_for<0, D>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    const R *base = ring_u + ax * PL;
                    u[ax] = base[r0 * D * PL + c0];
                    R lap_unused;
                    stencil_any<L, R>([&](auto I, int s) { return ring_at(base, D * PL, I, s); }, m, u[ax], R(0),
                                  gu[ax], lap_unused);
                });
                const R P = st_P[ss * TI + ti];
                const R rho = st_rho[ss * TI + ti];
                const R phihat = st_ph[ss * TI + ti];
                R hp[Q], gp[Q], hs[Q], gs[Q];
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    hp[i] = st_h[(ss * Q + i) * TI + ti];
                    gp[i] = st_g[(ss * Q + i) * TI + ti];
                });
                collide<L, R, false, C::kPdev>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, gp, hs, gs);
                compensate_h<L, C>(hs);
                const long long idx = (long long)zc * nx * ny + (long long)ys * nx + xs;
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    a.dst_h[(long long)i * N + idx] = C::template enc_h<i>(hs[i]);
                    a.dst_g[(long long)i * N + idx] = C::template enc_g<i>(gs[i]);
                });
                a.P_new[idx] = P;
                static_for<0, D>([&](auto A) {
                    constexpr int ax = decltype(A)::value;
                    a.u_new[(long long)ax * N + idx] = u[ax];
                });
                if (!(isfinite(phi) && isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2])))
                    atomicOr(a.err, 1);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Initialisation: populations at equilibrium from (phi0, P0, u0) (double).

template <class R, class S>
struct InitArgs {
    const double *phi0, *P0, *u0;  // u0: [3][N]
    S *h, *g;
    R *P, *u;                      // u: [D][N]
    const uint32_t *mask;
    int nx, ny, nz;
    long long N;
    int aa;                        // 1: in-place AA store (f*_i(x) goes to slot -i of x)
    SiteConsts<R> k;
};

template <class L, class R, class C, bool HAS_MASK>
__global__ void __launch_bounds__(128) init_kernel(const InitArgs<R, typename C::S> a)
{
    constexpr int D = L::D, Q = L::Q;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N) return;
    uint32_t m = 0;
    if constexpr (HAS_MASK) m = a.mask[idx];
    if (m & kSolidBit) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x = (int)(idx % nx);
    const int y = (int)((idx / nx) % ny);
    const int z = (int)(idx / ((long long)nx * ny));
    // neighbour x + s c_i (wrapped; a solid/outside neighbour is flagged by the mask)
    auto nb = [&](auto I, int s) -> long long {
        constexpr int i = decltype(I)::value;
        const int xx = wrapc(x + s * L::c(i, 0), nx);
        const int yy = wrapc(y + s * L::c(i, 1), ny);
        const int zz = (D == 3) ? wrapc(z + s * L::c(i, 2), nz) : 0;
        return ((long long)zz * ny + yy) * nx + xx;
    };
    const R phi = R(a.phi0[idx]);
    const R phihat = a.k.clamp ? clamp01(phi) : phi;
    const R rho = a.k.rho_a + phihat * a.k.drho;
    R gphi[3], lphi;
    stencil_any<L, R>([&](auto I, int s) { return R(a.phi0[nb(I, s)]); }, m, phi, phi, gphi, lphi);
    R u[3], gu[3][3];
    u[2] = R(0);
    gu[0][2] = gu[1][2] = gu[2][0] = gu[2][1] = gu[2][2] = R(0);
    static_for<0, D>([&](auto A) {
        constexpr int ax = decltype(A)::value;
        const double *f = a.u0 + (long long)ax * a.N;
        u[ax] = R(f[idx]);
        R lap_unused;
        stencil_any<L, R>([&](auto I, int s) { return R(f[nb(I, s)]); }, m, u[ax], R(0), gu[ax], lap_unused);
    });
    const R P = R(a.P0[idx]);
    R hs[Q], gs[Q];
    collide<L, R, true, C::kPdev>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, nullptr, nullptr, hs, gs);
    compensate_h<L, C>(hs);
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const long long off = (long long)(a.aa ? opp(i) : i) * a.N + idx;
        a.h[off] = C::template enc_h<i>(hs[i]);
        a.g[off] = C::template enc_g<i>(gs[i]);
    });
    a.P[idx] = P;
    static_for<0, D>([&](auto A) {
        constexpr int ax = decltype(A)::value;
        a.u[(long long)ax * a.N + idx] = u[ax];
    });
}

// ---------------------------------------------------------------------------
// Readout: phi = sum_i h*_i, P, u as double (solid sites 0).

template <class R, class S>
struct ReadArgs {
    const S *h, *g;
    const R *P, *u;
    const uint32_t *mask;
    double *phi_out, *P_out, *u_out;   // u_out: [3][N]
    double *hpop_out, *gpop_out;       // optional decoded populations [Q][N]
    const float4 *G;                   // BF16 storage: deferred odd part of g* (added when read), or NULL
    long long N;
    R cP;
    int aa;                            // 0: ping-pong layout; 1 + parity: in-place AA layout
    int nx, ny, nz;
};

// The deferred odd part w_i c_i . V_g(x) of g*_i(x), 0 when nothing is deferred.
template <class L, int i, class RA>
__device__ __forceinline__ float g_deferred(const RA &a, long long idx)
{
    if constexpr (i == 0) {
        return 0.f;
    } else {
        if (!a.G) return 0.f;
        const float4 v4 = a.G[idx];
        const float v[3] = {v4.x, v4.y, v4.z};
        return float(L::w(i)) * dot_c<L, i>(v);
    }
}

// Offset of the post-collision f*_i(x) in the current state.
template <class L, int i, class RA>
__device__ __forceinline__ long long state_off(const RA &a, long long idx)
{
    if (a.aa == 0) return (long long)i * a.N + idx;
    const uint32_t m = a.mask ? a.mask[idx] : 0u;
    const Nbr nb(idx, a.nx, a.ny, L::D == 3 ? a.nz : 1);
    return aa_state_off<L, i>(nb, idx, a.N, m, a.mask != nullptr, a.aa - 1);
}

// Completes BF16 g populations stored without their odd part into g*:
// g*_i(x) = stored_i(x) + w_i c_i . V_g(x).
template <class L, class C>
__global__ void __launch_bounds__(128) fold_g_kernel(const ReadArgs<float, typename C::S> a, typename C::S *g,
                                                     const float4 *__restrict__ G)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N) return;
    if (a.mask && (a.mask[idx] & kSolidBit)) return;
    const float4 v4 = G[idx];
    const float v[3] = {v4.x, v4.y, v4.z};
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const long long off = state_off<L, i>(a, idx);
        const float gv = C::template dec_g<i>(g[off]);
        g[off] = C::template enc_g<i>(gv + float(L::w(i)) * dot_c<L, i>(v));
    });
}

template <class L, class R, class C, bool HAS_MASK>
__global__ void __launch_bounds__(256) read_kernel(const ReadArgs<R, typename C::S> a)
{
    constexpr int D = L::D, Q = L::Q;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.N) return;
    bool solid = false;
    if constexpr (HAS_MASK) solid = (a.mask[idx] & kSolidBit) != 0;
    const R P = solid ? R(0) : a.P[idx];
    if (a.phi_out) {
        R phi = R(0);
        if (!solid) {
            phi = C::template dec_h<0>(a.h[idx]);
            static_for<1, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                phi = phi + C::template dec_h<i>(a.h[state_off<L, i>(a, idx)]);
            });
        }
        a.phi_out[idx] = (double)phi;
    }
    if (a.P_out) a.P_out[idx] = (double)P;
    if (a.u_out) {
        static_for<0, 3>([&](auto A) {
            constexpr int ax = decltype(A)::value;
            double v = 0.0;
            if (ax < D && !solid) v = (double)a.u[(long long)(ax < D ? ax : 0) * a.N + idx];
            a.u_out[(long long)ax * a.N + idx] = v;
        });
    }
    if (a.hpop_out || a.gpop_out) {
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            if (a.hpop_out) a.hpop_out[(long long)i * a.N + idx] =
                solid ? 0.0 : (double)C::template dec_h<i>(a.h[state_off<L, i>(a, idx)]);
            if (a.gpop_out) a.gpop_out[(long long)i * a.N + idx] =
                solid ? 0.0
                      : (double)(C::template view_g<i>(a.g[state_off<L, i>(a, idx)], P, a.cP) +
                                 g_deferred<L, i>(a, idx));
        });
    }
}

// Gather of the state at chosen sites (decoded, double).
template <class L, class R, class C>
__global__ void __launch_bounds__(128) probe_kernel(const ReadArgs<R, typename C::S> a, const long long *sites, int n,
                                                    double *hp, double *gp, double *P, double *u)
{
    constexpr int D = L::D, Q = L::Q;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long idx = sites[j];
    if (idx < 0 || idx >= a.N) return;
    if (a.mask && (a.mask[idx] & kSolidBit)) {     // solid sites hold no state
        if (P) P[j] = 0.0;
        for (int ax = 0; ax < 3 && u; ++ax) u[(long long)j * 3 + ax] = 0.0;
        for (int i = 0; i < Q; ++i) {
            if (hp) hp[(long long)j * Q + i] = 0.0;
            if (gp) gp[(long long)j * Q + i] = 0.0;
        }
        return;
    }
    const R Ps = a.P[idx];
    if (P) P[j] = (double)Ps;
    if (u) {
        static_for<0, 3>([&](auto A) {
            constexpr int ax = decltype(A)::value;
            u[(long long)j * 3 + ax] = (ax < D) ? (double)a.u[(long long)(ax < D ? ax : 0) * a.N + idx] : 0.0;
        });
    }
    static_for<0, Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        if (hp) hp[(long long)j * Q + i] = (double)C::template dec_h<i>(a.h[state_off<L, i>(a, idx)]);
        if (gp)
            gp[(long long)j * Q + i] =
                (double)(C::template view_g<i>(a.g[state_off<L, i>(a, idx)], Ps, a.cP) + g_deferred<L, i>(a, idx));
    });
}

// ---------------------------------------------------------------------------
// FP64 reductions, deterministic two-pass: per-block partials, then one block
// sums the partials in a fixed order.

constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 1024;
constexpr int kRedVals = 5;

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh /* [NV][kRedThreads] */)
{
    const int t = threadIdx.x;
    for (int j = 0; j < NV; ++j) sh[j * kRedThreads + t] = v[j];
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int j = 0; j < NV; ++j) sh[j * kRedThreads + t] += sh[j * kRedThreads + t + s];
        __syncthreads();
    }
    for (int j = 0; j < NV; ++j) v[j] = sh[j * kRedThreads];
}

// sums: phi, rho u_x, rho u_y, rho u_z, fluid sites
template <class L, class R, class C, bool HAS_MASK>
__global__ void __launch_bounds__(kRedThreads) reduce_kernel(const ReadArgs<R, typename C::S> a, R rho_a, R drho,
                                                             int clamp, double *partials)
{
    constexpr int D = L::D, Q = L::Q;
    __shared__ double sh[kRedVals * kRedThreads];
    double v[kRedVals] = {0, 0, 0, 0, 0};
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.N;
         idx += (long long)gridDim.x * blockDim.x) {
        if constexpr (HAS_MASK)
            if (a.mask[idx] & kSolidBit) continue;
        double phi = 0.0;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            phi += (double)C::template dec_h<i>(a.h[state_off<L, i>(a, idx)]);
        });
        const double ph = clamp ? fmin(1.0, fmax(0.0, phi)) : phi;
        const double rho = (double)rho_a + ph * (double)drho;
        v[0] += phi;
        static_for<0, D>([&](auto A) {
            constexpr int ax = decltype(A)::value;
            v[1 + ax] += rho * (double)a.u[(long long)ax * a.N + idx];
        });
        v[4] += 1.0;
    }
    block_sum<kRedVals>(v, sh);
    if (threadIdx.x == 0)
        for (int j = 0; j < kRedVals; ++j) partials[(long long)blockIdx.x * kRedVals + j] = v[j];
}

// Laplace jump sums: P inside r_in, count inside, P outside r_out, count outside.
template <class R, bool HAS_MASK>
__global__ void __launch_bounds__(kRedThreads) pjump_kernel(const R *P, const uint32_t *mask, int nx, int ny, int nz,
                                                            long long N, double cx, double cy, double cz, double r_in,
                                                            double r_out, double *partials)
{
    __shared__ double sh[4 * kRedThreads];
    double v[4] = {0, 0, 0, 0};
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        if constexpr (HAS_MASK)
            if (mask[idx] & kSolidBit) continue;
        const int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((long long)nx * ny));
        double dx = fabs(x - cx), dy = fabs(y - cy), dz = fabs(z - cz);
        dx = fmin(dx, nx - dx);
        dy = fmin(dy, ny - dy);
        dz = fmin(dz, nz - dz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double p = (double)P[idx];
        if (r < r_in) { v[0] += p; v[1] += 1.0; }
        if (r > r_out) { v[2] += p; v[3] += 1.0; }
    }
    block_sum<4>(v, sh);
    if (threadIdx.x == 0)
        for (int j = 0; j < 4; ++j) partials[(long long)blockIdx.x * 4 + j] = v[j];
}

// Second pass: one block adds nblocks partial vectors of NV values in a fixed order.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) finish_kernel(const double *partials, int nblocks, double *out)
{
    __shared__ double sh[NV * kRedThreads];
    double v[NV];
    for (int j = 0; j < NV; ++j) v[j] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int j = 0; j < NV; ++j) v[j] += partials[(long long)b * NV + j];
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0)
        for (int j = 0; j < NV; ++j) out[j] = v[j];
}

}  // namespace lbm
