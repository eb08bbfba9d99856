// Fused step kernel with an asynchronous copy pipeline (3D lattices, 4-byte
// population storage).
//
// Same work decomposition as step_kernel (32 x 8 threads cover a 30 x 6
// interior tile plus its one-site halo and march in z; one launch is one
// time step), but the global loads run one plane ahead of the arithmetic:
// while the block computes the moments of plane z and collides plane z-1,
// every thread has already issued cp.async copies (global -> shared, no
// register round trip) of the pulled populations of its site on plane z+1,
// and the block has issued the copies of the P^n and u^n planes the moments
// of plane z+1 need.  Bounce-back is resolved when a copy is issued (a solid
// source is replaced by the site's own opposite population), so the shared
// population ring holds exactly the pulled populations S1 and the collision
// read.  Shared memory per block (FP32 D3Q27): populations 3 x 54 x 256 x 4 B
// = 166 KB, P^n / u^n rings 18 KB, moment ring 12 KB, interior scalars 4 KB.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

template <class L>
struct TileV2 {
    static constexpr int SX = 32, SY = 8;
    static constexpr int TX = SX - 2, TY = SY - 2, TI = TX * TY;
    static constexpr int PL = SX * SY;          // S1 sites per plane
    static constexpr int PX = SX + 2, PY = SY + 2, PPL = PX * PY;  // P^n region per plane
    static constexpr int NT = PL;
};

template <class L, class R, class S>
__host__ __device__ constexpr size_t step_v2_smem_bytes()
{
    using Tl = TileV2<L>;
    return sizeof(R) * (size_t)(4 * Tl::PPL + 4 * L::D * Tl::PL + 3 * (1 + L::D) * Tl::PL + 2 * 3 * Tl::TI) +
           sizeof(S) * (size_t)(3 * 2 * L::Q * Tl::PL);
}

template <class L, class R, class C, bool HAS_MASK>
__global__ void __launch_bounds__(TileV2<L>::NT, 1)
step_kernel_v2(const StepArgs<R, typename C::S> a)
{
    using S = typename C::S;
    using Tl = TileV2<L>;
    constexpr int D = L::D, Q = L::Q;
    static_assert(D == 3, "pipelined step kernel is for 3D lattices");
    static_assert(sizeof(S) == 4, "cp.async of 4-byte populations");
    constexpr int SX = Tl::SX, TX = Tl::TX, TY = Tl::TY, TI = Tl::TI, PL = Tl::PL;
    constexpr int PX = Tl::PX, PPL = Tl::PPL;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *pbuf = reinterpret_cast<R *>(smem_raw);     // [4][PPL]        P^n planes
    R *ubuf = pbuf + 4 * PPL;                      // [4][D][PL]      u^n planes
    R *ring = ubuf + 4 * D * PL;                   // [3][1+D][PL]    phi, u^{n+1}
    R *st = ring + 3 * (1 + D) * PL;               // [2][3][TI]      P^{n+1}, rho, phihat
    S *pop = reinterpret_cast<S *>(st + 2 * 3 * TI);  // [3][2Q][PL]  pulled h, g

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * SX + tx;
    const int X0 = blockIdx.x * TX, Y0 = blockIdx.y * TY;
    const int xs = X0 - 1 + tx, ys = Y0 - 1 + ty;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const long long N = a.N, nxy = (long long)nx * ny;
    const int zb = blockIdx.z * a.zchunk;
    const int ze = min(nz, zb + a.zchunk);
    const bool in_tile = (tx >= 1 && tx <= TX && ty >= 1 && ty <= TY && xs < nx && ys < ny);
    const int ti = (ty - 1) * TX + (tx - 1);

    bool xy_ok = true;
    int xw = xs, yw = ys;
    if (xs < 0 || xs >= nx) { if (a.per_x) xw = wrapc(xs, nx); else xy_ok = false; }
    if (ys < 0 || ys >= ny) { if (a.per_y) yw = wrapc(ys, ny); else xy_ok = false; }
    int xo[3], yo[3];
    xo[0] = wrapc(xw - 1, nx); xo[1] = xw; xo[2] = wrapc(xw + 1, nx);
    yo[0] = wrapc(yw - 1, ny) * nx; yo[1] = yw * nx; yo[2] = wrapc(yw + 1, ny) * nx;
    const int xy = yo[1] + xo[1];

    // my elements of the P^n region (origin X0 - 2, Y0 - 2): e = tid and tid + 256
    bool pe_ok[2];
    int pe_off[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int e = tid + r * PL;
        pe_ok[r] = e < PPL;
        pe_off[r] = 0;
        if (pe_ok[r]) {
            int gx = X0 - 2 + e % PX, gy = Y0 - 2 + e / PX;
            if (gx < 0 || gx >= nx) { if (a.per_x) gx = wrapc(gx, nx); else pe_ok[r] = false; }
            if (gy < 0 || gy >= ny) { if (a.per_y) gy = wrapc(gy, ny); else pe_ok[r] = false; }
            if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) pe_ok[r] = false;
            pe_off[r] = gy * nx + gx;
        }
    }

    // plane z -> wrapped plane, or -1 when outside a non-periodic edge
    auto zwrap = [&](int z) -> int {
        if (z >= 0 && z < nz) return z;
        if (!a.per_z) return -1;
        return wrapc(z, nz);
    };
    auto mask_at = [&](int z) -> uint32_t {
        const int zw = zwrap(z);
        if (!xy_ok || zw < 0) return kSolidBit;
        if constexpr (HAS_MASK) return a.mask[(long long)zw * nxy + xy];
        else return 0u;
    };
    auto slot3 = [](int z) { return (z + 3) % 3; };
    auto slot4 = [](int z) { return (z + 4) & 3; };

    // copies of the pulled populations of my site on plane zp (mask m)
    auto issue_pops = [&](int zp, uint32_t m) {
        if (m & kSolidBit) return;
        const int zw = zwrap(zp);
        const long long pl = (long long)zw * nxy;
        long long zo[3];
        zo[0] = (long long)wrapc(zw - 1, nz) * nxy;
        zo[1] = pl;
        zo[2] = (long long)wrapc(zw + 1, nz) * nxy;
        const long long idx = pl + xy;
        S *dst = pop + (size_t)slot3(zp) * 2 * Q * PL + tid;
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
            long long off;
            if constexpr (i == 0) {
                off = idx;
            } else {
                const bool bb = HAS_MASK && ((m >> i) & 1u);
                off = bb ? (long long)opp(i) * N + idx : (long long)i * N + zo[1 - cz] + yo[1 - cy] + xo[1 - cx];
            }
            cp_async4(dst + i * PL, a.src_h + off);
            cp_async4(dst + (Q + i) * PL, a.src_g + off);
        });
    };
    // copies of the P^n region and of my u^n site on plane zq
    auto issue_fields = [&](int zq) {
        const int zw = zwrap(zq);
        if (zw < 0) return;
        const long long pl = (long long)zw * nxy;
        const int sl = slot4(zq);
#pragma unroll
        for (int r = 0; r < 2; ++r)
            if (pe_ok[r]) cp_async4(pbuf + sl * PPL + tid + r * PL, a.P_old + pl + pe_off[r]);
        if (xy_ok) {
            static_for<0, D>([&](auto A) {
                constexpr int ax = decltype(A)::value;
                cp_async4(ubuf + (sl * D + ax) * PL + tid, a.u_old + (long long)ax * N + pl + xy);
            });
        }
    };

    // prologue: populations of plane zb-1 and the field planes zb-2 .. zb
    uint32_t m_cur = mask_at(zb - 1);      // mask of the plane whose S1 runs next
    uint32_t m_next = mask_at(zb);         // mask of the plane whose copies are issued next
    uint32_t m_prev = kSolidBit;           // mask of the plane collided next
    issue_pops(zb - 1, m_cur);
    issue_fields(zb - 2);
    issue_fields(zb - 1);
    issue_fields(zb);
    cp_async_commit();

    for (int zz = zb - 1; zz <= ze; ++zz) {
        cp_async_wait<0>();
        __syncthreads();
        // ---- issue the copies for plane zz+1 (consumed next iteration) ----
        uint32_t m_next2 = kSolidBit;
        if (zz + 1 <= ze) {
            issue_pops(zz + 1, m_next);
            issue_fields(zz + 2);
            if (zz + 2 <= ze) m_next2 = mask_at(zz + 2);
        }
        cp_async_commit();
        // ---- S1 on plane zz ----
        {
            const uint32_t m = m_cur;
            const bool interior = in_tile && zz >= zb && zz < ze;
            if (!(m & kSolidBit)) {
                const S *src = pop + (size_t)slot3(zz) * 2 * Q * PL + tid;
                const int s0 = slot4(zz), sm = slot4(zz - 1), sp = slot4(zz + 1);
                const int pc = (ty + 1) * PX + (tx + 1);
                const R P0 = pbuf[s0 * PPL + pc];
                R hp[Q], gp[Q], Pn[Q], K[Q];
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                    hp[i] = C::template dec_h<i>(src[i * PL]);
                    gp[i] = C::template dec_g<i>(src[(Q + i) * PL]);
                    if constexpr (i == 0) {
                        Pn[0] = P0;
                    } else {
                        const int sl = (cz == 0) ? s0 : (cz > 0 ? sm : sp);
                        const R v = pbuf[sl * PPL + pc - cy * PX - cx];
                        Pn[i] = (HAS_MASK && ((m >> i) & 1u)) ? P0 : v;
                    }
                });
                R phi, phihat, rho, u[3], sumg, sumK;
                if constexpr (kPairForms<R>) s1_pairs<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, sumg, sumK);
                else s1_moments<L, R>(a.k, hp, gp, Pn, P0, phi, phihat, rho, u, K);
                const int rs = slot3(zz);
                ring[(rs * (1 + D)) * PL + tid] = phi;
                ring[(rs * (1 + D) + 1) * PL + tid] = u[0];
                ring[(rs * (1 + D) + 2) * PL + tid] = u[1];
                ring[(rs * (1 + D) + 3) * PL + tid] = u[2];
                if (interior) {
                    R sum_wcu = R(0);
                    static_for<1, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                        if (!(HAS_MASK && ((m >> i) & 1u))) {
                            const int sl = (cz == 0) ? s0 : (cz > 0 ? sm : sp);
                            const R *ub = ubuf + sl * D * PL + tid - cy * SX - cx;
                            R un[3];
                            un[0] = (cx != 0) ? ub[0] : R(0);
                            un[1] = (cy != 0) ? ub[PL] : R(0);
                            un[2] = (cz != 0) ? ub[2 * PL] : R(0);
                            sum_wcu = sum_wcu + R(L::w(i)) * dot_c<L, i>(un);
                        }
                    });
                    R Pnew;
                    if constexpr (kPairForms<R>) Pnew = s1_pressure_pairs<R, C::kPdev>(a.k, rho, sumg, sumK, sum_wcu, P0);
                    else Pnew = s1_pressure<L, R, C::kPdev>(a.k, gp, K, rho, sum_wcu, P0);
                    const int ss = zz & 1;
                    st[(ss * 3 + 0) * TI + ti] = Pnew;
                    st[(ss * 3 + 1) * TI + ti] = rho;
                    st[(ss * 3 + 2) * TI + ti] = phihat;
                }
            }
        }
        __syncthreads();
        // ---- S2..S5 on plane zc = zz - 1 ----
        const int zc = zz - 1;
        if (zc >= zb && in_tile && !(m_prev & kSolidBit)) {
            const uint32_t m = m_prev;
            const int r0 = slot3(zc), rm = slot3(zc - 1), rp = slot3(zc + 1);
            constexpr int RS = (1 + D) * PL;
            auto ring_at = [&](int field, auto I, int s) -> R {
                constexpr int i = decltype(I)::value;
                constexpr int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
                const int r = (cz == 0) ? r0 : ((cz * s > 0) ? rp : rm);
                return ring[r * RS + field * PL + tid + s * (cy * SX + cx)];
            };
            const R phi = ring[r0 * RS + tid];
            R gphi[3], lphi;
            stencil_any<L, R>([&](auto I, int s) { return ring_at(0, I, s); }, m, phi, phi, gphi, lphi);
            R u[3], gu[3][3];
            static_for<0, 3>([&](auto A) {
                constexpr int ax = decltype(A)::value;
                u[ax] = ring[r0 * RS + (1 + ax) * PL + tid];
                R lap_unused;
                stencil_any<L, R>([&](auto I, int s) { return ring_at(1 + ax, I, s); }, m, u[ax], R(0), gu[ax],
                              lap_unused);
            });
            const int ss = zc & 1;
            const R P = st[(ss * 3 + 0) * TI + ti];
            const R rho = st[(ss * 3 + 1) * TI + ti];
            const R phihat = st[(ss * 3 + 2) * TI + ti];
            const S *src = pop + (size_t)slot3(zc) * 2 * Q * PL + tid;
            R hp[Q], gp[Q], hs[Q], gs[Q];
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                hp[i] = C::template dec_h<i>(src[i * PL]);
                gp[i] = C::template dec_g<i>(src[(Q + i) * PL]);
            });
            collide<L, R, false, C::kPdev>(a.k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, gp, hs, gs);
            compensate_h<L, C>(hs);
            const long long idx = (long long)zc * nxy + (long long)ys * nx + xs;
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                a.dst_h[(long long)i * N + idx] = C::template enc_h<i>(hs[i]);
                a.dst_g[(long long)i * N + idx] = C::template enc_g<i>(gs[i]);
            });
            a.P_new[idx] = P;
            a.u_new[idx] = u[0];
            a.u_new[N + idx] = u[1];
            a.u_new[2 * N + idx] = u[2];
            if (!(isfinite(phi) && isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2])))
                atomicOr(a.err, 1);
        }
        m_prev = m_cur;
        m_cur = m_next;
        m_next = m_next2;
    }
    cp_async_wait<0>();
}

}  // namespace lbm
