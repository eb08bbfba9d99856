// Per-site arithmetic of the coupled LB step (Otomo et al., Sec. II).
//
// Every formula is evaluated in one fixed order: the order the paper writes
// its terms, with T = 1/3 substituted exactly (1/T = 3, 1/(2T) = 3/2,
// 1/(2T^2) = 9/2, 2/T = 6, T/2 = 1/6), sums over directions in ascending
// direction index, and terms whose lattice coefficient c is 0 dropped (they
// only add +-0).  Built without FMA contraction (FP64 units) this reproduces,
// operation for operation, any FP64 evaluation that follows the same order;
// the method is not Lipschitz where |grad phi| -> 0 (the unit normal n) or
// lap phi -> 0 (the sign s of delta-theta), so FP64 results of two
// implementations only stay equal when their rounding is identical.
#pragma once

#include <type_traits>

#include "lbm_lattice.cuh"

namespace lbm {

// Run constants, precomputed on the host in double and converted to R.
template <class R>
struct SiteConsts {
    R rho_a;        // rho_air = rho_ref
    R drho;         // rho_w - rho_a
    R om1;          // omega_max - 1 = rho_w / rho_a - 1
    R rhoref_T;     // rho_ref * T
    R cP;           // 1 / (rho_ref T) = 3 / rho_a
    R tau_a;        // nu_a / T + 1/2
    R dtau;         // tau_w - tau_a
    R inv_tau_phi;  // 1 / (M / T + 1/2)
    R lambda_b;
    R M3;           // M / T
    R W;
    R eps;
    R phi_n, phi_m, D;
    R invW, invD;   // 1 / W, 1 / D (the FP32 forms multiply by them)
    R dt_pref;      // gamma M / (T W)
    R A_mu;         // 48 sigma / W
    R B_mu;         // 3 sigma W / 2
    R g[3];         // body acceleration
    int clamp;
    int full_trace;
    int coupling;   // 1: the omega-term of P takes u^{n+1} (added by the collision launch)
};

template <class R>
__device__ __forceinline__ R clamp01(R v)
{
    return fmin(R(1), fmax(R(0), v));
}

// First direction component with c != 0 (3 if none).
template <class L, int i>
__host__ __device__ constexpr int first_nz()
{
    return L::c(i, 0) ? 0 : (L::c(i, 1) ? 1 : (L::c(i, 2) ? 2 : 3));
}

// c_i . v = (c_0 v_0 + c_1 v_1) + c_2 v_2 with the zero terms dropped.
template <class L, int i, class R>
__device__ __forceinline__ R dot_c(const R *v)
{
    constexpr int f = first_nz<L, i>();
    if constexpr (f == 3) {
        return R(0);
    } else {
        R acc = (L::c(i, f) > 0) ? v[f] : -v[f];
        static_for<f + 1, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (L::c(i, a) > 0) acc = acc + v[a];
            else if constexpr (L::c(i, a) < 0) acc = acc - v[a];
        });
        return acc;
    }
}

// acc += t * c_ia  (c in {-1, 0, 1})
template <int ca, class R>
__device__ __forceinline__ void acc_c(R &acc, R t)
{
    if constexpr (ca > 0) acc = acc + t;
    else if constexpr (ca < 0) acc = acc - t;
}

// Gamma_i = w_i { 1 + c.u/T + (c.u)^2/(2T^2) - u^2/(2T) }   (Sec. II)
template <class L, int i, class R>
__device__ __forceinline__ R gamma_i(const R *u, R uu)
{
    const R cu = dot_c<L, i>(u);
    return R(L::w(i)) * (R(1) + R(3) * cu + R(4.5) * (cu * cu) - R(1.5) * uu);
}

// Gamma_i - w_i = w_i { c.u/T + (c.u)^2/(2T^2) - u^2/(2T) }, evaluated directly
// (the form in which Gamma_i enters g_eq; no cancellation against w_i).
template <class L, int i, class R>
__device__ __forceinline__ R gamma_dev_i(const R *u, R uu)
{
    const R cu = dot_c<L, i>(u);
    return R(L::w(i)) * (R(3) * cu + R(4.5) * (cu * cu) - R(1.5) * uu);
}

// Central-difference gradient and Laplacian (Sec. II, nearest neighbours):
//   d_a f = sum_i {f(x+c_i) - f(x-c_i)} c_ia w_i / (2T),  lap f = 2 sum_i {f(x+c_i) - f(x)} w_i / T
// at(i, s) returns f(x + s c_i); mask bit i set <=> x - c_i is solid/outside,
// where f takes the value fsol.
template <class L, class R, class At>
__device__ __forceinline__ void stencil(At &&at, uint32_t mask, R f0, R fsol, R (&grad)[3], R &lap)
{
    grad[0] = R(0); grad[1] = R(0); grad[2] = R(0);
    lap = R(0);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const R fp = ((mask >> opp(i)) & 1u) ? fsol : at(I, 1);
        const R fm = ((mask >> i) & 1u) ? fsol : at(I, -1);
        const R d = fp - fm;
        const R wi = R(L::w(i));
        static_for<0, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (L::c(i, a) != 0) acc_c<L::c(i, a)>(grad[a], d * wi);
        });
        lap = lap + (fp - f0) * wi;
    });
    grad[0] = grad[0] * R(1.5);
    grad[1] = grad[1] * R(1.5);
    grad[2] = grad[2] * R(1.5);
    lap = lap * R(6);
}

// ---------------------------------------------------------------------------
// Pair-summed forms for FP32 arithmetic.  Directions come in pairs (c, -c)
// at indices (2k-1, 2k); every sum over directions with an odd coefficient
// (a gradient, a first moment) or an even one (a Laplacian, a second moment)
// is evaluated once per pair.  Algebraically identical to the canonical
// forms above, in half the operations; the FP64 path keeps the canonical
// order (its results must reproduce the oracle bit for bit).

template <class R>
inline constexpr bool kPairForms = std::is_same<R, float>::value;

// Gradient and Laplacian of the stencil (Sec. II) per pair:
//   d_a f = (1/T) sum_pairs c_ia w_i {f(x+c_i) - f(x-c_i)}
//   lap f = (2/T) {sum_pairs w_i (f(x+c_i) + f(x-c_i)) - (1 - w_0) f(x)}
// MASKED = false: no solid/outside neighbour (mask == 0).
template <class L, class R, bool MASKED, class At>
__device__ __forceinline__ void stencil_pairs(At &&at, uint32_t mask, R f0, R fsol, R (&grad)[3], R &lap)
{
    grad[0] = R(0); grad[1] = R(0); grad[2] = R(0);
    R s = R(0);
    static_for<0, (L::Q - 1) / 2>([&](auto P) {
        constexpr int i = 2 * decltype(P)::value + 1;
        const auto I = std::integral_constant<int, i>{};
        R fp = at(I, 1), fm = at(I, -1);
        if constexpr (MASKED) {
            if ((mask >> (i + 1)) & 1u) fp = fsol;   // x + c_i = x - c_{-i}
            if ((mask >> i) & 1u) fm = fsol;
        }
        const R wi = R(L::w(i));
        const R d = (fp - fm) * wi;
        static_for<0, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (L::c(i, a) != 0) acc_c<L::c(i, a)>(grad[a], d);
        });
        s = s + (fp + fm) * wi;
    });
    grad[0] = grad[0] * R(3);
    grad[1] = grad[1] * R(3);
    grad[2] = grad[2] * R(3);
    lap = (s - R(1.0 - L::w(0)) * f0) * R(6);
}

// Gradient and Laplacian of phi and velocity gradient gu[a][b] = d_b u_a
// from packed (u, phi) words, per pair as in stencil_pairs.  A solid or
// outside neighbour contributes phi = phi(x) and u = 0.
template <class L, bool MASKED, class At>
__device__ __forceinline__ void stencil_packed(At &&at, uint32_t mask, float phi0, float (&gphi)[3], float &lphi,
                                               float (&gu)[3][3])
{
    static_for<0, 3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        gu[a][0] = 0.f; gu[a][1] = 0.f; gu[a][2] = 0.f;
        gphi[a] = 0.f;
    });
    float sphi = 0.f;
    static_for<0, (L::Q - 1) / 2>([&](auto Pr) {
        constexpr int i = 2 * decltype(Pr)::value + 1;
        const auto I = std::integral_constant<int, i>{};
        float4 fp = at(I, 1), fm = at(I, -1);
        if constexpr (MASKED) {
            if ((mask >> (i + 1)) & 1u) fp = make_float4(0.f, 0.f, 0.f, phi0);
            if ((mask >> i) & 1u) fm = make_float4(0.f, 0.f, 0.f, phi0);
        }
        const float wi = float(L::w(i));
        const float d[4] = {(fp.x - fm.x) * wi, (fp.y - fm.y) * wi, (fp.z - fm.z) * wi, (fp.w - fm.w) * wi};
        static_for<0, 3>([&](auto B) {
            constexpr int b = decltype(B)::value;
            if constexpr (L::c(i, b) != 0) {
                acc_c<L::c(i, b)>(gphi[b], d[3]);
                static_for<0, L::D>([&](auto Ax) {
                    constexpr int ax = decltype(Ax)::value;
                    acc_c<L::c(i, b)>(gu[ax][b], d[ax]);
                });
            }
        });
        sphi = sphi + (fp.w + fm.w) * wi;
    });
    static_for<0, 3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        gu[a][0] = gu[a][0] * 3.f; gu[a][1] = gu[a][1] * 3.f; gu[a][2] = gu[a][2] * 3.f;
        gphi[a] = gphi[a] * 3.f;
    });
    lphi = (sphi - float(1.0 - L::w(0)) * phi0) * 6.f;
}

// Stencil dispatch: pair-summed for FP32 (with a branch for sites without a
// solid/outside neighbour), canonical for FP64.
template <class L, class R, class At>
__device__ __forceinline__ void stencil_any(At &&at, uint32_t mask, R f0, R fsol, R (&grad)[3], R &lap)
{
    if constexpr (kPairForms<R>) {
        if (mask == 0u) stencil_pairs<L, R, false>(at, mask, f0, fsol, grad, lap);
        else stencil_pairs<L, R, true>(at, mask, f0, fsol, grad, lap);
    } else {
        stencil<L, R>(at, mask, f0, fsol, grad, lap);
    }
}

// Moments of one site (S1) per pair.  Outputs phi, phihat, rho, u^{n+1} and
// the sums the pressure needs: sumg = sum_i g_i, sumK = sum_i K_i.
// Pn: P^n(x - c_i), already replaced by P^n(x) for a solid source.
template <class L, class R>
__device__ __forceinline__ void s1_pairs(const SiteConsts<R> &k, const R *hp, const R *gp, const R *Pn, R P0,
                                         R &phi, R &phihat, R &rho, R (&u)[3], R &sumg, R &sumK)
{
    phi = hp[0];
    static_for<1, L::Q>([&](auto I) { phi = phi + hp[decltype(I)::value]; });
    phihat = k.clamp ? clamp01(phi) : phi;
    rho = k.rho_a + phihat * k.drho;
    const R kfac = R(3) / rho;                          // 1 / (T rho)
    // u = sum_i (g_i + K_i) c_i, K_i = w_i/(T rho) {P(x-c_i) - P(x)}: the
    // g differences and the weighted P differences are summed apart and
    // 1/(T rho) applied once, as the split form's moments launch does
    R ug[3] = {R(0), R(0), R(0)}, up[3] = {R(0), R(0), R(0)};
    sumg = gp[0];
    R swP = R(0);
    static_for<0, (L::Q - 1) / 2>([&](auto Pp) {
        constexpr int i = 2 * decltype(Pp)::value + 1;
        constexpr int io = i + 1;
        const R wi = R(L::w(i));
        const R dg = gp[i] - gp[io], dp = wi * (Pn[i] - Pn[io]);
        static_for<0, 3>([&](auto A) {
            constexpr int a = decltype(A)::value;
            if constexpr (L::c(i, a) != 0) {
                acc_c<L::c(i, a)>(ug[a], dg);
                acc_c<L::c(i, a)>(up[a], dp);
            }
        });
        sumg = sumg + (gp[i] + gp[io]);
        swP = swP + wi * (Pn[i] + Pn[io]);
    });
    static_for<0, 3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        u[a] = ug[a] + kfac * up[a];
    });
    sumK = kfac * (swP - R(1.0 - L::w(0)) * P0);
}

// Pressure from the pair sums (same formula as s1_pressure).
template <class R, bool PDEV>
__device__ __forceinline__ R s1_pressure_pairs(const SiteConsts<R> &k, R rho, R sumg, R sumK, R sum_wcu, R P0)
{
    const R omega = (rho - k.rho_a) / k.drho * k.om1;
    const R s = sumg + (R(1) + omega) * sumK;
    if constexpr (PDEV) return P0 + k.rhoref_T * s + omega * k.rho_a * sum_wcu;
    else return k.rhoref_T * s + omega * k.rho_a * sum_wcu;
}

// Moments of one site (S1).  hp, gp: pulled populations; Pn: P^n(x - c_i)
// (P^n(x) for a solid source); P0 = P^n(x).  Outputs phi, phihat, rho and
// u^{n+1} (components [0, D)).  Returns kfac = 1/(T rho) and leaves K_i in K.
template <class L, class R>
__device__ __forceinline__ void s1_moments(const SiteConsts<R> &k, const R *hp, const R *gp, const R *Pn,
                                           R P0, R &phi, R &phihat, R &rho, R (&u)[3], R *K)
{
    phi = hp[0];
    static_for<1, L::Q>([&](auto I) { phi = phi + hp[decltype(I)::value]; });
    phihat = k.clamp ? clamp01(phi) : phi;
    rho = k.rho_a + phihat * k.drho;
    const R kfac = R(3) / rho;                          // 1 / (T rho)
    u[0] = R(0); u[1] = R(0); u[2] = R(0);
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        // K_i = w_i / (T rho) { P(x - c_i) - P(x) }   (Eq. Kiterm)
        K[i] = R(L::w(i)) * kfac * (Pn[i] - P0);
        if constexpr (i > 0) {
            const R t = gp[i] + K[i];                   // u = sum_i (g_i + K_i) c_i
            static_for<0, 3>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (L::c(i, a) != 0) acc_c<L::c(i, a)>(u[a], t);
            });
        }
    });
}

// Pressure of one site (S1):
//   P = rho_ref T sum_i (g_i + (1 + omega) K_i) + omega rho_ref sum_i w_i (c_i . u^n)|_{x - c_i}
// sum_wcu = sum_i w_i (c_i . u^n(x - c_i)) accumulated by the caller.
// PDEV (reduced-precision paths): the rest population is held as
// g_0 - P^n / (rho_ref T), the part of g_eq_0 other than P^n / (rho_ref T);
// since rho_ref T * (1 / (rho_ref T)) = 1 the same P is P^n + rho_ref T (...),
// and P^n is carried exactly instead of through a number 1/(rho_ref T) times
// larger than P.
template <class L, class R, bool PDEV>
__device__ __forceinline__ R s1_pressure(const SiteConsts<R> &k, const R *gp, const R *K, R rho, R sum_wcu, R P0)
{
    // omega = (rho - rho_a) / (rho_w - rho_a) (omega_max - 1)
    const R omega = (rho - k.rho_a) / k.drho * k.om1;
    const R op1 = R(1) + omega;
    R s = gp[0];
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        s = s + (gp[i] + op1 * K[i]);
    });
    if constexpr (PDEV) return P0 + k.rhoref_T * s + omega * k.rho_a * sum_wcu;
    else return k.rhoref_T * s + omega * k.rho_a * sum_wcu;
}

// S3..S5 of one site in FP32, per direction pair.  For the pair (c, -c),
// h_eq and g_eq split into a part even in c and a part odd in c:
//   h_eq(+-c) = w { phi (1 - u^2/(2T)) + phi (c.u)^2/(2T^2) } +- w c.(phi u/T + theta n)
//   g_eq(+-c) = w { (c.u)^2/(2T^2) - u^2/(2T) + B div/T } +- w c.(u/T + F/(rho T) + sigma grad rho/(rho^2 T))
// so each pair needs one c.u and two dot products with per-site vectors.
// The same formulas as the canonical collide below, regrouped; divisions by
// per-site quantities become one reciprocal each.
// GMOM: instead of the pulled g (gp), the filter gets its second moments
// pig = sum_i c_ia c_ib g_i (xx, xy, xz, yy, yz, zz in 3D; xx, xy, yy in 2D):
// Pi = pig - sum_i c_ia c_ib g_eq_i is all the filter needs of g.
template <int D>
__host__ __device__ constexpr int pig_slot(int a, int b)
{
    return D == 3 ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (a == 0 ? b : 2);
}

// Knuth's TwoSum: s = RN(a + b) and the exact rounding error e, s + e = a + b
// (round-to-nearest intrinsics, so nothing is contracted or reassociated).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// GODD: g* is returned without its odd first-order part w_i c_i . V_g, and
// V_g = u/T + F/(rho T) + sigma grad rho/(rho^2 T) is returned in vgout.
template <class L, bool INIT, bool PDEV, bool GMOM = false, bool GODD = false>
__device__ __forceinline__ void collide_pairs(const SiteConsts<float> &k, float phi, float phihat, float rho,
                                              float P, const float (&u)[3], const float (&gphi)[3], float lphi,
                                              const float (&gu)[3][3], const float *hp, const float *gp, float *hs,
                                              float *gs, const float *pig = nullptr, float *vgout = nullptr)
{
    constexpr int D = L::D;
    constexpr int NP = (L::Q - 1) / 2;
    // --- S3
    float gg = gphi[0] * gphi[0] + gphi[1] * gphi[1];
    if constexpr (D == 3) gg = gg + gphi[2] * gphi[2];
    const float gnorm = sqrtf(gg);
    const float ninv = 1.f / (gnorm + k.eps);
    float n[3];
    n[0] = gphi[0] * ninv;
    n[1] = gphi[1] * ninv;
    n[2] = (D == 3) ? gphi[2] * ninv : 0.f;
    const float theta = k.M3 * ((1.f - 4.f * (phi - 0.5f) * (phi - 0.5f)) * k.invW);
    float dtheta;
    {
        const float s = lphi / (fabsf(lphi) + k.eps);
        const float Y1 = fminf(fmaxf(0.f, fminf(1.f, (phi - k.phi_n) * k.invD)),
                               fmaxf(0.f, fminf(1.f, (1.f - phi) * k.invD)));
        const float Y2 = fminf(fmaxf(0.f, fminf(1.f, phi * k.invD)),
                               fmaxf(0.f, fminf(1.f, (k.phi_m - phi) * k.invD)));
        dtheta = k.dt_pref * gnorm * ((1.f + s) * Y1 + (1.f - s) * Y2);
    }
    const float theta_tot = theta + dtheta;
    const float mu = k.A_mu * phi * (phi - 1.f) * (phi - 0.5f) - k.B_mu * lphi;
    float F[3];
    F[0] = rho * k.g[0] + mu * gphi[0];
    F[1] = rho * k.g[1] + mu * gphi[1];
    F[2] = (D == 3) ? rho * k.g[2] + mu * gphi[2] : 0.f;
    const float tau = k.tau_a + phihat * k.dtau;
    const float nu = (tau - 0.5f) * (1.f / 3.f);
    const float B = (2.f / 3.f) * (nu - k.lambda_b) + (1.f / 6.f);
    float div = gu[0][0] + gu[1][1];
    if constexpr (D == 3) div = div + gu[2][2];
    float grho[3];
    grho[0] = k.drho * gphi[0];
    grho[1] = k.drho * gphi[1];
    grho[2] = (D == 3) ? k.drho * gphi[2] : 0.f;
    float sg[3];
    {
        const float rnu = rho * nu;
        const float bulk = rho * (2.f / 3.f) * (k.lambda_b - nu) * div;
        float sig[3][3];
        static_for<0, D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            static_for<0, D>([&](auto Bb) {
                constexpr int b = decltype(Bb)::value;
                if constexpr (a == b) sig[a][b] = rnu * (gu[a][b] + gu[b][a]) + bulk;
                else sig[a][b] = rnu * (gu[a][b] + gu[b][a]);
            });
        });
        static_for<0, D>([&](auto A) {
            constexpr int l = decltype(A)::value;
            float t = sig[l][0] * grho[0] + sig[l][1] * grho[1];
            if constexpr (D == 3) t = t + sig[l][2] * grho[2];
            sg[l] = t;
        });
        if constexpr (D == 2) sg[2] = 0.f;
    }
    float uu = u[0] * u[0] + u[1] * u[1];
    if constexpr (D == 3) uu = uu + u[2] * u[2];

    // per-site parts of the equilibria
    const float rinv = 1.f / rho;
    const float kF = 3.f * rinv;          // 1 / (rho T)
    const float kS = kF * rinv;           // 1 / (rho^2 T)
    const float bdiv = B * div * 3.f;     // B div / T
    // D2Q9: the odd part of g_eq, w_i c_i . (u/T + F/(rho T) + ...), with one
    // rounding in place of three.  Formed as 3 c.u + c.V_f in one float, the
    // body force of a slow steady flow (1e-7 against u/T ~ 0.3) loses a few
    // per cent at every step in the same direction, and the velocity drifts
    // by 1e-5 of itself in 1000 steps; kept exact as a float pair (an FMA
    // for the product by 3, TwoSum for the sum, w_i as a float pair) it is
    // rounded once, and the drift stays at the level of the storage.
    constexpr bool kCompOdd = L::Q == 9;
    float Vh[3], Vg[3];
    [[maybe_unused]] float Vf[3];
    static_for<0, 3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        Vh[a] = 3.f * phi * u[a] + theta_tot * n[a];
        Vg[a] = 3.f * u[a] + F[a] * kF + sg[a] * kS;
        if constexpr (kCompOdd) Vf[a] = F[a] * kF + sg[a] * kS;
    });
    if constexpr (GODD) {
        vgout[0] = Vg[0];
        vgout[1] = Vg[1];
        vgout[2] = Vg[2];
    }
    const float Eh0 = phi * (1.f - 1.5f * uu);
    const float Eg0 = bdiv - 1.5f * uu;
    const float p45 = 4.5f * phi;

    // --- S4 and S5, rest direction (h: after the pairs)
    const float w0 = float(L::w(0));
    float geq0 = w0 * (-1.5f * uu) + (w0 - 1.f) * bdiv;
    if constexpr (!PDEV) geq0 = P * k.cP + geq0;
    if constexpr (INIT) gs[0] = geq0;
    float eg[NP], og[NP], ne[NP];
    float seh = 0.f;                                    // sum of the pairs' even h_eq parts
    static_for<0, NP>([&](auto Pp) {
        constexpr int p = decltype(Pp)::value;
        constexpr int i = 2 * p + 1;
        const float wi = float(L::w(i));
        const float cu = dot_c<L, i>(u);
        const float cu2 = cu * cu;
        const float eh = wi * (Eh0 + p45 * cu2);
        const float oh = wi * dot_c<L, i>(Vh);
        seh = __fadd_rn(seh, eh);                    // no contraction: every kernel rounds eh alike
        eg[p] = wi * (Eg0 + 4.5f * cu2);
        if constexpr (kCompOdd) {
            constexpr float whi = float(L::w(i));
            constexpr float wlo = float(L::w(i) - double(whi));
            const float p3 = __fmul_rn(3.f, cu);
            const float e1 = fmaf(3.f, cu, -p3);              // 3 c.u = p3 + e1 exactly
            float sv, e2;
            two_sum(p3, dot_c<L, i>(Vf), sv, e2);
            const float lo = __fadd_rn(e1, e2);
            og[p] = fmaf(whi, sv, fmaf(whi, lo, __fmul_rn(wlo, sv)));
        } else {
            og[p] = wi * dot_c<L, i>(Vg);
        }
        if constexpr (INIT) {
            hs[i] = eh + oh;
            hs[i + 1] = eh - oh;
            gs[i] = eg[p] + og[p];
            gs[i + 1] = eg[p] - og[p];
        } else {
            hs[i] = hp[i] - (hp[i] - (eh + oh)) * k.inv_tau_phi;
            hs[i + 1] = hp[i + 1] - (hp[i + 1] - (eh - oh)) * k.inv_tau_phi;
            if constexpr (GMOM) ne[p] = -2.f * eg[p];      // - g_eq summed over the pair
            else ne[p] = (gp[i] + gp[i + 1]) - 2.f * eg[p];   // (g - g_eq) summed over the pair
        }
    });
    // sum_i h_eq_i = phi (sum_i Gamma_i = 1, the odd parts cancel): the rest
    // direction takes phi minus the moving directions, so the zeroth moment
    // does not depend on the FP32 weights, whose sum exceeds 1 by 7e-9 (D2Q9,
    // D3Q27) or 1.5e-8 (D3Q19) and would add that fraction of the phase mass
    // every step.  In exact arithmetic this is w_0 phi (1 - u^2 / (2T)).
    const float heq0 = phi - 2.f * seh;
    if constexpr (INIT) {
        hs[0] = heq0;
    } else {
        // The BGK step keeps sum_i h_i = phi (sum_i h_eq_i = phi), so the rest
        // population is what the moving ones leave of phi, the sum of the
        // pulled h: the rounding of the moving populations then does not
        // accumulate in the phase mass.  In exact arithmetic this is
        // h_0 - (h_0 - h_eq_0) / tau_phi.
        float sm = 0.f;
        static_for<1, L::Q>([&](auto I) { sm = __fadd_rn(sm, hs[decltype(I)::value]); });
        hs[0] = __fsub_rn(phi, sm);
    }
    if constexpr (!INIT) {
        // Pi_ab = sum_k c_ka c_kb (g_k - g_eq_k), per pair (c_ka c_kb is even in c)
        float Pi[3][3];
        static_for<0, D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            static_for<a, D>([&](auto Bb) {
                constexpr int b = decltype(Bb)::value;
                float acc = 0.f;
                if constexpr (GMOM) acc = pig[pig_slot<D>(a, b)];
                static_for<0, NP>([&](auto Pp) {
                    constexpr int p = decltype(Pp)::value;
                    constexpr int cc = L::c(2 * p + 1, a) * L::c(2 * p + 1, b);
                    if constexpr (cc != 0) acc_c<cc>(acc, ne[p]);
                });
                Pi[a][b] = acc;
                if constexpr (a != b) Pi[b][a] = acc;
            });
        });
        float tr = Pi[0][0] + Pi[1][1];
        if constexpr (D == 3) tr = tr + Pi[2][2];
        if (!k.full_trace) {
            const float trd = tr * (1.f / float(D));
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                Pi[a][a] = Pi[a][a] - trd;
            });
            tr = 0.f;
        }
        // (c_ia c_ib - T delta_ab) Pi_ab = c_ia c_ib Pi_ab - T tr Pi, the same for c and -c
        const float om = 1.f - 1.f / tau;
        const float base = -(1.f / 3.f) * tr;
        gs[0] = geq0 + om * (w0 * 4.5f) * base;
        static_for<0, NP>([&](auto Pp) {
            constexpr int p = decltype(Pp)::value;
            constexpr int i = 2 * p + 1;
            float contr = base;
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                if constexpr (L::c(i, a) != 0) contr = contr + Pi[a][a];
                static_for<a + 1, D>([&](auto Bb) {
                    constexpr int b = decltype(Bb)::value;
                    constexpr int cc = L::c(i, a) * L::c(i, b);
                    if constexpr (cc != 0) acc_c<cc>(contr, 2.f * Pi[a][b]);
                });
            });
            const float e = eg[p] + om * (float(L::w(i)) * 4.5f) * contr;
            if constexpr (GODD) {
                gs[i] = e;
                gs[i + 1] = e;
            } else {
                gs[i] = e + og[p];
                gs[i + 1] = e - og[p];
            }
        });
    }
}

// S3..S5 of one site: from phi, phihat, rho, P = P^{n+1}, u = u^{n+1}, the
// stencils and the pulled populations (hp, gp), the post-collision
// populations hs, gs.  INIT: return the equilibria (start state).
// PDEV: the rest population is produced without its P / (rho_ref T) term
// (see s1_pressure).
template <class L, class R, bool INIT, bool PDEV = false>
__device__ __forceinline__ void collide(const SiteConsts<R> &k, R phi, R phihat, R rho, R P, const R (&u)[3],
                                        const R (&gphi)[3], R lphi, const R (&gu)[3][3], const R *hp,
                                        const R *gp, R *hs, R *gs)
{
    if constexpr (kPairForms<R>) {
        collide_pairs<L, INIT, PDEV>(k, phi, phihat, rho, P, u, gphi, lphi, gu, hp, gp, hs, gs);
        return;
    }
    constexpr int D = L::D;
    // --- S3: normal, theta, delta-theta, chemical potential, force
    R gg = gphi[0] * gphi[0] + gphi[1] * gphi[1];
    if constexpr (D == 3) gg = gg + gphi[2] * gphi[2];
    const R gnorm = sqrt(gg);
    R n[3];
    n[0] = gphi[0] / (gnorm + k.eps);
    n[1] = gphi[1] / (gnorm + k.eps);
    n[2] = (D == 3) ? gphi[2] / (gnorm + k.eps) : R(0);
    // theta = (M/T) (1 - 4 (phi - 1/2)^2) / W    (Eq. theta_phai_LBeq)
    const R theta = k.M3 * ((R(1) - R(4) * (phi - R(0.5)) * (phi - R(0.5))) / k.W);
    // delta-theta with s = lap / (|lap| + eps)
    R dtheta;
    {
        const R s = lphi / (fabs(lphi) + k.eps);
        const R Y1 = fmin(fmax(R(0), fmin(R(1), (phi - k.phi_n) / k.D)),
                          fmax(R(0), fmin(R(1), -(phi - R(1)) / k.D)));
        const R Y2 = fmin(fmax(R(0), fmin(R(1), phi / k.D)),
                          fmax(R(0), fmin(R(1), -(phi - k.phi_m) / k.D)));
        dtheta = k.dt_pref * gnorm * ((R(1) + s) * Y1 + (R(1) - s) * Y2);
    }
    const R theta_tot = theta + dtheta;
    // mu = (48 sigma / W) phi (phi - 1)(phi - 1/2) - (3 sigma W / 2) lap phi
    const R mu = k.A_mu * phi * (phi - R(1)) * (phi - R(0.5)) - k.B_mu * lphi;
    R F[3];
    F[0] = rho * k.g[0] + mu * gphi[0];
    F[1] = rho * k.g[1] + mu * gphi[1];
    F[2] = (D == 3) ? rho * k.g[2] + mu * gphi[2] : R(0);
    // tau_mix (Eq. tau_interpolate), nu = T (tau - 1/2), B = 2/3 (nu - lambda_b) + T/2
    const R tau = k.tau_a + phihat * k.dtau;
    const R nu = (tau - R(0.5)) * R(1.0 / 3.0);
    const R B = R(2.0 / 3.0) * (nu - k.lambda_b) + R(1.0 / 6.0);
    R div = gu[0][0] + gu[1][1];
    if constexpr (D == 3) div = div + gu[2][2];
    // sigma_lm grad_m rho with grad rho = (rho_w - rho_a) grad phi
    R grho[3];
    grho[0] = k.drho * gphi[0];
    grho[1] = k.drho * gphi[1];
    grho[2] = (D == 3) ? k.drho * gphi[2] : R(0);
    R sg[3];
    {
        const R rnu = rho * nu;
        const R bulk = rho * R(2.0 / 3.0) * (k.lambda_b - nu) * div;
        R sig[3][3];
        static_for<0, D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            static_for<0, D>([&](auto Bb) {
                constexpr int b = decltype(Bb)::value;
                if constexpr (a == b) sig[a][b] = rnu * (gu[a][b] + gu[b][a]) + bulk;
                else sig[a][b] = rnu * (gu[a][b] + gu[b][a]);
            });
        });
        static_for<0, D>([&](auto A) {
            constexpr int l = decltype(A)::value;
            R t = sig[l][0] * grho[0] + sig[l][1] * grho[1];
            if constexpr (D == 3) t = t + sig[l][2] * grho[2];
            sg[l] = t;
        });
        if constexpr (D == 2) sg[2] = R(0);
    }
    R uu = u[0] * u[0] + u[1] * u[1];
    if constexpr (D == 3) uu = uu + u[2] * u[2];

    // --- S4: h_eq = phi Gamma_i + theta w_i (c_i . n); BGK with tau_phi
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const R heq = phi * gamma_i<L, i>(u, uu) + theta_tot * R(L::w(i)) * dot_c<L, i>(n);
        if constexpr (INIT) hs[i] = heq;
        else hs[i] = hp[i] - (hp[i] - heq) * k.inv_tau_phi;
    });

    // --- S5: g_eq (Eq. BGK_LBeq_hydroeq) and the filter collision
    const R kF = R(3) / rho;        // 1 / (rho T)
    const R kS = kF / rho;          // 1 / (rho^2 T)
    const R bdiv = B * div * R(3);  // B div / T
    R geq[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const R wi = R(L::w(i));
        R v;
        if constexpr (i == 0 && !PDEV) v = P * k.cP + gamma_dev_i<L, i>(u, uu);
        else v = gamma_dev_i<L, i>(u, uu);
        if constexpr (i != 0) v = v + wi * dot_c<L, i>(F) * kF;
        if constexpr (i == 0) v = v + (wi - R(1)) * bdiv;
        else v = v + wi * bdiv;
        if constexpr (i != 0) v = v + wi * dot_c<L, i>(sg) * kS;
        geq[i] = v;
    });
    if constexpr (INIT) {
        static_for<0, L::Q>([&](auto I) { gs[decltype(I)::value] = geq[decltype(I)::value]; });
        return;
    } else {
        // Pi_ab = sum_k c_ka c_kb (g_k - g_eq_k)
        R Pi[3][3];
        static_for<0, D>([&](auto A) {
            constexpr int a = decltype(A)::value;
            static_for<a, D>([&](auto Bb) {
                constexpr int b = decltype(Bb)::value;
                R acc = R(0);
                static_for<1, L::Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int cc = L::c(i, a) * L::c(i, b);
                    if constexpr (cc != 0) acc_c<cc>(acc, gp[i] - geq[i]);
                });
                Pi[a][b] = acc;
                if constexpr (a != b) Pi[b][a] = acc;
            });
        });
        if (!k.full_trace) {
            // trace-free part: Pi - (tr Pi / d) delta
            R tr = Pi[0][0] + Pi[1][1];
            if constexpr (D == 3) tr = tr + Pi[2][2];
            const R trd = tr / R(D);
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                Pi[a][a] = Pi[a][a] - trd;
            });
        }
        // g*_i = g_eq_i + (1 - 1/tau) w_i/(2T^2) (c_ia c_ib - T delta_ab) Pi_ab
        const R om = R(1) - R(1) / tau;
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            R contr = R(0);
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                static_for<0, D>([&](auto Bb) {
                    constexpr int b = decltype(Bb)::value;
                    constexpr int cc = L::c(i, a) * L::c(i, b);
                    if constexpr (a == b) {
                        if constexpr (cc != 0) contr = contr + R(1.0 - 1.0 / 3.0) * Pi[a][b];
                        else contr = contr - R(1.0 / 3.0) * Pi[a][b];
                    } else if constexpr (cc != 0) {
                        acc_c<cc>(contr, Pi[a][b]);
                    }
                });
            });
            gs[i] = geq[i] + om * (R(L::w(i)) * R(4.5)) * contr;
        });
    }
}

}  // namespace lbm
