/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the coupled lattice
 * Boltzmann step of Otomo et al., "Lattice Boltzmann models for the
 * hydrodynamic equations in multiphase flow with high density ratio"
 * (arXiv 2512.01027), Sec. II.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) links, loads or calls this file; only tests/,
 * __graft_entry__.smoke() and the cpu_baseline / reference leg of bench.py
 * do.  It shares no code, header, table or constant with the CUDA path: the
 * lattice tables below are written out here from the lattice definitions.
 *
 * Every step is a direct, unblocked loop over sites and directions written
 * in the order the paper states the equations:
 *   S0  pull-streaming of h_i and g_i                         (Eq. LB_phi_filter_col, Eq. LB_filter_col: left-hand sides)
 *   S1  phi = sum h_i, K_i, u = sum (g_i + K_i) c_i, omega, P  (Eq. Kiterm and the P, u definitions beside it)
 *   S2  central-difference gradients / Laplacian              (nearest-neighbour stencils, Sec. II)
 *   S3  n, theta, delta-theta, mu, F, tau_mix, nu, B, sigma    (Eqs. theta_phai_LBeq, delta-theta, mu, F, tau_interpolate, B, stress)
 *   S4  h_eq and the phase-field BGK collision               (Eq. LB_phi_filter_col, h_eq, Gamma_i)
 *   S5  g_eq, Pi and the filter collision                     (Eq. BGK_LBeq_hydroeq g_eq, Eqs. momentum_flux0/1, LB_filter_col)
 *
 * Readings where the paper is silent or ambiguous:
 *   - K_i uses P^n (previous step) at x and x - c_i; the omega-term of P uses
 *     u^n(x - c_i), the velocity of the previous step (one LKS pass started
 *     from the previous step).  Using u^{n+1} there instead (coupling_unew =
 *     1, the alternative reading) makes the liquid unstable under shear next
 *     to walls and at nu < 5e-3.
 *   - The filter carries over only the trace-free part of Pi (the printed
 *     form, with the trace, is linearly unstable at the paper's viscosities);
 *     filter_full_trace = 1 restores the printed form.
 *   - "u = sum (f_i + K_i) c_i" is read with f == g.
 *   - rho(phi) = rho_a + phi_hat (rho_w - rho_a), with phi_hat = phi clamped
 *     to [0, 1] for the material properties rho, tau_mix (nu) and omega only
 *     (switchable by clamp_phi_props); phi itself is never clamped.
 *   - s = lap(phi) / (|lap(phi)| + eps) (the printed |lap + eps| form is
 *     singular at lap = -eps).
 *   - theta in h_eq is theta + delta-theta.
 *   - Gamma_i in h_eq and g_eq uses the new velocity u^{n+1}.
 *   - nu in B and sigma is the local nu = T (tau_mix - 1/2).
 *   - grad(rho) = (rho_w - rho_a) grad(phi) with the phi stencil.
 *   - F_ext = rho * g_ext (body acceleration).
 *   - Walls: halfway bounce-back; a solid (or non-periodic outside) neighbour
 *     contributes phi(solid) := phi(x), P(solid) := P(x), u(solid) := 0.
 *   - The 2/3 factors of B and of the bulk stress term are used as printed,
 *     also for the 2D lattice.
 *
 * Pins (tests/test_oracle_pins.py) check every function here against
 * closed forms, invariants and special cases, except one term: the bulk part
 * of the stress, rho (2/3)(lambda_b - nu) div(u) delta, which enters only
 * through sigma . grad(rho) / rho^2 in g_eq.  No closed form isolates it, so
 * its parity is unpinned: only the independent NumPy transcription
 * (crosscheck_np.py) checks it.
 *
 * Layout: populations are [Q][N], N = nx*ny*nz, x fastest.  Vector fields
 * are [3][N] (z component zero in 2D).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_D2Q9 0
#define ORC_D3Q19 1
#define ORC_D3Q27 2
#define QMAX 27

/* Lattice temperature T = 1/3 (Sec. II, below Eq. theta_phai_LBeq). */
static const double T = 1.0 / 3.0;

typedef struct {
    double rho_w, rho_a, nu_w, nu_a, sigma, M, W, lambda_b, gamma, phi_n, phi_m, D, eps;
    double g_ext[3];
    int32_t clamp_phi_props;
    int32_t filter_full_trace; /* 0: trace-free Pi (default reading); 1: Pi as printed */
    int32_t coupling_unew;     /* 0: the omega-term of P takes u^n (default reading); 1: u^{n+1} */
} orc_params;

typedef struct {
    int d, Q, rest;
    int c[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
} olat;

typedef struct {
    olat L;
    int nx, ny, nz;
    long N;
    int periodic[3];
    unsigned char *solid; /* N bytes, 1 = solid */
    orc_params p;
    double *h, *g;        /* post-collision populations h*, g*  [Q][N] */
    double *P, *u;        /* P^n [N], u^n [3][N] */
    double *hn, *gn;      /* next post-collision populations     [Q][N] */
    double *hp, *gp;      /* pulled (pre-collision) populations  [Q][N] */
    double *phi1, *P1, *u1, *rho1, *phh1; /* S1 results */
    long steps;
} orc_state;

/* ------------------------------------------------------------------ */
/* Lattices: direction order is rest first, then pairs (c, -c).        */

static int lattice_fill(int lattice, olat *L)
{
    static const int c9[9][3] = {
        {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    static const int c27[27][3] = {
        {0, 0, 0},
        {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
        {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
        {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
        {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
        {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
    int i, j, a;
    memset(L, 0, sizeof(*L));
    if (lattice == ORC_D2Q9) {
        L->d = 2; L->Q = 9;
        for (i = 0; i < 9; ++i) for (a = 0; a < 3; ++a) L->c[i][a] = c9[i][a];
    } else if (lattice == ORC_D3Q19 || lattice == ORC_D3Q27) {
        L->d = 3; L->Q = (lattice == ORC_D3Q19) ? 19 : 27;
        for (i = 0; i < L->Q; ++i) for (a = 0; a < 3; ++a) L->c[i][a] = c27[i][a];
    } else {
        return -1;
    }
    for (i = 0; i < L->Q; ++i) {
        int cc = L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2];
        double wv = 0.0;
        if (lattice == ORC_D2Q9) {
            wv = (cc == 0) ? 4.0 / 9.0 : (cc == 1) ? 1.0 / 9.0 : 1.0 / 36.0;
        } else if (lattice == ORC_D3Q19) {
            wv = (cc == 0) ? 1.0 / 3.0 : (cc == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
        } else {
            wv = (cc == 0) ? 8.0 / 27.0 : (cc == 1) ? 2.0 / 27.0 : (cc == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
        }
        L->w[i] = wv;
        if (cc == 0) L->rest = i;
    }
    for (i = 0; i < L->Q; ++i) {
        L->opp[i] = -1;
        for (j = 0; j < L->Q; ++j)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    return 0;
}

int orc_lattice_info(int lattice, int *d, int *Q, int *c /* [Q][3] */, double *w /* [Q] */)
{
    olat L;
    int i, a;
    if (lattice_fill(lattice, &L) != 0) return -1;
    if (d) *d = L.d;
    if (Q) *Q = L.Q;
    for (i = 0; i < L.Q; ++i) {
        if (c) for (a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        if (w) w[i] = L.w[i];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Grid helpers                                                        */

/* Index of site (x,y,z) + (dx,dy,dz), or -1 when that site is solid or lies
 * outside a non-periodic edge (treated as solid). */
static long neighbour(const orc_state *s, int x, int y, int z, int dx, int dy, int dz)
{
    long idx;
    x += dx; y += dy; z += dz;
    if (x < 0 || x >= s->nx) { if (!s->periodic[0]) return -1; x = (x % s->nx + s->nx) % s->nx; }
    if (y < 0 || y >= s->ny) { if (!s->periodic[1]) return -1; y = (y % s->ny + s->ny) % s->ny; }
    if (z < 0 || z >= s->nz) { if (!s->periodic[2]) return -1; z = (z % s->nz + s->nz) % s->nz; }
    idx = (long)x + (long)s->nx * ((long)y + (long)s->ny * (long)z);
    if (s->solid && s->solid[idx]) return -1;
    return idx;
}

static void coords(const orc_state *s, long idx, int *x, int *y, int *z)
{
    *x = (int)(idx % s->nx);
    *y = (int)((idx / s->nx) % s->ny);
    *z = (int)(idx / ((long)s->nx * s->ny));
}

/* K_i = w_i / (T rho) { P(x - c_i) - P(x) }  (Eq. Kiterm) at site idx =
 * (x, y, z) for the pressure field P (the previous step's P^n), with
 * kfac = 1/(T rho); a solid or outside source x - c_i takes P(x).  The only
 * evaluation of K_i: the S1 step (both its velocity and its pressure sums)
 * and the pin entry point orc_k_terms call it. */
static double k_term(const orc_state *s, const double *P, long idx, int x, int y, int z, int i, double kfac)
{
    const olat *L = &s->L;
    long src = neighbour(s, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
    double Psrc = (src >= 0) ? P[src] : P[idx];
    return L->w[i] * kfac * (Psrc - P[idx]);
}

/* w_i (c_i . u)|_{x - c_i}, the summand of the omega-term of P (Sec. II,
 * pressure formula), for the velocity field u [3][N] (the previous step's
 * u^n); a solid or outside source contributes u = 0.  Used by the S1 step
 * and by orc_k_terms. */
static double wcu_term(const orc_state *s, const double *u, long idx, int x, int y, int z, int i)
{
    const olat *L = &s->L;
    const long N = s->N;
    long src = neighbour(s, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
    double un[3];
    int a;
    (void)idx;
    for (a = 0; a < 3; ++a) un[a] = (src >= 0) ? u[a * N + src] : 0.0;
    return L->w[i] * (L->c[i][0] * un[0] + L->c[i][1] * un[1] + L->c[i][2] * un[2]);
}

/* Central-difference gradient and Laplacian of a scalar field f at site idx
 * (Sec. II, nearest-neighbour stencils):
 *   d_a f  = sum_i { f(x + c_i) - f(x - c_i) } c_ia w_i / (2T)
 *   lap f  = 2 sum_i { f(x + c_i) - f(x) } w_i / T
 * A solid or outside neighbour takes the value f_solid. */
static void stencil(const orc_state *s, const double *f, long idx, double f_solid,
                    double grad[3], double *lap)
{
    const olat *L = &s->L;
    int x, y, z, i, a;
    double acc[3] = {0.0, 0.0, 0.0}, lacc = 0.0;
    coords(s, idx, &x, &y, &z);
    for (i = 0; i < L->Q; ++i) {
        long ip = neighbour(s, x, y, z, L->c[i][0], L->c[i][1], L->c[i][2]);
        long im = neighbour(s, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
        double fp = (ip >= 0) ? f[ip] : f_solid;
        double fm = (im >= 0) ? f[im] : f_solid;
        for (a = 0; a < 3; ++a) acc[a] += (fp - fm) * L->c[i][a] * L->w[i];
        lacc += (fp - f[idx]) * L->w[i];
    }
    for (a = 0; a < 3; ++a) grad[a] = acc[a] * 1.5;   /* 1/(2T), T = 1/3 */
    *lap = lacc * 6.0;                              /* 2/T */
}

/* F(x) = max{0, min{1, x}} of the delta-theta correction. */
static double Fclip(double x)
{
    return fmax(0.0, fmin(1.0, x));
}

/* delta-theta anti-rarefaction correction (Sec. II, equation after
 * Eq. theta_phai_LBeq), with s = lap / (|lap| + eps):
 *   dtheta = gamma M/(T W) |grad phi| { (1+s) Y1 + (1-s) Y2 } */
double orc_delta_theta(const orc_params *p, double phi, double grad_norm, double lap)
{
    double s = lap / (fabs(lap) + p->eps);
    double Y1 = fmin(Fclip((phi - p->phi_n) / p->D), Fclip(-(phi - 1.0) / p->D));
    double Y2 = fmin(Fclip(phi / p->D), Fclip(-(phi - p->phi_m) / p->D));
    double pref = p->gamma * p->M * 3.0 / p->W;     /* gamma M / (T W) */
    return pref * grad_norm * ((1.0 + s) * Y1 + (1.0 - s) * Y2);
}

/* Gamma_i = w_i { 1 + c.u/T + (c.u)^2/(2T^2) - u^2/(2T) }  (Sec. II),
 * with 1/T = 3, 1/(2T^2) = 9/2, 1/(2T) = 3/2. */
static double Gamma(const olat *L, int i, const double u[3])
{
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * (1.0 + 3.0 * cu + 4.5 * (cu * cu) - 1.5 * uu);
}

/* Gamma_i - w_i = w_i { c.u/T + (c.u)^2/(2T^2) - u^2/(2T) }: the same
 * polynomial without its constant term, the form in which Gamma_i enters
 * g_eq (evaluated directly, not as a difference of two numbers near w_i). */
static double Gamma_minus_w(const olat *L, int i, const double u[3])
{
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[i] * (3.0 * cu + 4.5 * (cu * cu) - 1.5 * uu);
}

/* h_eq_i = phi Gamma_i + theta_tot w_i (c_i . n)  (Sec. II). */
static void h_equilibrium(const olat *L, double phi, const double u[3], const double n[3],
                          double theta_tot, double *heq)
{
    int i;
    for (i = 0; i < L->Q; ++i) {
        double cn = L->c[i][0] * n[0] + L->c[i][1] * n[1] + L->c[i][2] * n[2];
        heq[i] = phi * Gamma(L, i, u) + theta_tot * L->w[i] * cn;
    }
}

/* g_eq_i (Eq. BGK_LBeq_hydroeq equilibrium):
 *   P/(rho_ref T) delta_{i,ist} + Gamma_i - w_i + w_i c_i.F/(rho T)
 *   + B (w_i - delta_{i,ist}) div(u) / T + w_i c_il sigma_lm d_m rho / (rho^2 T)
 * evaluated left to right with the factors 1/(rho_ref T) = 3/rho_ref,
 * 1/(rho T) = 3/rho and 1/(rho^2 T) = (3/rho)/rho. */
static void g_equilibrium(const olat *L, const orc_params *p, double P, double rho,
                          const double u[3], const double F[3], double B, double div,
                          const double sig[3][3], const double grho[3], double *geq)
{
    const double cP = 3.0 / p->rho_a;        /* 1/(rho_ref T), rho_ref = rho_air */
    const double kF = 3.0 / rho;             /* 1/(rho T) */
    const double kS = kF / rho;              /* 1/(rho^2 T) */
    const double bdiv = B * div * 3.0;       /* B div / T */
    double sg[3];
    int i, l;
    for (l = 0; l < 3; ++l) sg[l] = sig[l][0] * grho[0] + sig[l][1] * grho[1] + sig[l][2] * grho[2];
    for (i = 0; i < L->Q; ++i) {
        double delta = (i == L->rest) ? 1.0 : 0.0;
        double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
        double csg = L->c[i][0] * sg[0] + L->c[i][1] * sg[1] + L->c[i][2] * sg[2];
        double v = (i == L->rest) ? P * cP : 0.0;
        v = v + Gamma_minus_w(L, i, u);                 /* Gamma_i - w_i */
        v = v + L->w[i] * cF * kF;
        v = v + (L->w[i] - delta) * bdiv;
        v = v + L->w[i] * csg * kS;
        geq[i] = v;
    }
}

/* Filter collision (Eqs. momentum_flux0, momentum_flux, LB_filter_col):
 *   Pi_ab  = sum_k c_ka c_kb (g_k - g_eq_k)
 *   g*_i   = g_eq_i + (1 - 1/tau) w_i/(2T^2) (c_ia c_ib - T delta_ab) Pi_ab
 * Reading (see the file header): unless full_trace is set, the trace of Pi
 * is removed before the projection, i.e. only the trace-free (shear) part of
 * the non-equilibrium momentum flux is carried over; the bulk part relaxes to
 * the equilibrium each step and the bulk behaviour is set by the B term of
 * g_eq.  With the trace kept the linearised step is unstable at every
 * viscosity the paper simulates (spectral radius ~1.04 at nu = 0.0167). */
static void filter_collision(const olat *L, double tau, const double *g, const double *geq, double *gs,
                             int full_trace)
{
    double Pi[3][3] = {{0}};
    int i, k, a, b;
    for (k = 0; k < L->Q; ++k)
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b)
                Pi[a][b] += L->c[k][a] * L->c[k][b] * (g[k] - geq[k]);
    if (!full_trace) {
        double tr = 0.0;
        for (a = 0; a < L->d; ++a) tr += Pi[a][a];
        for (a = 0; a < L->d; ++a) Pi[a][a] -= tr / (double)L->d;
    }
    for (i = 0; i < L->Q; ++i) {
        double contr = 0.0;
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b)
                contr += (L->c[i][a] * L->c[i][b] - (a == b ? T : 0.0)) * Pi[a][b];
        gs[i] = geq[i] + (1.0 - 1.0 / tau) * (L->w[i] * 4.5) * contr;   /* w_i/(2T^2) */
    }
}

/* Local state of one site entering S3..S5. */
typedef struct {
    double phi, phihat, rho, P;
    double u[3];
    double gphi[3], lphi;
    double gu[3][3]; /* gu[a][b] = d u_a / d x_b */
} site_in;

/* S3..S5 at one site.  init != 0: return the equilibria (start state). */
static void collide_site(const orc_state *s, const site_in *in, const double *hp, const double *gp,
                         double *hs, double *gs, int init)
{
    const olat *L = &s->L;
    const orc_params *p = &s->p;
    double heq[QMAX], geq[QMAX];
    double n[3], F[3], grho[3], sig[3][3];
    double gnorm, theta, dtheta, mu, tau, nu, B, div, tau_phi, inv_tau_phi, tau_w, tau_a;
    int i, a, b;

    /* S3: interface normal, theta, delta-theta, chemical potential, force */
    gnorm = sqrt(in->gphi[0] * in->gphi[0] + in->gphi[1] * in->gphi[1] + in->gphi[2] * in->gphi[2]);
    for (a = 0; a < 3; ++a) n[a] = in->gphi[a] / (gnorm + p->eps);
    /* theta = (M/T) (1 - 4 (phi - 1/2)^2) / W */
    theta = (p->M * 3.0) * ((1.0 - 4.0 * (in->phi - 0.5) * (in->phi - 0.5)) / p->W);
    dtheta = orc_delta_theta(p, in->phi, gnorm, in->lphi);
    /* mu = (48 sigma / W) phi (phi - 1)(phi - 1/2) - (3 sigma W / 2) lap(phi) */
    mu = (48.0 * p->sigma / p->W) * in->phi * (in->phi - 1.0) * (in->phi - 0.5)
       - (1.5 * p->sigma * p->W) * in->lphi;
    for (a = 0; a < 3; ++a) F[a] = in->rho * p->g_ext[a] + mu * in->gphi[a];
    /* relaxation time mixing (Eq. tau_interpolate): tau_k = nu_k / T + 1/2 */
    tau_w = p->nu_w * 3.0 + 0.5;
    tau_a = p->nu_a * 3.0 + 0.5;
    tau = tau_a + in->phihat * (tau_w - tau_a);
    nu = (tau - 0.5) * T;                                    /* nu = T (tau - 1/2) */
    B = (2.0 / 3.0) * (nu - p->lambda_b) + (1.0 / 6.0);      /* 2/3 (nu - lambda_b) + T/2 */
    div = in->gu[0][0] + in->gu[1][1] + in->gu[2][2];
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b)
            sig[a][b] = in->rho * nu * (in->gu[a][b] + in->gu[b][a])
                      + (a == b ? in->rho * (2.0 / 3.0) * (p->lambda_b - nu) * div : 0.0);
    for (a = 0; a < 3; ++a) grho[a] = (p->rho_w - p->rho_a) * in->gphi[a];

    /* S4: phase-field equilibrium and BGK collision (Eq. LB_phi_filter_col) */
    h_equilibrium(L, in->phi, in->u, n, theta + dtheta, heq);
    tau_phi = p->M * 3.0 + 0.5;                              /* M/T + 1/2 */
    inv_tau_phi = 1.0 / tau_phi;
    for (i = 0; i < L->Q; ++i)
        hs[i] = init ? heq[i] : hp[i] - (hp[i] - heq[i]) * inv_tau_phi;

    /* S5: hydrodynamic equilibrium and filter collision (Eq. LB_filter_col) */
    g_equilibrium(L, p, in->P, in->rho, in->u, F, B, div, sig, grho, geq);
    if (init) {
        for (i = 0; i < L->Q; ++i) gs[i] = geq[i];
    } else {
        filter_collision(L, tau, gp, geq, gs, p->filter_full_trace);
    }
}

/* ------------------------------------------------------------------ */
/* State                                                               */

static double *zalloc(long n)
{
    return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
}

void orc_destroy(void *vs)
{
    orc_state *s = (orc_state *)vs;
    if (!s) return;
    free(s->solid); free(s->h); free(s->g); free(s->P); free(s->u);
    free(s->hn); free(s->gn); free(s->hp); free(s->gp);
    free(s->phi1); free(s->P1); free(s->u1); free(s->rho1); free(s->phh1);
    free(s);
}

void *orc_create(int lattice, int nx, int ny, int nz, const int32_t periodic[3],
                 const unsigned char *solid, const orc_params *p)
{
    orc_state *s;
    long N;
    int Q;
    if (nx <= 0 || ny <= 0 || nz <= 0 || !p) return NULL;
    s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    if (lattice_fill(lattice, &s->L) != 0) { free(s); return NULL; }
    if (s->L.d == 2 && nz != 1) { free(s); return NULL; }
    s->nx = nx; s->ny = ny; s->nz = nz;
    N = (long)nx * ny * nz;
    s->N = N;
    s->periodic[0] = periodic ? periodic[0] : 1;
    s->periodic[1] = periodic ? periodic[1] : 1;
    s->periodic[2] = periodic ? periodic[2] : 1;
    s->p = *p;
    Q = s->L.Q;
    s->solid = (unsigned char *)calloc((size_t)N, 1);
    if (solid) memcpy(s->solid, solid, (size_t)N);
    s->h = zalloc(Q * N); s->g = zalloc(Q * N);
    s->hn = zalloc(Q * N); s->gn = zalloc(Q * N);
    s->hp = zalloc(Q * N); s->gp = zalloc(Q * N);
    s->P = zalloc(N); s->u = zalloc(3 * N);
    s->phi1 = zalloc(N); s->P1 = zalloc(N); s->u1 = zalloc(3 * N);
    s->rho1 = zalloc(N); s->phh1 = zalloc(N);
    if (!s->solid || !s->h || !s->g || !s->hn || !s->gn || !s->hp || !s->gp || !s->P || !s->u ||
        !s->phi1 || !s->P1 || !s->u1 || !s->rho1 || !s->phh1) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

static double clamp01(double v)
{
    return fmin(1.0, fmax(0.0, v));
}

/* Collide every fluid site from the S1 fields (phi1, u1, P1, rho1, phh1)
 * and the pulled populations (hp, gp) into (hn, gn). */
static void collide_all(orc_state *s, int init)
{
    const long N = s->N;
    const int Q = s->L.Q;
    long idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < N; ++idx) {
        site_in in;
        double hpi[QMAX], gpi[QMAX], hsi[QMAX], gsi[QMAX];
        int i, a;
        if (s->solid[idx]) continue;
        in.phi = s->phi1[idx];
        in.phihat = s->phh1[idx];
        in.rho = s->rho1[idx];
        in.P = s->P1[idx];
        for (a = 0; a < 3; ++a) in.u[a] = s->u1[a * N + idx];
        stencil(s, s->phi1, idx, s->phi1[idx], in.gphi, &in.lphi);
        for (a = 0; a < 3; ++a) {
            double lap_unused;
            stencil(s, s->u1 + a * N, idx, 0.0, in.gu[a], &lap_unused);
        }
        for (i = 0; i < Q; ++i) { hpi[i] = s->hp[i * N + idx]; gpi[i] = s->gp[i * N + idx]; }
        collide_site(s, &in, hpi, gpi, hsi, gsi, init);
        for (i = 0; i < Q; ++i) { s->hn[i * N + idx] = hsi[i]; s->gn[i * N + idx] = gsi[i]; }
    }
    /* post-collision state becomes current */
    {
        double *t;
        t = s->h; s->h = s->hn; s->hn = t;
        t = s->g; s->g = s->gn; s->gn = t;
    }
}

/* Initial state from fields phi0, P0, u0 ([3][N] or [d][N]): populations
 * start at equilibrium (Sec. I, after Eq. feq_expansion).  u0 has `ncomp`
 * component planes (2 or 3). */
int orc_init(void *vs, const double *phi0, const double *P0, const double *u0, int ncomp)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    long idx;
    int a;
    if (!s || !phi0 || !P0 || !u0 || ncomp < s->L.d || ncomp > 3) return -1;
    memset(s->u, 0, sizeof(double) * 3 * N);
    memset(s->P, 0, sizeof(double) * N);
    memset(s->h, 0, sizeof(double) * s->L.Q * N);
    memset(s->g, 0, sizeof(double) * s->L.Q * N);
    memset(s->hn, 0, sizeof(double) * s->L.Q * N);
    memset(s->gn, 0, sizeof(double) * s->L.Q * N);
    memset(s->phi1, 0, sizeof(double) * N);
    memset(s->u1, 0, sizeof(double) * 3 * N);
    for (idx = 0; idx < N; ++idx) {
        if (s->solid[idx]) continue;
        s->phi1[idx] = phi0[idx];
        s->phh1[idx] = s->p.clamp_phi_props ? clamp01(phi0[idx]) : phi0[idx];
        s->rho1[idx] = s->p.rho_a + s->phh1[idx] * (s->p.rho_w - s->p.rho_a);
        s->P1[idx] = P0[idx];
        s->P[idx] = P0[idx];
        for (a = 0; a < s->L.d; ++a) {
            s->u1[a * N + idx] = u0[a * N + idx];
            s->u[a * N + idx] = u0[a * N + idx];
        }
    }
    collide_all(s, 1);
    s->steps = 0;
    return 0;
}

/* One time step n -> n+1 (S0..S5 at every fluid site). */
static void step_once(orc_state *s)
{
    const olat *L = &s->L;
    const orc_params *p = &s->p;
    const long N = s->N;
    const int Q = L->Q;
    const double rho_ref = p->rho_a;                 /* rho_ref = rho_air (Sec. II) */
    const double omega_max = p->rho_w / p->rho_a;    /* no LKS iteration: omega_max = rho_ratio */
    long idx;

    /* S0 and the first part of S1: phi, rho, K_i, u^{n+1} */
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < N; ++idx) {
        double hpi[QMAX], gpi[QMAX], K[QMAX];
        double phi, phihat, rho, kfac;
        int x, y, z, i, a;
        if (s->solid[idx]) continue;
        coords(s, idx, &x, &y, &z);
        /* S0: pull h_i(x) = h*_i(x - c_i); bounce-back from a solid source */
        for (i = 0; i < Q; ++i) {
            long src = neighbour(s, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
            if (src >= 0) {
                hpi[i] = s->h[i * N + src];
                gpi[i] = s->g[i * N + src];
            } else {
                hpi[i] = s->h[L->opp[i] * N + idx];
                gpi[i] = s->g[L->opp[i] * N + idx];
            }
            s->hp[i * N + idx] = hpi[i];
            s->gp[i * N + idx] = gpi[i];
        }
        /* order parameter and material properties */
        phi = 0.0;
        for (i = 0; i < Q; ++i) phi += hpi[i];
        phihat = p->clamp_phi_props ? clamp01(phi) : phi;
        rho = p->rho_a + phihat * (p->rho_w - p->rho_a);
        /* K_i = w_i / (T rho) { P(x - c_i) - P(x) }  (Eq. Kiterm), P = P^n */
        kfac = 3.0 / rho;                                    /* 1/(T rho) */
        for (i = 0; i < Q; ++i) K[i] = k_term(s, s->P, idx, x, y, z, i, kfac);
        /* u = sum_i (g_i + K_i) c_i */
        for (a = 0; a < 3; ++a) {
            double acc = 0.0;
            for (i = 0; i < Q; ++i) acc += (gpi[i] + K[i]) * L->c[i][a];
            s->u1[a * N + idx] = acc;
        }
        s->phi1[idx] = phi;
        s->phh1[idx] = phihat;
        s->rho1[idx] = rho;
    }

    /* Second part of S1: the pressure; the omega-term takes u^n(x - c_i)
     * (u^{n+1}(x - c_i), from the first part, with coupling_unew). */
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < N; ++idx) {
        double rho, omega, sum_gK, sum_wcu, kfac;
        int x, y, z, i;
        if (s->solid[idx]) continue;
        coords(s, idx, &x, &y, &z);
        rho = s->rho1[idx];
        kfac = 3.0 / rho;
        /* omega = (rho - rho_a)/(rho_w - rho_a) (omega_max - 1) */
        omega = (rho - p->rho_a) / (p->rho_w - p->rho_a) * (omega_max - 1.0);
        /* P = rho_ref T sum_i (g_i + (1 + omega) K_i) + omega rho_ref sum_i w_i (c_i . u)|_{x - c_i} */
        sum_gK = 0.0;
        sum_wcu = 0.0;
        for (i = 0; i < Q; ++i) {
            double K = k_term(s, s->P, idx, x, y, z, i, kfac);
            sum_gK += s->gp[i * N + idx] + (1.0 + omega) * K;
            sum_wcu += wcu_term(s, p->coupling_unew ? s->u1 : s->u, idx, x, y, z, i);
        }
        s->P1[idx] = rho_ref * T * sum_gK + omega * rho_ref * sum_wcu;
    }

    /* S2..S5 need phi^{n+1}, u^{n+1} of all neighbours: second sweep. */
    collide_all(s, 0);
    {
        double *t;
        t = s->P; s->P = s->P1; s->P1 = t;
        t = s->u; s->u = s->u1; s->u1 = t;
    }
    s->steps += 1;
}

int orc_step(void *vs, long nsteps)
{
    orc_state *s = (orc_state *)vs;
    long k;
    if (!s || nsteps < 0) return -1;
    for (k = 0; k < nsteps; ++k) step_once(s);
    return 0;
}

/* Reported fields after step n: phi^n = sum_i h*_i, P^n, u^n (solid: 0). */
int orc_fields(void *vs, double *phi, double *P, double *u /* [3][N] */)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    long idx;
    int i, a;
    if (!s) return -1;
    for (idx = 0; idx < N; ++idx) {
        int sol = s->solid[idx];
        if (phi) {
            double acc = 0.0;
            if (!sol) for (i = 0; i < s->L.Q; ++i) acc += s->h[i * N + idx];
            phi[idx] = acc;
        }
        if (P) P[idx] = sol ? 0.0 : s->P[idx];
        if (u) for (a = 0; a < 3; ++a) u[a * N + idx] = sol ? 0.0 : s->u[a * N + idx];
    }
    return 0;
}

/* Raw state access: h*, g* [Q][N], P^n [N], u^n [3][N]. */
int orc_get_state(void *vs, double *h, double *g, double *P, double *u)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    if (!s) return -1;
    if (h) memcpy(h, s->h, sizeof(double) * s->L.Q * N);
    if (g) memcpy(g, s->g, sizeof(double) * s->L.Q * N);
    if (P) memcpy(P, s->P, sizeof(double) * N);
    if (u) memcpy(u, s->u, sizeof(double) * 3 * N);
    return 0;
}

int orc_set_state(void *vs, const double *h, const double *g, const double *P, const double *u)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    if (!s) return -1;
    if (h) memcpy(s->h, h, sizeof(double) * s->L.Q * N);
    if (g) memcpy(s->g, g, sizeof(double) * s->L.Q * N);
    if (P) memcpy(s->P, P, sizeof(double) * N);
    if (u) memcpy(s->u, u, sizeof(double) * 3 * N);
    return 0;
}

long orc_steps_done(void *vs)
{
    return vs ? ((orc_state *)vs)->steps : -1;
}

/* ------------------------------------------------------------------ */
/* Per-function entry points used by the pin tests.                    */

/* Stencil of a whole field: grad [3][N], lap [N]; solid neighbours take the
 * centre value (mode 0) or zero (mode 1). */
int orc_grad_lap(void *vs, const double *f, int solid_mode, double *grad, double *lap)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    long idx;
    if (!s || !f) return -1;
    for (idx = 0; idx < N; ++idx) {
        double gr[3], lp;
        int a;
        if (s->solid[idx]) {
            for (a = 0; a < 3; ++a) grad[a * N + idx] = 0.0;
            lap[idx] = 0.0;
            continue;
        }
        stencil(s, f, idx, solid_mode == 0 ? f[idx] : 0.0, gr, &lp);
        for (a = 0; a < 3; ++a) grad[a * N + idx] = gr[a];
        lap[idx] = lp;
    }
    return 0;
}

/* K_i at every fluid site for a given P field and density field:
 * K [Q][N]; also sum_i w_i c_i . u(x - c_i) into wcu [N].  Through the same
 * k_term and wcu_term the S1 step evaluates (kfac = 3 / rho as there). */
int orc_k_terms(void *vs, const double *P, const double *rho, const double *u, double *K, double *wcu)
{
    orc_state *s = (orc_state *)vs;
    const long N = s->N;
    long idx;
    if (!s) return -1;
    for (idx = 0; idx < N; ++idx) {
        int x, y, z, i;
        double acc = 0.0, kfac;
        if (s->solid[idx]) continue;
        coords(s, idx, &x, &y, &z);
        kfac = 3.0 / rho[idx];
        for (i = 0; i < s->L.Q; ++i) {
            K[i * N + idx] = k_term(s, P, idx, x, y, z, i, kfac);
            acc += wcu_term(s, u, idx, x, y, z, i);
        }
        wcu[idx] = acc;
    }
    return 0;
}

int orc_h_eq(int lattice, double phi, const double u[3], const double n[3], double theta_tot, double *heq)
{
    olat L;
    if (lattice_fill(lattice, &L) != 0) return -1;
    h_equilibrium(&L, phi, u, n, theta_tot, heq);
    return 0;
}

int orc_g_eq(int lattice, const orc_params *p, double P, double rho, const double u[3], const double F[3],
             double B, double div, const double sig9[9], const double grho[3], double *geq)
{
    olat L;
    double sig[3][3];
    int a, b;
    if (lattice_fill(lattice, &L) != 0) return -1;
    for (a = 0; a < 3; ++a) for (b = 0; b < 3; ++b) sig[a][b] = sig9[3 * a + b];
    g_equilibrium(&L, p, P, rho, u, F, B, div, sig, grho, geq);
    return 0;
}

int orc_filter(int lattice, double tau, const double *g, const double *geq, double *gs, int full_trace)
{
    olat L;
    if (lattice_fill(lattice, &L) != 0) return -1;
    filter_collision(&L, tau, g, geq, gs, full_trace);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
