"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them compares the oracle
with itself: closed-form moments, exact stencil identities, invariants,
special cases that reduce to another lattice, an independent NumPy
transcription, linear stability, and the analytic targets (Laplace law,
layered Poiseuille flow, Galilean invariance) the paper validates against.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from oracle.crosscheck_np import CrossCheck2D

T = 1.0 / 3.0
EPS = np.finfo(np.float64).eps
LATTICES = ["D2Q9", "D3Q19", "D3Q27"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def rng(seed):
    return np.random.default_rng(seed)


def moments(f, c):
    m0 = f.sum()
    m1 = c.T.astype(float) @ f
    m2 = np.einsum("i,ia,ib->ab", f, c.astype(float), c.astype(float))
    return m0, m1, m2


# ---------------------------------------------------------------------------
# Lattice tables (Sec. II: D3Q19 with T = 1/3; the D2Q9 / D3Q27 configs use
# the same T): isotropy to fourth order fixes every weight.

@pytest.mark.parametrize("lat", LATTICES)
def test_lattice_isotropy(lat):
    d, Q, c, w = oracle.lattice_info(lat)
    cf = c.astype(float)[:, :d]
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(cf.T @ w).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, cf, cf), T * np.eye(d), atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf)
    I = np.eye(d)
    want = T * T * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                    + np.einsum("ad,bc->abcd", I, I))
    assert np.allclose(m4, want, atol=1e-16)
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf)).max() < 1e-16
    # rest first, then pairs (c, -c)
    assert (c[0] == 0).all()
    for i in range(1, Q, 2):
        assert (c[i] == -c[i + 1]).all()


def test_paper_constants_are_the_defaults():
    """The parameter defaults are the values printed in Sec. II / III."""
    g = json.load(open(GOLDEN))
    p = W.base_params()
    assert p["gamma"] == g["gamma"]["value"]
    assert p["phi_n"] == g["phi_n"]["value"] and p["phi_m"] == g["phi_m"]["value"]
    assert p["D"] == g["D"]["value"] and p["eps"] == g["epsilon_normal"]["value"]
    assert p["lambda_b"] == g["lambda_b"]["value"]
    assert p["M"] == g["M"]["value"] and p["W"] == g["W"]["value"]
    assert p["rho_w"] / p["rho_a"] == pytest.approx(g["rho_ratio"]["value"])


@pytest.mark.parametrize("case", ["bubble_case1", "bubble_case2"])
def test_bubble_table_numbers(case):
    """Table tab_bubblerise: Re and We follow from rho1, mu1, sigma, R, g."""
    g = json.load(open(GOLDEN))[case]
    Ug = np.sqrt(2 * g["R"] * g["g"])
    Re = g["rho1"] * Ug * 2 * g["R"] / g["mu1"]
    We = g["rho1"] * Ug ** 2 * 2 * g["R"] / g["sigma"]
    assert Re == pytest.approx(g["Re"], rel=0.01)
    assert We == pytest.approx(g["We"], rel=0.01)


# ---------------------------------------------------------------------------
# P1: closed-form moments of h_eq (Sec. II: h_eq = phi Gamma + theta w (c.n))

@pytest.mark.parametrize("lat", LATTICES)
def test_heq_moments(lat):
    d, Q, c, w = oracle.lattice_info(lat)
    r = rng(1)
    for _ in range(20):
        phi = r.uniform(-0.1, 1.1)
        u = np.zeros(3); u[:d] = r.uniform(-0.1, 0.1, d)
        n = np.zeros(3); n[:d] = r.normal(size=d); n /= np.linalg.norm(n)
        th = r.uniform(-0.1, 0.1)
        heq = oracle.h_eq(lat, phi, u, n, th)
        m0, m1, m2 = moments(heq, c)
        assert abs(m0 - phi) < 1e-14
        assert np.abs(m1 - (phi * u + th * T * n)).max() < 1e-14
        want2 = phi * (T * np.eye(3) + np.outer(u, u))
        want2[d:, :] = 0; want2[:, d:] = 0
        assert np.abs(m2 - want2).max() < 1e-14


# ---------------------------------------------------------------------------
# P2: closed-form moments of g_eq (Eq. BGK_LBeq_hydroeq)
#   sum g_eq = P/(rho_ref T); sum g_eq c = u + F/rho + sigma.grad(rho)/rho^2;
#   sum g_eq cc = uu + B div delta

@pytest.mark.parametrize("lat", LATTICES)
def test_geq_moments(lat):
    d, Q, c, w = oracle.lattice_info(lat)
    r = rng(2)
    p = oracle.make_params(rho_a=1e-3)
    for _ in range(20):
        P = r.uniform(-1e-3, 1e-3)
        rho = r.uniform(1e-3, 1.0)
        u = np.zeros(3); u[:d] = r.uniform(-0.1, 0.1, d)
        F = np.zeros(3); F[:d] = r.uniform(-1e-5, 1e-5, d)
        B = r.uniform(0, 0.3)
        div = r.uniform(-1e-3, 1e-3)
        sig = np.zeros((3, 3)); s = r.uniform(-1e-4, 1e-4, (d, d)); sig[:d, :d] = s + s.T
        grho = np.zeros(3); grho[:d] = r.uniform(-0.1, 0.1, d)
        geq = oracle.g_eq(lat, p, P, rho, u, F, B, div, sig.ravel(), grho)
        m0, m1, m2 = moments(geq, c)
        assert m0 == pytest.approx(P / (1e-3 * T), abs=1e-12)
        want1 = u + F / rho + sig @ grho / rho ** 2
        assert np.abs(m1 - want1).max() < 1e-13
        want2 = np.outer(u, u) + B * div * np.eye(3)
        want2[d:, :] = 0; want2[:, d:] = 0
        assert np.abs(m2 - want2).max() < 1e-14


# ---------------------------------------------------------------------------
# P3: the filter (Eqs. momentum_flux0/1, LB_filter_col) keeps the zeroth and
# first moments of g_eq and sets the second to g_eq's plus (1-1/tau) Pi
# (trace-free Pi under the adopted reading; full Pi as printed).

@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("full", [False, True])
def test_filter_moments(lat, full):
    d, Q, c, w = oracle.lattice_info(lat)
    r = rng(3)
    for _ in range(10):
        geq = w * (1 + r.uniform(-0.2, 0.2, Q))
        g = geq + r.uniform(-1e-3, 1e-3, Q)
        tau = r.uniform(0.51, 1.5)
        gs = oracle.filter_collision(lat, tau, g, geq, full_trace=full)
        cf = c.astype(float)[:, :d]
        Pi = np.einsum("i,ia,ib->ab", g - geq, cf, cf)
        if not full:
            Pi = Pi - np.trace(Pi) / d * np.eye(d)
        m0, m1, m2 = moments(gs, c[:, :d])
        e0, e1, e2 = moments(geq, c[:, :d])
        assert abs(m0 - e0) < 1e-15
        assert np.abs(m1 - e1).max() < 1e-15
        assert np.abs(m2 - (e2 + (1 - 1 / tau) * Pi)).max() < 1e-15


# ---------------------------------------------------------------------------
# P4: nearest-neighbour stencils (Sec. II) are exact on quadratic fields, and
# the K_i terms (Eq. Kiterm) satisfy sum K = lap(P)/(2 rho),
# sum K c = -grad(P)/rho, sum w c.u(x-c) = -T div(u).  orc_k_terms evaluates
# K_i and the omega-term summands through the same functions the S1 step
# calls (k_term, wcu_term), so these identities pin the step's own code,
# including its wall rule (a solid source contributes P(x) and u = 0, the
# values the stencil takes for a solid neighbour).

@pytest.mark.parametrize("lat,shape", [("D2Q9", (9, 8, 1)), ("D3Q19", (7, 6, 5)),
                                       ("D3Q27", (6, 7, 5))])
def test_stencil_exact_on_quadratics(lat, shape):
    r = rng(4)
    o = oracle.Oracle(lat, shape, periodic=(0, 0, 0))
    d = o.d
    nx, ny, nz = shape
    x, y, z = W.grid_coords(nx, ny, nz)
    X = np.stack([x, y, z])[:d]
    a0 = r.normal()
    b = r.normal(size=d)
    Cm = r.normal(size=(d, d)); Cm = Cm + Cm.T
    f = a0 + np.einsum("a,a...->...", b, X) + np.einsum("a...,ab,b...->...", X, Cm, X)
    grad, lap = o.grad_lap(f)
    want_g = b[:, None, None, None] + 2 * np.einsum("ab,b...->a...", Cm, X)
    want_l = 2 * np.trace(Cm)
    inner = (slice(1, -1) if nz > 2 else slice(None), slice(1, -1), slice(1, -1))
    scale = np.abs(f).max()
    for a in range(d):
        assert np.abs(grad[a][inner] - want_g[a][inner]).max() < 1e-12 * scale
    assert np.abs(lap[inner] - want_l).max() < 1e-12 * scale


@pytest.mark.parametrize("lat,shape", [("D2Q9", (12, 10, 1)), ("D3Q19", (5, 6, 7)), ("D3Q27", (6, 5, 7))])
@pytest.mark.parametrize("walls", [False, True])
def test_k_term_identities(lat, shape, walls):
    r = rng(5)
    periodic, solid = (1, 1, 1), None
    if walls:
        # closed in y, 10 % random solid sites
        periodic = (1, 0, 1)
        solid = (r.uniform(size=shape[::-1]) < 0.1).astype(np.uint8)
    o = oracle.Oracle(lat, shape, periodic=periodic, solid=solid)
    N = o.N
    fluid = np.ones(N, bool) if solid is None else solid.reshape(N) == 0
    P = r.normal(size=N) * 1e-3
    rho = r.uniform(1e-3, 1, N)
    u = np.zeros((3, N)); u[:o.d] = r.normal(size=(o.d, N)) * 1e-2
    K, wcu = o.k_terms(P, rho, u)
    K = K.reshape(o.Q, N)[:, fluid]
    gP, lP = o.grad_lap(P)
    gP = gP.reshape(3, N)[:, fluid]; lP = lP.reshape(N)[fluid]
    rf = rho[fluid]
    assert np.abs(K.sum(0) - lP / (2 * rf)).max() < 1e-12 * np.abs(lP / rf).max()
    Kc = o.c.T.astype(float) @ K
    assert np.abs(Kc - (-gP / rf)).max() < 1e-12 * np.abs(gP / rf).max()
    div = sum(o.grad_lap(u[a], solid_value_zero=True)[0].reshape(3, N)[a] for a in range(o.d))
    assert np.abs(wcu.reshape(N)[fluid] - (-T * div[fluid])).max() < 1e-13


# ---------------------------------------------------------------------------
# P13: delta-theta (Sec. II) branch table and its vanishing on regular
# interfaces.

def test_delta_theta_branches():
    p = oracle.make_params()
    pref = p.gamma * p.M / (T * p.W)
    g = 0.05
    # inside (phi_n, 1) with lap > 0: (1+s) Y1 with Y1 = 1
    # (s = lap/(|lap| + eps) differs from +-1 by eps/|lap| = 1e-10 at |lap| = 1)
    assert oracle.delta_theta(p, 0.9, g, 1.0) == pytest.approx(2 * pref * g, rel=1e-9)
    # inside (phi_n, 1) with lap < 0: Y2 = 0 -> no correction (regular interface)
    assert abs(oracle.delta_theta(p, 0.9, g, -1.0)) < 1e-9 * abs(pref * g)
    # inside (0, phi_m) with lap < 0: (1-s) Y2 with Y2 = 1
    assert oracle.delta_theta(p, 0.1, g, -1.0) == pytest.approx(2 * pref * g, rel=1e-9)
    # inside (0, phi_m) with lap > 0: Y1 = 0 -> none
    assert abs(oracle.delta_theta(p, 0.1, g, 1.0)) < 1e-9 * abs(pref * g)
    # mid-interface: both Y vanish
    assert oracle.delta_theta(p, 0.5, g, 1e-3) == 0.0
    assert oracle.delta_theta(p, 0.5, g, -1e-3) == 0.0
    # ramps of width D at the ends: F((phi - phi_n)/D) = 1/2
    assert oracle.delta_theta(p, 0.8 + 0.5e-4, g, 1.0) == pytest.approx(pref * g * 2 * 0.5, rel=1e-6)
    # no gradient, no correction
    assert oracle.delta_theta(p, 0.9, 0.0, 1e-3) == 0.0


def test_delta_theta_zero_on_tanh_profile():
    """A planar equilibrium profile has lap(phi) < 0 where phi > 1/2 and > 0
    where phi < 1/2 (Sec. II: the correction stays off on regular interfaces,
    up to the eps regularisation of s, which leaves |delta-theta| << theta)."""
    p = oracle.make_params()
    y = np.arange(40.0)
    phi = W.tanh_profile(19.5 - y, 4.0)
    lap = np.zeros_like(phi)
    lap[1:-1] = phi[2:] - 2 * phi[1:-1] + phi[:-2]
    for j in range(2, 38):
        gn = abs(phi[j + 1] - phi[j - 1]) / 2
        full = abs(p.gamma * p.M / (T * p.W) * gn)      # strength with a Y-term switched on
        assert abs(oracle.delta_theta(p, phi[j], gn, lap[j])) <= 1e-5 * full


# ---------------------------------------------------------------------------
# P5 / P6: a uniform state is a fixed point (rest) and moves unchanged
# (uniform flow): all stencils vanish and streaming of a uniform field is the
# identity.

@pytest.mark.parametrize("lat,shape", [("D2Q9", (8, 8, 1)), ("D3Q27", (5, 4, 4))])
@pytest.mark.parametrize("phi0", [0.0, 0.37, 1.0])
def test_rest_and_uniform_flow(lat, shape, phi0):
    nx, ny, nz = shape
    d = 2 if lat == "D2Q9" else 3
    for U in ([0.0, 0.0, 0.0], [0.03, -0.02, 0.01]):
        o = oracle.Oracle(lat, shape, oracle.make_params())
        g = (nz, ny, nx)
        u0 = np.zeros((3,) + g)
        for a in range(d):
            u0[a] = U[a]
        o.init(np.full(g, phi0), np.full(g, 2e-4), u0)
        o.step(50)
        phi, P, u = o.fields()
        assert np.abs(phi - phi0).max() < 50 * 10 * EPS
        assert np.abs(P - 2e-4).max() < 1e-15
        for a in range(d):
            assert np.abs(u[a] - U[a]).max() < 1e-15


# ---------------------------------------------------------------------------
# P7: phase mass sum(phi) is conserved: sum h_eq = phi (P1), the BGK step
# conserves sum h, periodic streaming and halfway bounce-back permute.

def test_mass_conservation_droplet():
    c = W.droplet_2d(48, 12.0)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
    o.init(c.phi0, c.P0, c.u0[:2])
    m0 = o.fields()[0].sum()
    o.step(1000)
    m1 = o.fields()[0].sum()
    assert abs(m1 / m0 - 1) < 1000 * 9 * EPS


def test_mass_conservation_walls():
    c = W.poiseuille_2d(nx=8, ny=24, g=1e-6)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params), periodic=c.periodic,
                      solid=c.solid)
    o.init(c.phi0, c.P0, c.u0[:2])
    m0 = o.fields()[0].sum()
    o.step(1000)
    m1 = o.fields()[0].sum()
    assert abs(m1 / m0 - 1) < 1000 * 9 * EPS


# ---------------------------------------------------------------------------
# P8: no absolute-pressure dependence (Sec. I, the P0 = 0.01 vs 1.0 static
# droplet test): a constant c added to P0 enters only g_ist through
# P/(rho_ref T); phi and u are unchanged and P is shifted by c.

def test_absolute_pressure_independence():
    c = W.droplet_2d(40, 10.0)
    runs = []
    for P0 in (0.01, 1.0):
        o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
        o.init(c.phi0, c.P0 + P0, c.u0[:2])
        o.step(40)
        runs.append(o.fields())
    (f1, P1, u1), (f2, P2, u2) = runs
    assert np.abs(f1 - f2).max() < 1e-12
    assert np.abs(u1 - u2).max() < 1e-11
    assert np.abs(P2 - P1 - 0.99).max() < 1e-12


# ---------------------------------------------------------------------------
# P9: two-layer Poiseuille flow (Sec. III.B): mu_k u'' = -rho_k g, u = 0 at
# the walls, u and mu u' continuous at the interface.  From rest to steady
# state in a 32-wide channel; the heavy layer follows the sharp-interface
# profile, the light layer is stiffened by the diffuse interface (width W)
# and is compared only away from it.

def test_single_phase_poiseuille_parabola():
    nu = 0.05
    c = W.poiseuille_2d(nx=1, ny=34, g=1e-6, nu_w=nu, nu_a=nu, start_analytic=False)
    phi = np.where(c.solid.astype(bool), 0.0, 1.0)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params), periodic=c.periodic,
                      solid=c.solid)
    o.init(phi, c.P0, c.u0[:2])
    o.step(60000)
    ux = o.fields()[2][0, 0, :, 0]
    y = np.arange(34.0)
    want = 1e-6 / (2 * nu) * (y - 0.5) * (32.5 - y)
    assert np.abs(ux[1:-1] - want[1:-1]).max() < 0.01 * want.max()


def test_two_layer_poiseuille():
    c = W.poiseuille_2d(nx=1, ny=34, g=5e-7, nu_w=0.011, nu_a=0.167, start_analytic=False)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params), periodic=c.periodic,
                      solid=c.solid)
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(150000)
    ux = o.fields()[2][0, 0, :, 0]
    an = c.meta["analytic"]
    heavy = slice(1, int(c.meta["y_int"] - 4))        # liquid, more than W from the interface
    assert np.abs(ux[heavy] - an[heavy]).max() < 0.03 * an.max()
    assert np.abs(ux).max() == pytest.approx(an.max(), rel=0.05)
    assert np.all(np.isfinite(ux))


# ---------------------------------------------------------------------------
# P10: Laplace law (Sec. III.A): dP = sigma / R in 2D.

def test_laplace_law():
    c = W.droplet_2d(64, 16.0)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(10000)
    phi, P, u = o.fields()
    x, y, _ = W.grid_coords(64, 64, 1)
    R = np.sqrt(phi.sum() / np.pi)
    r = np.sqrt((x - 31.5) ** 2 + (y - 31.5) ** 2)
    dP = P[r < R / 2].mean() - P[r > R + 2 * 4.0].mean()
    assert abs(dP * R / 1e-3 - 1) < 0.05
    assert np.abs(u).max() < 1e-4          # spurious currents well below the capillary scale


# ---------------------------------------------------------------------------
# P11: Galilean invariance (Sec. I and III.A): a droplet in a uniform stream
# u_x = 0.025 is the static droplet in the moving frame; after 1280 steps it
# has moved 32 sites and keeps its shape.

def test_galilean_invariance():
    res = []
    for ux in (0.0, 0.025):
        c = W.droplet_2d(80, 16.0, ux=ux)
        o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
        o.init(c.phi0, c.P0, c.u0[:2])
        o.step(1280)
        res.append(o.fields()[0][0])
    static, moving = res
    x = np.arange(80.0)
    def cx(f):
        # centroid on a periodic axis via the phase of the first Fourier mode
        m = f.sum(axis=0)
        return (np.angle((m * np.exp(2j * np.pi * x / 80)).sum()) * 80 / (2 * np.pi)) % 80
    shift = (cx(moving) - cx(static)) % 80
    assert shift == pytest.approx(32.0, abs=0.5)
    assert np.abs(np.roll(static, 32, axis=1) - moving).max() < 0.05


# ---------------------------------------------------------------------------
# P12: D3Q27 weights factor as w(cx) w(cy) w(cz), so on z-uniform data the
# D3Q27 step reduces exactly to D2Q9 (with the printed, full-trace filter;
# the trace-free projection depends on d and breaks the reduction).

@pytest.mark.parametrize("nz", [1, 3])
def test_d3q27_reduces_to_d2q9(nz):
    c = W.droplet_2d(24, 7.0, center=(11.2, 12.1), ux=0.01, nu_w=0.1, filter_full_trace=1)
    o3 = oracle.Oracle("D3Q27", (24, 24, nz), oracle.make_params(**c.params))
    o3.init(np.repeat(c.phi0, nz, 0), np.repeat(c.P0, nz, 0), np.repeat(c.u0, nz, axis=1))
    o2 = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
    o2.init(c.phi0, c.P0, c.u0[:2])
    o2.step(40)
    o3.step(40)
    a, b = o2.fields(), o3.fields()
    for k in range(nz):
        assert np.abs(b[0][k] - a[0][0]).max() < 1e-13
        assert np.abs(b[1][k] - a[1][0]).max() < 1e-12 * np.abs(a[1]).max()
        assert np.abs(b[2][:2, k] - a[2][:2, 0]).max() < 1e-12 * np.abs(a[2]).max()
        assert np.abs(b[2][2]).max() < 1e-15


# ---------------------------------------------------------------------------
# P14: mirror symmetry of symmetric data under central stencils.

def test_mirror_symmetry():
    c = W.droplet_2d(48, 12.0)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params))
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(50)
    phi, P, u = o.fields()
    f = phi[0]
    assert np.abs(f - f[:, ::-1]).max() < 1e-10
    assert np.abs(f - f.T).max() < 1e-10
    assert np.abs(u[0, 0] + u[0, 0][:, ::-1]).max() < 1e-12


# ---------------------------------------------------------------------------
# P15: independent NumPy transcription (D2Q9, periodic) agrees.

def test_numpy_crosscheck():
    c = W.droplet_2d(16, 5.0, center=(7.3, 8.1), ux=0.01)
    r = W.uniform_pm1(7, 3 * 256).reshape(3, 16, 16)
    prm = dict(c.params)
    prm["g_ext"] = (1e-5, -2e-5, 0.0)
    u0 = np.zeros((2, 1, 16, 16))
    u0[0, 0] = 0.01 + 1e-3 * r[0]
    u0[1, 0] = 1e-3 * r[1]
    P0 = 1e-4 * r[2][None]
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**prm))
    o.init(c.phi0, P0, u0)
    x = CrossCheck2D(prm, c.phi0[0], P0[0], u0[0, 0], u0[1, 0])
    o.step(20)
    x.step(20)
    phi, P, u = o.fields()
    f2, P2, ux2, uy2 = x.fields()
    assert np.abs(phi[0] - f2).max() < 1e-13
    assert np.abs(P[0] - P2).max() < 1e-12 * np.abs(P2).max()
    assert np.abs(u[0, 0] - ux2).max() < 1e-13 * np.abs(ux2).max()
    assert np.abs(u[1, 0] - uy2).max() < 1e-13 * np.abs(ux2).max()


# ---------------------------------------------------------------------------
# Linear stability of the step (the reason for the trace-free reading of Pi):
# Jacobian of one oracle step around a uniform state, spectral radius.

def _spectral_radius(phi_val, nu, full_trace, n=8, coupling_unew=0):
    p = oracle.make_params(nu_w=nu, nu_a=nu, filter_full_trace=1 if full_trace else 0,
                           coupling_unew=coupling_unew)
    o = oracle.Oracle("D2Q9", (n, n, 1), p)
    o.init(np.full((1, n, n), phi_val), np.zeros((1, n, n)), np.zeros((2, 1, n, n)))
    h0, g0, P0, u0 = o.get_state()
    x0 = np.concatenate([h0.ravel(), g0.ravel(), P0.ravel(), u0.ravel()])
    Q, N = 9, n * n

    def f(x):
        o.set_state(x[:Q * N], x[Q * N:2 * Q * N], x[2 * Q * N:2 * Q * N + N], x[2 * Q * N + N:])
        o.step(1)
        return np.concatenate([a.ravel() for a in o.get_state()])

    f0 = f(x0)
    J = np.empty((x0.size, x0.size))
    for j in range(x0.size):
        x = x0.copy()
        x[j] += 1e-7
        J[:, j] = (f(x) - f0) / 1e-7
    return np.abs(np.linalg.eigvals(J)).max()


@pytest.mark.parametrize("phi_val", [0.0, 1.0])
def test_linear_stability_adopted_reading(phi_val):
    for nu in (3.67e-4, 8.35e-3, 0.0167):
        assert _spectral_radius(phi_val, nu, full_trace=False) < 1 + 1e-6


def test_printed_full_trace_filter_is_unstable():
    assert _spectral_radius(1.0, 0.0167, full_trace=True) > 1.01


def test_unew_coupling_is_unstable_at_low_viscosity():
    """The alternative reading of the pressure formula's omega-term (Sec. II),
    u^{n+1}(x - c_i) in place of u^n(x - c_i): the liquid (phi = 1) grows at
    the lowest viscosity the paper simulates, nu = 3.67e-4, where the adopted
    reading is stable (test_linear_stability_adopted_reading); at nu =
    0.0167 both are stable."""
    assert _spectral_radius(1.0, 3.67e-4, full_trace=False, coupling_unew=1) > 1.003
    assert _spectral_radius(1.0, 0.0167, full_trace=False, coupling_unew=1) < 1 + 1e-6


# ---------------------------------------------------------------------------
# P16: the rising bubble's early rise against the added-mass closed form

@pytest.mark.slow
@pytest.mark.parametrize("case", [1, 2])
def test_bubble_early_rise_added_mass(case):
    """Sec. III.D, at half size (100 x 200, R = 25; the time scale
    2R / sqrt(2Rg) is 60600 steps).  A 2D cylinder of density rho_2 in a
    liquid of density rho_1 starts to accelerate at a = g (rho_1 - rho_2) /
    (rho_2 + rho_1) (added mass of a circular cylinder, C_a = 1).  Drag, the
    pressure waves that set up the hydrostatic state and the finite interface
    only slow it, so after 10000 steps the rise lies below a t^2 / 2, and
    this early not far below it.  A reversed gravity, a missing buoyancy
    term or a doubled force falls outside [0.3, 1.02] of that value."""
    c = W.rising_bubble_2d(case, nx=100, ny=200, R=25.0, center=(50.0, 50.0))
    o = oracle.Oracle(c.lattice, c.shape, oracle.make_params(**c.params), periodic=c.periodic, solid=c.solid)
    o.init(c.phi0, c.P0, c.u0)

    def centroid_y(phi):
        b = ((1.0 - phi) * (1 - c.solid))[0, 10:120, 10:90]
        ys = np.arange(10, 120)[:, None]
        return float((b * ys).sum() / b.sum())

    t = 10000
    o.step(t)
    rise = centroid_y(o.fields()[0]) - centroid_y(c.phi0)
    a = c.meta["g"] * (c.meta["rho1"] - c.meta["rho2"]) / (c.meta["rho2"] + c.meta["rho1"])
    ideal = 0.5 * a * t * t
    assert 0.3 * ideal <= rise <= 1.02 * ideal, f"rise {rise:.4f} vs inviscid {ideal:.4f}"


# ---------------------------------------------------------------------------
# P17: shear-wave decay.  The target momentum equation (Sec. I, with the
# stress tensor printed there) reduces for a small transverse wave
# u_x = U sin(k y) in a single phase (grad rho = 0, div u = 0) to
# du/dt = nu d2u/dy2, so the amplitude decays as exp(-nu k^2 t).  The
# viscosity is the local one of Eq. tau_interpolate, nu = T (tau_mix - 1/2),
# with tau_mix linear in phi: a slip in tau_k = nu_k / T + 1/2, in the mixing,
# in nu, or in the filter's factor (1 - 1/tau) or w_i / (2 T^2) moves the rate
# by far more than the 0.5 % allowed (the O(k^2) lattice correction at k =
# 2 pi / 64 is below 0.1 %).

def _mode_amplitude(f, mode):
    return float((f * mode).sum() / (mode * mode).sum())


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("phi_val,nu_w,nu_a,nu_mix", [
    (1.0, 0.0167, 0.167, 0.0167),
    (0.0, 0.0167, 0.167, 0.167),
    (0.3, 0.0167, 0.167, 0.167 + 0.3 * (0.0167 - 0.167)),
    (1.0, 0.05, 0.05, 0.05),
    (1.003, 0.0167, 0.167, 0.0167),
    (-0.003, 0.0167, 0.167, 0.167),
])
def test_shear_wave_decay(lat, phi_val, nu_w, nu_a, nu_mix):
    """A uniform mixture (phi = 0.3) checks the linear mixing of tau.  It is
    not a steady state of the phase field with the paper's eps = 1e-10: the
    normal n = grad phi / (|grad phi| + eps) turns rounding noise into unit
    vectors and the theta n term of h_eq then separates the mixture (as the
    conservative Allen-Cahn equation does).  With eps = 1 the theta n term is
    a weak diffusion and the mixture stays uniform; the g step does not use
    eps.  phi = 1.003 and -0.003 check the reading that clamps phi to [0, 1]
    for the material properties: the bulk viscosities stay nu_w and nu_a
    (unclamped, 1.003 would give 2.7 % less, and -0.003 a negative
    density)."""
    ny = 64
    shape = (4, ny, 1) if lat == "D2Q9" else (4, ny, 2)
    nx, _, nz = shape
    extra = {"eps": 1.0} if phi_val not in (0.0, 1.0) else {}
    o = oracle.Oracle(lat, shape, oracle.make_params(nu_w=nu_w, nu_a=nu_a, **extra))
    k = 2 * np.pi / ny
    y = np.broadcast_to(np.arange(ny, dtype=float)[None, :, None], (nz, ny, nx))
    mode = np.sin(k * y)
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = 1e-4 * mode
    o.init(np.full((nz, ny, nx), phi_val), np.zeros((nz, ny, nx)), u0)
    t0, t1 = 200, 2000
    o.step(t0)
    a0 = _mode_amplitude(o.fields()[2][0], mode)
    o.step(t1 - t0)
    a1 = _mode_amplitude(o.fields()[2][0], mode)
    rate = -np.log(a1 / a0) / (t1 - t0)
    assert rate == pytest.approx(nu_mix * k * k, rel=5e-3)


# ---------------------------------------------------------------------------
# P18: plane acoustic wave.  Sec. I: the pressure equation and the momentum
# equation combine into a sound wave of speed sqrt(T).  A standing wave
# P = dP cos(k x), u = 0 in a single phase oscillates at omega = sqrt(T) k
# and decays as exp(-Gamma k^2 t / 2), Gamma the longitudinal viscosity.
# Gamma follows from the collision operator by a Chapman-Enskog expansion
# (Sec. I, feq_expansion; the filter of Eq. LB_filter_col):
#   - the filter relaxes the trace-free part of Pi with tau_mix, which gives
#     the shear stress rho nu (grad u + grad u^T - (2/d) div u delta);
#   - with the adopted reading the trace of Pi relaxes to equilibrium every
#     step (a relaxation time of 1), which adds rho (T/2)(2/d) div u delta;
#   - the B term of g_eq puts B div u delta into the equilibrium momentum
#     flux, i.e. - rho B div u delta into the stress.
# For a longitudinal wave that is
#   Gamma = (4/3 - 2/d) nu + (2/3) lambda_b + T (1/d - 1/2).
# With the printed filter (full Pi relaxed with tau_mix) the stress is
# rho nu (grad u + grad u^T) - rho B div u delta, i.e.
#   Gamma = (4/3) nu + (2/3) lambda_b - T/2,
# which is negative at low nu (the printed form's instability).  The target
# stress of Sec. I has Gamma = (4/3) nu + (2/3) lambda_b: the adopted reading
# recovers its lambda_b term exactly and its nu term less (2/d) nu (d = 2) or
# (2/3) nu + T/6 (d = 3).  A sign or coefficient slip in B (its nu, its
# lambda_b, its T/2), in the trace handling or in K_i and the omega-term of P
# (which set the sound speed) moves Gamma by 15 % or more; the lattice
# correction at k = 2 pi / 64 is below 2 %.

def _acoustic(lat, phi_val, nu, lam, full_trace, n=64, steps=3000, every=3, **extra):
    from scipy.optimize import curve_fit

    o = oracle.Oracle(lat, (n, 1, 1), oracle.make_params(nu_w=nu, nu_a=nu, lambda_b=lam,
                                                         filter_full_trace=full_trace, **extra))
    k = 2 * np.pi / n
    mode = np.cos(k * np.arange(n, dtype=float))
    dP = 1e-6
    o.init(np.full((1, 1, n), phi_val), (dP * mode)[None, None, :], np.zeros((3, 1, 1, n)))
    t, amp = [], []
    for s in range(every, steps + 1, every):
        o.step(every)
        t.append(s)
        amp.append(_mode_amplitude(o.fields()[1][0, 0], mode) / dP)
    t, amp = np.array(t, float), np.array(amp)

    def model(t, A, gam, om, ph):
        return A * np.exp(-gam * t) * np.cos(om * t + ph)

    (A, gam, om, ph), _ = curve_fit(model, t, amp, p0=[1.0, 1e-4, np.sqrt(T) * k, 0.0])
    return 2 * gam / k ** 2, om / k


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
@pytest.mark.parametrize("phi_val", [0.0, 1.0])
@pytest.mark.parametrize("nu,lam", [(0.0167, 1.0 / 6.0), (0.167, 0.05), (0.05, 0.3)])
def test_acoustic_wave_speed_and_damping(lat, phi_val, nu, lam):
    d = 2 if lat == "D2Q9" else 3
    gamma, c = _acoustic(lat, phi_val, nu, lam, full_trace=0)
    assert c == pytest.approx(np.sqrt(T), rel=5e-3)
    want = (4.0 / 3.0 - 2.0 / d) * nu + (2.0 / 3.0) * lam + T * (1.0 / d - 0.5)
    assert gamma == pytest.approx(want, rel=3e-2)


@pytest.mark.parametrize("phi_val", [1.0, 0.5])
def test_acoustic_wave_density_ratio_10(phi_val):
    """At a density ratio of 10 the pressure formula's (1 + omega) rho_ref
    must equal rho (omega of Sec. II with omega_max = rho_ratio and the
    linear rho(phi) reading); a slip there (omega_max in place of
    omega_max - 1, say) moves the sound speed by 5 %.  phi = 0.5 is a
    uniform mixture, kept uniform with eps = 1 (see the shear-wave pin)."""
    extra = {"rho_a": 0.1} if phi_val == 1.0 else {"rho_a": 0.1, "eps": 1.0}
    gamma, c = _acoustic("D2Q9", phi_val, 0.0167, 1.0 / 6.0, full_trace=0, **extra)
    assert c == pytest.approx(np.sqrt(T), rel=5e-3)
    assert gamma == pytest.approx(0.0167 / 3 + 2.0 / 18.0, rel=3e-2)


def test_acoustic_wave_printed_filter():
    gamma, c = _acoustic("D2Q9", 1.0, 0.167, 1.0 / 6.0, full_trace=1)
    assert c == pytest.approx(np.sqrt(T), rel=5e-3)
    assert gamma == pytest.approx(4.0 / 3.0 * 0.167 + 2.0 / 9.0 * 0.5 - T / 2, rel=3e-2)


# ---------------------------------------------------------------------------
# P19: two-layer channel through the diffuse interface.  In steady layered
# flow the momentum equation of Sec. I reduces to d/dy (rho nu du/dy) =
# -rho g (div u = 0, so only the shear part of the stress acts).  The LB
# carries nu d2u/dy2 through the filter and the rest, nu (du/dy)(drho/dy) /
# rho, through the sigma . grad rho / rho^2 term of g_eq, so the steady
# profile must solve that equation with the step's own phi(y), rho(phi) and
# nu(phi) (halfway walls: u = 0 at y = 1/2 and ny - 3/2).  Across the
# interface rho changes by 1000 times, so a wrong sign or factor in the stress
# sigma_lm, in grad rho or in the rho^2 of that term leaves the light layer's
# slope far from the solution; the lattice's own error is 1.5 %.

def test_two_layer_channel_diffuse_interface_profile():
    ny, g, nu_w, nu_a = 34, 5e-7, 0.011, 0.167
    c = W.poiseuille_2d(nx=1, ny=ny, g=g, nu_w=nu_w, nu_a=nu_a, start_analytic=False)
    o = oracle.Oracle("D2Q9", c.shape, oracle.make_params(**c.params), periodic=c.periodic, solid=c.solid)
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(150000)
    phi, _, u = o.fields()
    f = slice(1, ny - 1)
    ux, ph = u[0, 0, f, 0], phi[0, f, 0]
    p = c.params
    phh = np.clip(ph, 0.0, 1.0)
    rho = p["rho_a"] + phh * (p["rho_w"] - p["rho_a"])
    tau = (3 * nu_a + 0.5) + phh * ((3 * nu_w + 0.5) - (3 * nu_a + 0.5))
    mu = rho * (tau - 0.5) / 3
    # conservative three-point form of d/dy (mu du/dy) = -rho g; a halfway
    # wall is a ghost value -u one site out
    n = ny - 2
    A = np.zeros((n, n))
    muh = 0.5 * (mu[1:] + mu[:-1])
    for j in range(n):
        if j > 0:
            A[j, j - 1] += muh[j - 1]
            A[j, j] -= muh[j - 1]
        else:
            A[j, j] -= 2 * mu[0]
        if j < n - 1:
            A[j, j + 1] += muh[j]
            A[j, j] -= muh[j]
        else:
            A[j, j] -= 2 * mu[-1]
    want = np.linalg.solve(A, -rho * g)
    assert np.abs(ux - want).max() < 0.03 * want.max()
    light = ph < 0.01
    slope = np.polyfit(np.arange(light.sum()), ux[light], 1)[0]
    slope_want = np.polyfit(np.arange(light.sum()), want[light], 1)[0]
    assert slope == pytest.approx(slope_want, rel=0.03)


# ---------------------------------------------------------------------------
# P20: phase-field diffusion.  The phase-field LB recovers the conservative
# Allen-Cahn equation of Sec. II, d phi/dt + div(phi u) = div[M (grad phi -
# theta n)], with the mobility M = T (tau_phi - 1/2) of Eq.
# LB_phi_filter_col.  A small wave phi = 1.001 + 5e-4 sin(k x) with
# sigma = 0 (no capillary force, so u stays 0) and eps = 1 (so the theta n
# term, quadratic in the perturbation, is negligible) decays at M k^2.  A
# slip in tau_phi, in the BGK relaxation of h or in h_eq's first moment
# (phi u + theta T n) moves the rate by more than the 0.3 % allowed; the
# lattice and theta corrections are 0.1 - 0.17 % here.

@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
@pytest.mark.parametrize("M", [0.166, 0.05, 0.3])
def test_phase_field_diffusion(lat, M):
    n = 128
    o = oracle.Oracle(lat, (n, 1, 1), oracle.make_params(sigma=0.0, eps=1.0, M=M))
    k = 2 * np.pi / n
    mode = np.sin(k * np.arange(n, dtype=float))
    base = 1.001
    o.init((base + 5e-4 * mode)[None, None, :], np.zeros((1, 1, n)), np.zeros((3, 1, 1, n)))
    t0, t1 = 200, 8000
    o.step(t0)
    a0 = _mode_amplitude(o.fields()[0][0, 0] - base, mode)
    o.step(t1 - t0)
    phi, _, u = o.fields()
    a1 = _mode_amplitude(phi[0, 0] - base, mode)
    assert np.abs(u).max() == 0.0
    assert -np.log(a1 / a0) / (t1 - t0) == pytest.approx(M * k * k, rel=3e-3)
