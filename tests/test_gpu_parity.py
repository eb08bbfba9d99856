"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

FP64 storage: both sides evaluate the paper's formulas in the same order
without FMA contraction, so fields agree to 1e-12 relative per field (the
bar the method's target sets after 1000 steps; in practice bit for bit).
FP32: max|du| <= 1e-5 max|u| and |dP| <= 1e-6 relative, on horizons where
the method's rounding sensitivity (unit normal n at |grad phi| -> 0) has not
amplified FP32 rounding.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def run_gpu(lbm, case, steps, storage="f64", **pkw):
    prm = dict(case.params)
    prm.update(pkw)
    g = prm.pop("g_ext", (0, 0, 0))
    lat = lbm.Lattice(case.lattice, case.shape, periodic=case.periodic, solid=case.solid,
                      storage=storage, g_ext=g, **prm)
    lat.init_fields(case.phi0, case.P0, case.u0)
    lat.step(steps)
    out = lat.read_fields()
    return lat, out


def run_oracle(case, steps, **pkw):
    prm = dict(case.params)
    prm.update(pkw)
    o = oracle.Oracle(case.lattice, case.shape, oracle.make_params(**prm), periodic=case.periodic,
                      solid=case.solid)
    o.init(case.phi0, case.P0, case.u0)
    o.step(steps)
    return o, o.fields()


def assert_fields(gpu, orc, tol, tol_P=None, d=3):
    (f1, P1, u1), (f2, P2, u2) = gpu, orc
    assert np.all(np.isfinite(f1)) and np.all(np.isfinite(P1)) and np.all(np.isfinite(u1))
    assert rel(f1, f2) <= tol, f"phi {rel(f1, f2):.3e}"
    assert rel(P1, P2) <= (tol_P if tol_P is not None else tol), f"P {rel(P1, P2):.3e}"
    assert rel(u1[:d], u2[:d]) <= tol, f"u {rel(u1[:d], u2[:d]):.3e}"


def small_3d(lattice, nx=37, ny=11, nz=13, walls=True):
    """Droplet over a film in a box with ragged tiles; walls at z = 0, nz-1."""
    x, y, z = W.grid_coords(nx, ny, nz)
    zi = 3.5
    cx, cy, cz = (nx - 1) / 2.0 + 0.3, (ny - 1) / 2.0 - 0.2, 3.5 + 2.0 + 4.0
    phi_f = W.tanh_profile(zi - z, 4.0)
    phi_d = W.tanh_profile(4.0 - np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2), 4.0)
    phi = np.maximum(phi_f, phi_d)
    solid = np.zeros(phi.shape, np.uint8)
    if walls:
        solid[0] = 1
        solid[-1] = 1
    u = np.zeros((3,) + phi.shape)
    u[2] = -0.02 * phi_d
    u[0] = 0.003
    u[:, solid.astype(bool)] = 0
    phi = np.where(solid.astype(bool), 0.0, phi)
    return W.Case("small3d", lattice, (nx, ny, nz), W.base_params(), phi, 1e-5 * phi, u,
                  (1, 1, 0) if walls else (1, 1, 1), solid if walls else None, 0)


# ---------------------------------------------------------------------------
# FP64: identical arithmetic

@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_init_state_f64(lbm, lat):
    c = W.droplet_2d(20, 5.0) if lat == "D2Q9" else small_3d(lat)
    L, _ = run_gpu(lbm, c, 0)
    o, _ = run_oracle(c, 0)
    h1, g1, P1, u1 = L.get_state()
    h2, g2, P2, u2 = o.get_state()
    assert np.array_equal(h1, h2)
    assert np.array_equal(g1, g2)
    assert np.array_equal(P1, P2)


def test_droplet_2d_f64_1000_steps(lbm):
    """64^2 periodic D2Q9 droplet, R = 16, density ratio 1000 (the small config)."""
    c = W.droplet_2d(64, 16.0)
    _, g = run_gpu(lbm, c, 1000)
    _, o = run_oracle(c, 1000)
    assert_fields(g, o, 1e-12, d=2)


def test_channel_2d_f64_1000_steps(lbm):
    """128 x 256 layered Poiseuille channel with solid rows, body force 1e-7."""
    c = W.poiseuille_2d(128, 256)
    _, g = run_gpu(lbm, c, 1000)
    _, o = run_oracle(c, 1000)
    assert_fields(g, o, 1e-12, d=2)


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_3d_f64_walls_ragged(lbm, lat):
    c = small_3d(lat)
    _, g = run_gpu(lbm, c, 120)
    _, o = run_oracle(c, 120)
    assert_fields(g, o, 1e-12)


def test_3d_f64_periodic_thin(lbm):
    """nz smaller than any z-chunk, nx < one tile, fully periodic."""
    c = small_3d("D3Q27", nx=9, ny=7, nz=5, walls=False)
    _, g = run_gpu(lbm, c, 60)
    _, o = run_oracle(c, 60)
    assert_fields(g, o, 1e-12)


def test_2d_f64_random_solids_closed_box(lbm):
    """Random solid sites, all axes non-periodic (closed by solid outside)."""
    c = W.droplet_2d(41, 9.0, center=(19.3, 21.7), ux=0.01)
    r = (W.uniform_pm1(11, 41 * 41).reshape(1, 41, 41) > 0.93).astype(np.uint8)
    r[:, 15:27, 14:28] = 0
    c.solid = r
    c.periodic = (0, 0, 1)
    c.phi0 = np.where(r.astype(bool), 0.0, c.phi0)
    c.u0[:, r.astype(bool)] = 0.0
    _, g = run_gpu(lbm, c, 300)
    _, o = run_oracle(c, 300)
    assert_fields(g, o, 1e-12, d=2)


def test_full_trace_filter_f64(lbm):
    c = W.droplet_2d(24, 6.0, nu_w=0.1)
    _, g = run_gpu(lbm, c, 100, filter_full_trace=1)
    _, o = run_oracle(c, 100, filter_full_trace=1)
    assert_fields(g, o, 1e-12, d=2)


# ---------------------------------------------------------------------------
# FP32 arithmetic against the FP64 oracle

def test_channel_2d_f32_1000_steps(lbm):
    c = W.poiseuille_2d(128, 256)
    _, g = run_gpu(lbm, c, 1000, storage="f32")
    _, o = run_oracle(c, 1000)
    f1, P1, u1 = g
    f2, P2, u2 = o
    assert np.abs(u1 - u2).max() <= 1e-5 * np.abs(u2).max()
    # P scale: the pressure unit rho_w T u_max^2 of the channel (P itself is ~0 here)
    Pscale = max(np.abs(P2).max(), 1.0 * (1.0 / 3.0) * np.abs(u2).max() ** 2)
    assert np.abs(P1 - P2).max() <= 1e-6 * Pscale
    assert np.abs(f1 - f2).max() <= 1e-5


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
def test_short_horizon_f32(lbm, lat):
    c = W.droplet_2d(48, 12.0, ux=0.01) if lat == "D2Q9" else small_3d(lat)
    _, g = run_gpu(lbm, c, 20, storage="f32")
    _, o = run_oracle(c, 20)
    (f1, P1, u1), (f2, P2, u2) = g, o
    assert np.abs(u1 - u2).max() <= 1e-5 * np.abs(u2).max()
    assert np.abs(P1 - P2).max() <= 1e-6 * max(np.abs(P2).max(), 1e-30) + 1e-12
    assert np.abs(f1 - f2).max() <= 1e-5


# ---------------------------------------------------------------------------
# Subsystems through the ABI

def test_checkpoint_resume_bitwise(lbm):
    c = small_3d("D3Q27", walls=True)
    L1, _ = run_gpu(lbm, c, 20, storage="f32")
    blob = L1.save_state()
    L1.step(15)
    a = L1.read_fields()
    L2 = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f32")
    L2.load_state(blob)
    assert L2.steps_done == 20
    L2.step(15)
    b = L2.read_fields()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_reductions_and_probe(lbm):
    c = W.droplet_2d(48, 12.0)
    L, (phi, P, u) = run_gpu(lbm, c, 200)
    r = L.reduce()
    assert r["fluid_sites"] == 48 * 48
    assert r["mass"] == pytest.approx(phi.sum(), rel=1e-13)
    rho = c.params["rho_a"] + np.clip(phi, 0, 1) * (c.params["rho_w"] - c.params["rho_a"])
    assert r["momentum"][0] == pytest.approx((rho * u[0]).sum(), abs=1e-15 * phi.size)
    # mass is conserved to rounding from the initial state
    assert r["mass"] / c.phi0.sum() - 1 == pytest.approx(0.0, abs=200 * 9 * 2.3e-16)
    # Laplace jump vs numpy on the read-back field
    x, y, _ = W.grid_coords(48, 48, 1)
    rr = np.sqrt((x - 23.5) ** 2 + (y - 23.5) ** 2)
    want = P[rr < 6].mean() - P[rr > 20].mean()
    assert L.pressure_jump((23.5, 23.5, 0.0), 6.0, 20.0) == pytest.approx(want, rel=1e-12, abs=1e-18)
    # probe agrees with the full state
    hs, gs, Ps, us = L.get_state()
    sites = np.array([0, 5, 48 * 20 + 17, 48 * 48 - 1])
    hp, gp, Pp, up = L.probe(sites)
    for j, s in enumerate(sites):
        assert np.array_equal(hp[j], hs.reshape(9, -1)[:, s])
        assert np.array_equal(gp[j], gs.reshape(9, -1)[:, s])
        assert Pp[j] == Ps.reshape(-1)[s]


def test_nonfinite_input_is_reported(lbm):
    """Host-side fault injection: a NaN in the initial field must surface as
    LBM_ERR_NONFINITE from read_fields (no GPU fault involved)."""
    c = W.droplet_2d(32, 8.0)
    phi = c.phi0.copy()
    phi[0, 3, 3] = np.nan
    L = lbm.Lattice("D2Q9", c.shape, storage="f32")
    L.init_fields(phi, c.P0, c.u0)
    L.step(3)
    with pytest.raises(lbm.LbmError) as e:
        L.read_fields()
    assert e.value.code == lbm.LBM_ERR_NONFINITE
    # a fresh init clears the flag
    L.init_fields(c.phi0, c.P0, c.u0)
    L.step(3)
    L.read_fields()


def test_rest_state_gpu(lbm):
    shape = (33, 7, 9)
    g = (9, 7, 33)
    L = lbm.Lattice("D3Q27", shape, storage="f32")
    L.init_fields(np.full(g, 1.0), np.full(g, 3e-4), np.zeros((3,) + g))
    L.step(25)
    phi, P, u = L.read_fields()
    assert np.abs(phi - 1).max() < 1e-6
    assert np.abs(P - 3e-4).max() < 1e-10
    assert np.abs(u).max() < 1e-10
