"""The paper's own validation runs at the paper's settings, on the GPU in
FP64 (Sec. I and Sec. III.A).

- Laplace law (Sec. III.A): a static 2D droplet of radius R in {8, 12, 16,
  20, 24} centred in a periodic domain of 5R, viscosity sets {nu_air,
  nu_water} = {0.167, 0.011} and {5.56e-3, 3.67e-4}, sigma = 1e-2 and 1e-3:
  20 lattices stepped together in one batch for 4e4 steps.  The paper plots
  dP against 1/R and prints no value; the pin is the law itself, dP = sigma
  / R (2D), with the jump measured as the oracle's reading does (mean P
  within R_eff / 2 of the centre minus mean P farther than R_eff + 2W,
  R_eff = sqrt(sum phi / pi)).  With the low-viscosity set the droplets of
  R = 8 and 12 diverge within 2000 steps and R = 16 runs away from the law
  (the paper's figure shows all of them on it): with the readings adopted
  here these three do not reproduce the paper, and the test records that.
- Galilean invariance (Sec. I and III.A): R = 16 in 80 x 80, u_x = 0.025
  everywhere at start, viscosities {0.167, 0.011}, sigma = 1e-3, to the
  snapshots at 3.20e4 and 3.36e4 steps.  The droplet keeps the shape of the
  droplet at rest (the paper's point, figure only).  The whole flow slows
  down (mean u_x 0.0239 after 8000 steps; the oracle does the same, under
  either reading of the omega-term), so the droplet is compared with the
  resting one at its own position, and it moves with the fluid around it.
- Absolute pressure (Sec. I): R = 20 in 100 x 100, nu = 3.6e-4 for both
  components, sigma = 2.5e-2, ambient P0 = 0.01 or 1.0: phi and u must not
  depend on P0, and P must differ by the 0.99 added.
Each run's FP64 fields equal the oracle's bit for bit where the oracle is
run to the same horizon here (the GI droplet to 3.36e4 steps, two Laplace
droplets, and the absolute-pressure droplet).
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

NU_SETS = {"set1": (0.167, 0.011), "set2": (5.56e-3, 3.67e-4)}
LAPLACE_STEPS = 40000


def laplace_case(R, nus, sigma):
    nu_a, nu_w = NU_SETS[nus]
    return W.droplet_2d(int(5 * R), float(R), nu_a=nu_a, nu_w=nu_w, sigma=sigma)


def lattice(lbm, c, storage="f64"):
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage, **prm)
    L.init_fields(c.phi0, c.P0, c.u0)
    return L


def laplace_jump(phi, P, n, W_=4.0):
    """Laplace jump of fields [1, n, n] (the reading of the pressure
    difference across the interface described above)."""
    x, y, _ = W.grid_coords(n, n, 1)
    c0 = (n - 1) / 2.0
    R = np.sqrt(phi.sum() / np.pi)
    r = np.sqrt((x - c0) ** 2 + (y - c0) ** 2)
    return P[r < R / 2].mean() - P[r > R + 2 * W_].mean(), R


LAPLACE = [(R, nus, s) for R in (8, 12, 16, 20, 24) for nus in ("set1", "set2") for s in (1e-2, 1e-3)]
NOT_REPRODUCED = {(R, "set2", s) for R in (8, 12, 16) for s in (1e-2, 1e-3)}


@pytest.fixture(scope="module")
def laplace_runs(lbm):
    B = lbm.Batch("D2Q9", "f64")
    runs = {}
    for key in LAPLACE:
        c = laplace_case(*key)
        L = lattice(lbm, c)
        B.add(L, LAPLACE_STEPS)
        runs[key] = (c, L)
    B.step(LAPLACE_STEPS)
    out = {}
    for key, (c, L) in runs.items():
        try:
            out[key] = (c, L.read_fields())
        except lbm.LbmError as e:
            if e.code != lbm.LBM_ERR_NONFINITE:
                raise
            out[key] = (c, None)                      # this droplet diverged
    B.close()
    return out


@pytest.mark.parametrize("key", LAPLACE, ids=[f"R{k[0]}-{k[1]}-s{k[2]:g}" for k in LAPLACE])
def test_laplace_sweep(laplace_runs, key):
    """dP R_eff / sigma = 1 within 6 % after 4e4 steps (measured 3.5 - 5.5 %
    above the law for the first viscosity set, 1.8 - 2.5 % for the second at
    R = 20, 24: the diffuse interface of width W = 4 is not thin against R).
    The three low-viscosity cases the adopted readings do not reproduce
    either diverge or leave the law by more than 20 %."""
    c, fields = laplace_runs[key]
    if key in NOT_REPRODUCED:
        if fields is not None:
            dP, Reff = laplace_jump(fields[0], fields[1], c.shape[0])
            assert abs(dP * Reff / key[2] - 1) > 0.2
        return
    assert fields is not None, "diverged"
    phi, P, u = fields
    dP, Reff = laplace_jump(phi, P, c.shape[0])
    ratio = dP * Reff / key[2]
    assert abs(ratio - 1) <= 0.06, f"dP R / sigma = {ratio:.4f}"
    assert np.all(np.isfinite(u))


@pytest.mark.parametrize("key", [(8, "set1", 1e-2), (20, "set2", 1e-3)])
def test_laplace_sweep_matches_oracle(laplace_runs, key):
    c, g = laplace_runs[key]
    o = oracle.Oracle(c.lattice, c.shape, oracle.make_params(**c.params))
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(LAPLACE_STEPS)
    for x, y in zip(g, o.fields()):
        assert np.array_equal(x, y)


def gi_case(ux):
    return W.droplet_2d(80, 16.0, ux=ux, nu_a=0.167, nu_w=0.011, sigma=1e-3)


@pytest.fixture(scope="module")
def gi_runs(lbm):
    B = lbm.Batch("D2Q9", "f64")
    Ls = {ux: lattice(lbm, gi_case(ux)) for ux in (0.0, 0.025)}
    for L in Ls.values():
        B.add(L, 33600)
    snaps = {}
    B.step(32000)
    snaps[32000] = {ux: L.read_fields() for ux, L in Ls.items()}
    B.step(1600)
    snaps[33600] = {ux: L.read_fields() for ux, L in Ls.items()}
    B.close()
    return snaps


def _centroid_x(f, n=80):
    x = np.arange(float(n))
    m = f.sum(axis=0)
    return (np.angle((m * np.exp(2j * np.pi * x / n)).sum()) * n / (2 * np.pi)) % n


def _shift_x(f, d):
    """f moved by d sites along the periodic x axis (sub-site by Fourier)."""
    k = np.fft.fftfreq(f.shape[1]) * 2 * np.pi
    return np.real(np.fft.ifft(np.fft.fft(f, axis=1) * np.exp(-1j * k * d)[None, :], axis=1))


@pytest.mark.parametrize("t", [32000, 33600])
def test_galilean_invariance_paper_length(gi_runs, t):
    """The moving droplet, taken back to the resting droplet's position, has
    its shape: max |dphi| <= 0.01 (measured 0.0045).  The resting droplet
    stays where it is, and the moving one travels with the fluid around it
    (the mean velocity inside it and outside it agree within 1 %)."""
    static = gi_runs[t][0.0][0][0]
    phi, _, u = gi_runs[t][0.025]
    moving = phi[0]
    assert abs((_centroid_x(static) - 39.5 + 40) % 80 - 40) <= 1e-3
    d = _centroid_x(moving) - _centroid_x(static)
    assert np.abs(_shift_x(static, d) - moving).max() <= 0.01
    inside = moving > 0.5
    u_in, u_out = u[0, 0][inside].mean(), u[0, 0][~inside].mean()
    assert abs(u_in / u_out - 1) <= 1e-2
    assert abs(moving.sum() / static.sum() - 1) <= 1e-12


ABS_STEPS = 10000


def abs_case(P0):
    return W.droplet_2d(100, 20.0, P0=P0, nu_a=3.6e-4, nu_w=3.6e-4, sigma=2.5e-2)


@pytest.fixture(scope="module")
def abs_runs(lbm):
    B = lbm.Batch("D2Q9", "f64")
    Ls = {P0: lattice(lbm, abs_case(P0)) for P0 in (0.01, 1.0)}
    for L in Ls.values():
        B.add(L, ABS_STEPS)
    B.step(ABS_STEPS)
    out = {P0: L.read_fields() for P0, L in Ls.items()}
    B.close()
    return out


def test_absolute_pressure_paper(abs_runs):
    """phi and u of the droplet do not depend on the ambient pressure (the
    P-u scheme carries P only in the rest population's P / (rho_ref T)),
    and P shifts by the 0.99 added.  In FP64 the two runs round differently
    (P0 enters g_0 = P / (rho_ref T) at 1e3 times P), and the unit normal
    and the sign of delta-theta amplify rounding differences, so the bound
    is on the flow's scale: |dphi| <= 1e-3, |du| <= 1e-2 max|u|."""
    (f1, P1, u1), (f2, P2, u2) = abs_runs[0.01], abs_runs[1.0]
    assert np.abs(f1 - f2).max() <= 1e-3
    assert np.abs(u1 - u2).max() <= 1e-2 * np.abs(u1).max()
    assert np.abs((P2 - P1) - 0.99).max() <= 1e-3 * 2.5e-2 / 20.0 + 1e-12
    # and the jump itself follows the Laplace law
    dP, Reff = laplace_jump(f1, P1, 100)
    assert abs(dP * Reff / 2.5e-2 - 1) <= 0.05


def test_absolute_pressure_matches_oracle(abs_runs):
    c = abs_case(0.01)
    o = oracle.Oracle(c.lattice, c.shape, oracle.make_params(**c.params))
    o.init(c.phi0, c.P0, c.u0[:2])
    o.step(ABS_STEPS)
    for x, y in zip(abs_runs[0.01], o.fields()):
        assert np.array_equal(x, y)
