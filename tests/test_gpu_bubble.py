"""2D rising bubble (Sec. III.D, Table tab_bubblerise): a light bubble
(density 0.22, R = 50) in a 200 x 400 liquid column under gravity, the two
cases of the table (liquid density 2.2 and 220).  Parity with the oracle in
FP64 and FP32, and the early rise against the inviscid added-mass value."""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import assert_fields, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def centroid_y(case, phi):
    """Height of the bubble's centre of mass: weights 1 - phi over a window
    that holds the bubble (x in [30, 170), y in [30, 200)), so that the
    liquid's own small departures from phi = 1 elsewhere do not enter."""
    b = ((1.0 - phi) * (1 - case.solid))[0, 30:200, 30:170]
    ys = np.arange(30, 200)[:, None]
    return float((b * ys).sum() / b.sum())


def interface_heights(phi, x=100):
    """Bottom and top phi = 1/2 crossings of the bubble on the line x = const
    (linear interpolation between sites)."""
    col = phi[0, :, x]
    inside = np.where(col[1:-1] < 0.5)[0] + 1
    lo, hi = inside.min(), inside.max()

    def cross(a, b):
        return a + (0.5 - col[a]) / (col[b] - col[a]) * (b - a)

    return cross(lo - 1, lo), cross(hi, hi + 1)


@pytest.mark.parametrize("case", [1, 2])
def test_bubble_f64_matches_oracle(lbm, case):
    c = W.rising_bubble_2d(case)
    _, g = run_gpu(lbm, c, 200, storage="f64")
    _, o = run_oracle(c, 200)
    assert_fields(g, o, 1e-12, d=2)


@pytest.mark.parametrize("case", [1, 2])
def test_bubble_f32_tracks_f64(lbm, case):
    """FP32 arithmetic against FP64 over 20000 steps.  Pointwise checks at a
    few steps do not suit this case: the velocities start at 1e-7, a
    millionth of the populations that carry them, so they sit at the FP32
    floor of those populations.  The quantities of the case do not: the rise
    of the bubble and its peak speed agree within 1 %, the interface heights
    on the centre line within 0.05 sites.  The phase mass: see
    test_bubble_f32_phase_mass."""
    c = W.rising_bubble_2d(case)
    t = 20000
    _, (f32, P32, u32) = run_gpu(lbm, c, t, storage="f32")
    _, (f64, P64, u64) = run_gpu(lbm, c, t, storage="f64")
    r32 = centroid_y(c, f32) - centroid_y(c, c.phi0)
    r64 = centroid_y(c, f64) - centroid_y(c, c.phi0)
    s32, s64 = np.abs(u32).max(), np.abs(u64).max()
    assert abs(r32 - r64) <= 1e-2 * abs(r64), f"rise {r32:.5f} vs {r64:.5f}"
    assert abs(s32 - s64) <= 1e-2 * s64, f"max|u| {s32:.4e} vs {s64:.4e}"
    for a, b in zip(interface_heights(f32), interface_heights(f64)):
        assert abs(a - b) <= 0.05, f"interface {a:.4f} vs {b:.4f}"


@pytest.mark.parametrize("case", [1, 2])
def test_bubble_rises_at_most_at_the_added_mass_rate(lbm, case):
    """Early on, a 2D cylinder of density rho_2 in a liquid of density rho_1
    accelerates at a = g (rho_1 - rho_2) / (rho_2 + C_a rho_1), C_a = 1 (the
    added mass of a circular cylinder).  Drag, the pressure waves that set
    up the hydrostatic state and the finite interface only slow it, so after
    t steps the rise lies below a t^2 / 2 and, this early (t well under the
    time scale 2R / sqrt(2 R g) = 86000 steps), not far below it.  The phase
    mass stays constant to rounding."""
    c = W.rising_bubble_2d(case)
    rho1, rho2, grav = c.meta["rho1"], c.meta["rho2"], c.meta["g"]
    t = 20000
    L, (phi, P, u) = run_gpu(lbm, c, t, storage="f64")
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(P)) and np.all(np.isfinite(u))
    rise = centroid_y(c, phi) - centroid_y(c, c.phi0)
    a = grav * (rho1 - rho2) / (rho2 + rho1)
    ideal = 0.5 * a * t * t
    assert 0.3 * ideal <= rise <= 1.02 * ideal, f"rise {rise:.4f} vs inviscid {ideal:.4f}"
    assert abs(phi.sum() / c.phi0.sum() - 1) <= 1e-10


@pytest.mark.parametrize("case", [1, 2])
def test_bubble_f32_phase_mass(lbm, case):
    """FP32 storage and the phase mass of the rising bubble over 20000 steps.
    The collision stores as the rest population what the moving ones leave
    of the pulled phi, which takes the weights' rounding and the moving
    populations' rounding out of the mass; what remains (2.8e-5 here) is the
    rounding of the two FP32 sums, which in a slow flow leans the same way
    at a site step after step.  Summing exactly and rounding that population
    without bias removed it (below 1e-6), but the random flips it puts into
    phi destabilised the sheared layered channel within 9000-16000 steps, so
    it is not built; the bound here guards the closure (without it: 1.6e-4)."""
    c = W.rising_bubble_2d(case)
    L, _ = run_gpu(lbm, c, 0, storage="f32")
    m0 = L.reduce()["mass"]
    L.step(20000)
    L.check()
    assert abs(L.reduce()["mass"] / m0 - 1) <= 1e-4


@pytest.mark.parametrize("case", [1, 2])
def test_bubble_batch_as_benchmarked(lbm, case):
    """The launch configuration bench.py --workload bubble1/2 times: 32
    lattices of the case in one FP32 batch at the shape lbm_batch_autotune
    picks.  Every member ends bit for bit like every other, and against the
    FP64 oracle after 50 steps phi is within 1e-5 (measured 3.7e-6), P within
    1e-4 of max|P| (measured 1.7e-5) and u within 2e-4 of max|u| (measured
    7e-5; u is still 1e-6, near the FP32 floor of the populations that carry
    it, see test_bubble_f32_tracks_f64)."""
    c = W.rising_bubble_2d(case)
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    steps = 50
    B = lbm.Batch("D2Q9", "f32")
    lats = []
    for _ in range(32):
        L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f32",
                        g_ext=c.params["g_ext"], **prm)
        L.init_fields(c.phi0, c.P0, c.u0)
        B.add(L, steps + 1000)
        lats.append(L)
    B.autotune(32)                               # restores every member's state and budget
    B.step(steps)
    _, (fo, Po, uo) = run_oracle(c, steps)
    first = lats[0].read_fields()
    for L in lats[1:]:
        for x, y in zip(first, L.read_fields()):
            assert np.array_equal(x, y)
    f, P, u = first
    assert np.abs(f - fo).max() <= 1e-5
    assert np.abs(P - Po).max() <= 1e-4 * np.abs(Po).max()
    assert np.abs(u - uo).max() <= 2e-4 * np.abs(uo).max()
    B.close()
    for L in lats:
        L.close()
