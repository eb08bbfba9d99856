"""Split form (two launches per step) and in-place AA streaming.

The split form evaluates the same per-site arithmetic as the fused kernels
in another data movement: FP64 must reproduce the oracle bit for bit (both
ping-pong and in-place stores), FP32 and 16-bit storage must reproduce the
fused kernels.  In-place streaming keeps one population store; after an odd
number of steps its slots are in the shifted AA layout, so read-out,
probes, reductions and checkpoints are checked after odd and even counts.
"""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import assert_fields, closed_box_3d, run_oracle, small_3d

pytestmark = pytest.mark.gpu


def make(lbm, c, storage="f64", variant=0, inplace=0):
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage,
                    g_ext=c.params.get("g_ext", (0, 0, 0)), inplace=inplace, **prm)
    if variant:
        L.set_tuning(variant, 0)
    L.init_fields(c.phi0, c.P0, c.u0)
    return L


def closed_box_2d():
    c = W.droplet_2d(41, 9.0, center=(19.3, 21.7), ux=0.01)
    r = (W.uniform_pm1(11, 41 * 41).reshape(1, 41, 41) > 0.93).astype(np.uint8)
    r[:, 15:27, 14:28] = 0
    c.solid = r
    c.periodic = (0, 0, 1)
    c.phi0 = np.where(r.astype(bool), 0.0, c.phi0)
    c.u0[:, r.astype(bool)] = 0.0
    return c


CASES = {
    "droplet_2d": lambda: W.droplet_2d(40, 10.0, ux=0.01),
    "channel_2d": lambda: W.poiseuille_2d(32, 64),
    "closed_box_2d": closed_box_2d,
    "walls_d3q19": lambda: small_3d("D3Q19"),
    "closed_box_d3q27": lambda: closed_box_3d("D3Q27"),
    "periodic_thin_d3q27": lambda: small_3d("D3Q27", nx=9, ny=7, nz=5, walls=False),
    "wide_walls_d3q27": lambda: small_3d("D3Q27", nx=64, ny=5, nz=7),
}


@pytest.mark.parametrize("inplace", [0, 1])
@pytest.mark.parametrize("steps", [37, 60])
@pytest.mark.parametrize("case", sorted(CASES))
def test_split_f64_matches_oracle(lbm, case, steps, inplace):
    c = CASES[case]()
    L = make(lbm, c, "f64", variant=3, inplace=inplace)
    L.step(steps)
    g = L.read_fields()
    _, o = run_oracle(c, steps)
    assert_fields(g, o, 1e-12, d=3 if c.lattice != "D2Q9" else 2)
    for x, y in zip(g, o):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", ["closed_box_d3q27", "walls_d3q19", "closed_box_2d"])
def test_split_matches_fused(lbm, case, storage):
    """Same formulas, other data movement: split ping-pong, split in-place and
    the plane-synchronous fused kernel.  The split form's two stores are one
    kernel pair and agree bit for bit.  Against the fused kernel, FP32
    arithmetic differs only where the compiler contracted a product and a sum
    into one FMA differently, a few ulp per step; with 16-bit storage such a
    difference can move a stored code by one step of the encoding, so after
    2 steps |dphi| <= 2 x 2 x (half the 16-bit spacing of t = h/w for t < 2:
    2^-11 FP16, 2^-8 BF16) summed over sum_i w_i = 1."""
    c = CASES[case]()
    steps = 23 if storage == "f32" else 2
    a = make(lbm, c, storage, variant=1)
    b = make(lbm, c, storage, variant=3)
    d = make(lbm, c, storage, inplace=1)
    for L in (a, b, d):
        L.step(steps)
    fa, fb, fd = a.read_fields(), b.read_fields(), d.read_fields()
    for y, z in zip(fb, fd):
        assert np.array_equal(y, z)
    if storage == "f32":
        for x, y in zip(fa, fb):
            assert np.abs(x - y).max() <= 1e-6 * max(np.abs(x).max(), 1e-30)
    else:
        half = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
        assert np.abs(fa[0] - fb[0]).max() <= 2 * steps * half
        # P and u: the same code flips seen through the velocity/pressure
        # moments; bounded by the 16-bit tests against the oracle.
        for x, y in zip(fa[1:], fb[1:]):
            assert np.abs(x - y).max() <= 1e-2 * max(np.abs(x).max(), 1e-30)


@pytest.mark.parametrize("steps", [0, 1, 2, 7])
def test_inplace_state_matches_ping_pong(lbm, steps):
    """Decoded populations (get_state, probe) of the in-place store equal the
    ping-pong store's after even and odd step counts, including sites next
    to solids and the non-periodic boundary."""
    c = closed_box_3d("D3Q19")
    a = make(lbm, c, "f64", variant=3)
    b = make(lbm, c, "f64", inplace=1)
    a.step(steps)
    b.step(steps)
    sa, sb = a.get_state(), b.get_state()
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)
    N = a.N
    sites = np.unique(np.r_[0, 1, N // 3, N // 2 + 5, N - 1, np.flatnonzero(c.solid.reshape(-1))[:3] + 1])
    pa, pb = a.probe(sites), b.probe(sites)
    for x, y in zip(pa, pb):
        assert np.array_equal(x, y)
    ra, rb = a.reduce(), b.reduce()
    assert ra["mass"] == rb["mass"]
    assert np.array_equal(ra["momentum"], rb["momentum"])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_inplace_checkpoint_resume(lbm, storage):
    """A checkpoint taken after an odd step count (shifted AA layout; with
    BF16 also the deferred odd part of g, folded into the populations when
    saved) resumes bit for bit."""
    c = small_3d("D3Q27")
    L1 = make(lbm, c, storage, inplace=1)
    L1.step(13)                                   # odd: shifted AA layout
    blob = L1.save_state()
    L1.step(8)
    want = L1.read_fields()
    L2 = make(lbm, c, storage, inplace=1)
    L2.load_state(blob)
    assert L2.steps_done == 13
    L2.step(8)
    for x, y in zip(want, L2.read_fields()):
        assert np.array_equal(x, y)
    # a ping-pong handle refuses the in-place layout and keeps its own state
    L3 = make(lbm, c, storage)
    before = L3.read_fields()
    with pytest.raises(lbm.LbmError) as e:
        L3.load_state(blob)
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG
    for x, y in zip(before, L3.read_fields()):
        assert np.array_equal(x, y)


def test_inplace_halves_population_memory(lbm):
    c = small_3d("D3Q27", nx=64, ny=32, nz=16)
    a = make(lbm, c, "f32")
    b = make(lbm, c, "f32", inplace=1)
    pop = 27 * c.phi0.size * 4                    # one population set, FP32
    assert a.footprint()[0] - b.footprint()[0] == 2 * pop


def test_inplace_refuses_fused_variants(lbm):
    c = small_3d("D3Q27")
    L = make(lbm, c, "f32", inplace=1)
    L.set_tuning(3, 0)
    for v in (1, 2):
        with pytest.raises(lbm.LbmError) as e:
            L.set_tuning(v, 0)
        assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("inplace", [0, 1])
@pytest.mark.parametrize("case", ["closed_box_d3q27", "periodic_thin_d3q27", "walls_d3q19", "droplet_2d",
                                  "closed_box_2d"])
def test_persistent_matches_split(lbm, case, storage, inplace):
    """The persistent split step (one launch per step, plane-ordered work
    items with waits) runs the split form's per-site code: it must agree with
    the two-launch form to rounding (the compiler may contract differently in
    another kernel), after odd and even step counts, with walls, random
    solids, z-periodic wrap and 2D lattices."""
    c = CASES[case]()
    for steps in (9, 14):
        a = make(lbm, c, storage, variant=3, inplace=inplace)
        b = make(lbm, c, storage, variant=4, inplace=inplace)
        a.step(steps)
        b.step(steps)
        b.check()
        fa, fb = a.read_fields(), b.read_fields()
        for x, y in zip(fa, fb):
            assert np.all(np.isfinite(y))
        if storage == "f32":
            for x, y in zip(fa, fb):
                assert np.abs(x - y).max() <= 1e-6 * max(np.abs(x).max(), 1e-30)
        else:
            # a rounding difference can move a 16-bit code by one step
            assert np.abs(fa[0] - fb[0]).max() <= 2 * steps * 2.0 ** -11
            for x, y in zip(fa[1:], fb[1:]):
                assert np.abs(x - y).max() <= 1e-2 * max(np.abs(x).max(), 1e-30)


def test_persistent_wait_runs_out_and_reports(lbm):
    """Failure path of the persistent step: with the moments of one plane
    left uncounted, the collisions that need it wait until their bounded wait
    (1 s on the GPU timer) runs out; the launch ends, the step reports
    LBM_ERR_TIMEOUT, and the handle, cleared and initialised again, steps
    exactly like a fresh one."""
    import time
    c = CASES["closed_box_d3q27"]()
    L = make(lbm, c, "f32", variant=4)
    L.debug_stall(1)
    t0 = time.perf_counter()
    L.step(1)
    with pytest.raises(lbm.LbmError) as e:
        L.check()
    assert e.value.code == lbm.LBM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    L.debug_stall(-1)
    L.init_fields(c.phi0, c.P0, c.u0)
    ref = make(lbm, c, "f32", variant=4)
    L.step(7)
    ref.step(7)
    L.check()
    for x, y in zip(L.read_fields(), ref.read_fields()):
        assert np.array_equal(x, y)
    with pytest.raises(lbm.LbmError) as e:
        L.debug_stall(10 ** 6)
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG


def test_persistent_refused_for_f64(lbm):
    c = CASES["walls_d3q19"]()
    L = make(lbm, c, "f64")
    with pytest.raises(lbm.LbmError) as e:
        L.set_tuning(4, 0)
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


def test_bf16_population_reads_change_nothing(lbm):
    """With BF16 storage part of g is kept beside the populations; reading
    the populations (get_state, probe) adds it on the fly, so a handle that
    was read continues bit for bit like one that was not."""
    c = small_3d("D3Q27")
    a = make(lbm, c, "bf16")
    b = make(lbm, c, "bf16")
    a.step(5)
    b.step(5)
    h1, g1, _, _ = a.get_state()
    a.probe(np.arange(0, a.N, 97))
    assert np.all(np.isfinite(g1))
    a.step(6)
    b.step(6)
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)
