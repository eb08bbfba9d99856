"""Cluster step (variant 5): one launch per step; a CTA owns one row of sites
and marches in z, and the CTAs of a thread-block cluster (consecutive rows)
share the moments of each plane through distributed shared memory.

The per-site arithmetic is the split form's.  With FP64 storage (built
without FMA contraction) it is the canonical order of the oracle, so every
field equals the oracle's bit for bit.  The cases cover walls and random
solid sites, closed and periodic y and z axes (the halo rows of a cluster
outside a closed axis, the z chunks that wrap), z chunks that do not divide
the grid, and clusters of 2, 4 and 8 rows.  With FP32 arithmetic it is
compared with the split form: only the compiler's contraction of a product
and a sum into one FMA may differ between the two kernels.
"""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import assert_fields, run_oracle, small_3d

pytestmark = pytest.mark.gpu


def closed_y_d3q19():
    c = small_3d("D3Q19", nx=32, ny=8, nz=9)
    r = (W.uniform_pm1(29, 32 * 8 * 9).reshape(9, 8, 32) > 0.95).astype(np.uint8)
    r[:, 2:6, 10:22] = 0
    r[0] = 1
    r[-1] = 1
    c.solid = r
    c.periodic = (1, 0, 0)
    c.phi0 = np.where(r.astype(bool), 0.0, c.phi0)
    c.u0[:, r.astype(bool)] = 0.0
    return c


# case -> (workload, cluster rows, planes per CTA)
CASES = {
    "walls_d3q27_rows4": (lambda: small_3d("D3Q27", nx=64, ny=8, nz=13), 4, 5),
    "closed_y_d3q19_rows2": (closed_y_d3q19, 2, 4),
    "periodic_d3q27_rows4": (lambda: small_3d("D3Q27", nx=64, ny=16, nz=10, walls=False), 4, 3),
    "walls_d3q27_rows8": (lambda: small_3d("D3Q27", nx=128, ny=16, nz=9), 8, 4),
}


def make(lbm, c, storage, variant, rows=0, zchunk=0, staged=-1):
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage,
                    g_ext=c.params.get("g_ext", (0, 0, 0)), **prm)
    if rows or staged != -1:
        L.set_cluster(rows, staged)
    L.set_tuning(variant, zchunk)
    L.init_fields(c.phi0, c.P0, c.u0)
    return L


@pytest.mark.parametrize("steps", [1, 9])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cluster_f64_matches_oracle(lbm, case, steps):
    fn, rows, zc = CASES[case]
    c = fn()
    L = make(lbm, c, "f64", 5, rows, zc)
    L.step(steps)
    L.check()
    g = L.read_fields()
    _, o = run_oracle(c, steps)
    assert_fields(g, o, 1e-12)
    for x, y in zip(g, o):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("staged", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_cluster_f32_matches_split(lbm, case, staged):
    """Rows read from the store (staged = 0) or staged in shared memory by
    bulk copies (staged = 1): the split form's FP32 arithmetic either way."""
    fn, rows, zc = CASES[case]
    c = fn()
    a = make(lbm, c, "f32", 5, rows, zc, staged)
    b = make(lbm, c, "f32", 3)
    for L in (a, b):
        L.step(23)
        L.check()
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.abs(x - y).max() <= 1e-6 * max(np.abs(y).max(), 1e-30)
    ra, rb = a.reduce(), b.reduce()
    assert abs(ra["mass"] / rb["mass"] - 1) <= 1e-7


@pytest.mark.parametrize("staged", [0, 1])
def test_cluster_f16_matches_split(lbm, staged):
    """16-bit storage: the same codes as the split form up to an FMA
    contraction that moves a stored code by one step of the encoding (the
    bound of the split form's own comparison with the fused kernel)."""
    fn, rows, zc = CASES["walls_d3q27_rows4"]
    c = fn()
    steps = 2
    a = make(lbm, c, "f16", 5, rows, zc, staged)
    b = make(lbm, c, "f16", 3)
    for L in (a, b):
        L.step(steps)
    fa, fb = a.read_fields(), b.read_fields()
    assert np.abs(fa[0] - fb[0]).max() <= 2 * steps * 2.0 ** -11
    for x, y in zip(fa[1:], fb[1:]):
        assert np.abs(x - y).max() <= 1e-2 * max(np.abs(y).max(), 1e-30)


def test_cluster_rows_and_chunks_do_not_change_results(lbm):
    c = small_3d("D3Q27", nx=128, ny=16, nz=11)
    runs = []
    for rows, zc in [(2, 11), (4, 3), (8, 1), (8, 0)]:
        L = make(lbm, c, "f64", 5, rows, zc)
        L.step(4)
        runs.append(L.read_fields())
    for r in runs[1:]:
        for x, y in zip(runs[0], r):
            assert np.array_equal(x, y)


def test_cluster_unsupported_shapes(lbm):
    c = small_3d("D3Q27", nx=37, ny=11, nz=13)          # nx not a multiple of 32
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f32", **prm)
    with pytest.raises(lbm.LbmError) as e:
        L.set_tuning(5, 0)
    assert e.value.code == 5
    c2 = W.droplet_2d(32, 8.0)                          # 2D
    L2 = lbm.Lattice(c2.lattice, c2.shape, storage="f64")
    with pytest.raises(lbm.LbmError):
        L2.set_tuning(5, 0)
    c3 = small_3d("D3Q27", nx=64, ny=8, nz=9)
    L3 = lbm.Lattice(c3.lattice, c3.shape, periodic=c3.periodic, solid=c3.solid, storage="bf16", **prm)
    with pytest.raises(lbm.LbmError):
        L3.set_tuning(5, 0)                             # BF16 odd-part deferral
    L4 = lbm.Lattice(c3.lattice, c3.shape, periodic=c3.periodic, solid=c3.solid, storage="f32", **prm)
    with pytest.raises(lbm.LbmError):
        L4.set_cluster(8)                               # 2 nx = 128 is not a multiple of 32 x 8
    with pytest.raises(lbm.LbmError):
        L4.set_cluster(3)
    with pytest.raises(lbm.LbmError):
        L4.set_cluster(4, 2)
