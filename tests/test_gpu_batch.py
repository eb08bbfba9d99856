"""Batched persistent launch (lbm_batch_*) and the autotuner.

A batch steps many lattices with two launches per time step for the whole
set.  Each site's arithmetic is the split form's, in one kernel whatever the
membership, so a lattice's results must not depend on its batch-mates
(bitwise), FP64 members must reproduce the oracle bit for bit, and step
budgets, chunking and graph replay must not change anything either.
"""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import closed_box_3d, run_oracle, small_3d

pytestmark = pytest.mark.gpu


def make(lbm, c, storage="f64", inplace=0):
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage=storage,
                    g_ext=c.params.get("g_ext", (0, 0, 0)), inplace=inplace, **prm)
    L.init_fields(c.phi0, c.P0, c.u0)
    return L


def cases_d3q19():
    a = small_3d("D3Q19")                                   # walls, ragged tiles
    b = closed_box_3d("D3Q19")                              # random solids, closed
    c = small_3d("D3Q19", nx=9, ny=7, nz=5, walls=False)    # periodic, thin
    return [a, b, c]


def test_batch_f64_matches_oracle(lbm):
    """Three different lattices (grids, walls, layouts) in one batch, budgets
    37 / 50 / 23 steps over chunks of 16: each equals the oracle bit for bit."""
    cs = cases_d3q19()
    budgets = [37, 50, 23]
    B = lbm.Batch("D3Q19", "f64")
    Ls = [make(lbm, c, "f64", inplace=j % 2) for j, c in enumerate(cs)]
    for L, n in zip(Ls, budgets):
        B.add(L, n)
    assert B.step(100) == 3
    for L, c, n in zip(Ls, cs, budgets):
        assert L.steps_done == n
        assert B.remaining(L) == 0
        g = L.read_fields()
        _, o = run_oracle(c, n)
        for x, y in zip(g, o):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_alone_vs_mixed_bitwise(lbm, storage):
    """A lattice stepped alone in a batch and stepped among others (which
    join late, leave early and use the other store layout) ends bit for bit
    the same; so do graph replay and plain launches, and any chunk length."""
    c = W.droplet_3d(24)
    others = [small_3d("D3Q27"), closed_box_3d("D3Q27"), small_3d("D3Q27", nx=40, ny=12, nz=21)]
    n = 41

    B1 = lbm.Batch("D3Q27", storage)
    A1 = make(lbm, c, storage)
    B1.add(A1, n)
    B1.step(n)
    want = A1.read_fields()

    B2 = lbm.Batch("D3Q27", storage)
    B2.set_tuning(chunk=5, use_graph=True)
    A2 = make(lbm, c, storage)
    O = [make(lbm, oc, storage, inplace=j % 2) for j, oc in enumerate(others)]
    B2.add(A2, n)
    B2.add(O[0], 7)                   # finishes inside the first chunks
    B2.step(12)
    B2.add(O[1], 100)                 # joins late
    B2.add(O[2], 100)
    B2.step(10)
    B2.remove(O[1])                   # leaves early
    B2.step(100)
    assert A2.steps_done == n and O[0].steps_done == 7
    for x, y in zip(want, A2.read_fields()):
        assert np.array_equal(x, y)

    B3 = lbm.Batch("D3Q27", storage)
    B3.set_tuning(chunk=1, use_graph=False)
    A3 = make(lbm, c, storage)
    B3.add(A3, n)
    B3.step(n)
    for x, y in zip(want, A3.read_fields()):
        assert np.array_equal(x, y)


def test_batch_matches_single_lattice_split(lbm):
    """The batch kernels and the single-lattice split kernels evaluate the
    same per-site code: FP64 bit for bit, FP32 to rounding."""
    c = small_3d("D3Q27")
    for storage in ("f64", "f32"):
        S = make(lbm, c, storage)
        S.set_tuning(3, 0)
        S.step(30)
        B = lbm.Batch("D3Q27", storage)
        L = make(lbm, c, storage)
        B.add(L, 30)
        B.step(30)
        for x, y in zip(S.read_fields(), L.read_fields()):
            if storage == "f64":
                assert np.array_equal(x, y)
            else:
                assert np.abs(x - y).max() <= 1e-5 * max(np.abs(x).max(), 1e-30)


def test_batch_rules(lbm):
    c = small_3d("D3Q27")
    B = lbm.Batch("D3Q27", "f32")
    L = make(lbm, c, "f32")
    B.add(L, 10)
    with pytest.raises(lbm.LbmError) as e:
        L.step(1)                      # stepped by its batch only
    assert e.value.code == lbm.LBM_ERR_INVALID_ARG
    with pytest.raises(lbm.LbmError):
        B.add(L, 5)                    # already a member
    with pytest.raises(lbm.LbmError):
        B.add(make(lbm, c, "f16"), 5)  # other storage
    with pytest.raises(lbm.LbmError):
        B.set_tuning(chunk=65)
    assert B.step(4) == 0 and B.remaining(L) == 6
    m, launches = B.info()
    assert m == 1 and launches == 2 * 4
    L.read_fields()                    # readable between batch steps
    B.remove(L)
    L.step(2)                          # its own again
    assert L.steps_done == 6
    # destroying a member detaches it
    L2 = make(lbm, c, "f32")
    B.add(L2, 3)
    L2.close()
    B.members.remove(L2)
    assert B.info()[0] == 0
    assert B.step(5) == 0


def test_autotune_keeps_state(lbm):
    c = small_3d("D3Q27", nx=48, ny=24, nz=20)
    L = make(lbm, c, "f32")
    L.step(3)
    v, z, ms = L.autotune(3)
    assert v in (1, 2, 3, 4, 5) and ms > 0
    assert L.steps_done == 3
    L.step(5)
    R = make(lbm, c, "f32")
    R.step(3)
    R.set_tuning(v, z)
    R.step(5)
    for x, y in zip(R.read_fields(), L.read_fields()):
        assert np.array_equal(x, y)
    # an in-place store has the split forms only
    I = make(lbm, c, "f32", inplace=1)
    assert I.autotune(2)[0] in (3, 4)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_autotune_keeps_results(lbm, storage):
    """The batch autotuner tries launch shapes (chunk, span, blocks per SM) on
    the members' own states, keeps the fastest and restores every member's
    state and budget: the members then step on exactly as an untuned batch
    does, bit for bit (every site runs the same arithmetic in any shape)."""
    cs = [small_3d("D3Q27", nx=64, ny=8, nz=9), small_3d("D3Q27", nx=37, ny=11, nz=13),
          small_3d("D3Q27", nx=32, ny=6, nz=8, walls=False)]
    ref, tuned = [], []
    for group in (ref, tuned):
        B = lbm.Batch("D3Q27", storage)
        Ls = [make(lbm, c, storage) for c in cs]
        for L, n in zip(Ls, (12, 9, 12)):
            B.add(L, n)
        group.append((B, Ls))
    (Br, Lr), (Bt, Lt) = ref[0], tuned[0]
    Br.step(5)
    Bt.step(5)
    K, span, bps, ms = Bt.autotune(8)
    assert K in (8, 16, 32) and span in (1, 2, 4, 8) and bps >= 0 and ms > 0
    assert [Bt.remaining(L) for L in Lt] == [7, 4, 7]
    assert [L.steps_done for L in Lt] == [5, 5, 5]
    Br.step(7)
    Bt.step(7)
    for a, b in zip(Lr, Lt):
        for x, y in zip(a.read_fields(), b.read_fields()):
            assert np.array_equal(x, y)
    # every shape gives the same bits
    Bt.set_shape(3, 1)
    Bt.set_tuning(chunk=5)
    for B, Ls in (ref[0], tuned[0]):
        for L in Ls:
            B.remove(L)
            B.add(L, 6)
    Br.set_shape(1, 0)
    Br.step(6)
    Bt.step(6)
    for a, b in zip(Lr, Lt):
        for x, y in zip(a.read_fields(), b.read_fields()):
            assert np.array_equal(x, y)
    for B, _ in (ref[0], tuned[0]):
        B.close()


@pytest.mark.parametrize("storage", ["f64", "f16"])
def test_paused_member_waits_and_resumes_bitwise(lbm, storage):
    """lbm_batch_pause: a paused member takes no steps (its budget and state
    stay) while the others advance; resumed, it ends bit for bit as it would
    have without the pause, in FP64 also equal to the oracle.  Odd pause
    lengths shift it against its batch-mates' in-place step parity."""
    a, b = small_3d("D3Q27"), closed_box_3d("D3Q27")
    B = lbm.Batch("D3Q27", storage)
    A = make(lbm, a, storage, inplace=1)
    O = make(lbm, b, storage)
    B.add(A, 30)
    B.add(O, 60)
    B.step(7)
    B.pause(A)
    before = A.read_fields()
    B.step(13)
    assert B.remaining(A) == 23 and B.remaining(O) == 40
    for x, y in zip(before, A.read_fields()):
        assert np.array_equal(x, y)
    B.pause(A, False)
    assert B.step(100) == 2
    R = make(lbm, a, storage, inplace=1)
    B2 = lbm.Batch("D3Q27", storage)
    B2.add(R, 30)
    B2.step(30)
    for x, y in zip(R.read_fields(), A.read_fields()):
        assert np.array_equal(x, y)
    if storage == "f64":
        _, o = run_oracle(a, 30)
        for x, y in zip(A.read_fields(), o):
            assert np.array_equal(x, y)
    with pytest.raises(lbm.LbmError):
        B2.pause(O)                      # not a member of B2
