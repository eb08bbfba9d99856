"""The alternative reading of the pressure formula (Sec. II): the omega-term
omega rho_ref sum_i w_i (c_i . u)|_{x - c_i} with the new velocity u^{n+1}
(coupling_unew = 1) instead of the previous step's u^n.

The split form takes the new velocity's neighbours in its collision launch;
with FP64 storage it evaluates the oracle's sum in the oracle's order, so the
fields equal the oracle's (coupling_unew = 1) bit for bit, in a single
lattice, both stores and a batch.  The host pin
test_unew_coupling_is_unstable_at_low_viscosity shows why it is not the
default.
"""
import numpy as np
import pytest

import workloads as W
from test_gpu_parity import assert_fields, closed_box_3d, run_gpu, run_oracle, small_3d
from test_gpu_split import closed_box_2d

pytestmark = pytest.mark.gpu

CASES = {
    "droplet_2d": lambda: W.droplet_2d(40, 10.0, ux=0.01),
    "closed_box_2d": closed_box_2d,
    "walls_d3q27": lambda: small_3d("D3Q27"),
    "closed_box_d3q19": lambda: closed_box_3d("D3Q19"),
}


@pytest.mark.parametrize("inplace", [0, 1])
@pytest.mark.parametrize("case", sorted(CASES))
def test_unew_coupling_f64_matches_oracle(lbm, case, inplace):
    c = CASES[case]()
    steps = 25
    _, g = run_gpu(lbm, c, steps, "f64", coupling_unew=1, inplace=inplace)
    _, o = run_oracle(c, steps, coupling_unew=1)
    assert_fields(g, o, 1e-12, d=2 if c.lattice == "D2Q9" else 3)
    for x, y in zip(g, o):
        assert np.array_equal(x, y)
    # the flag changes the result (the omega-term is not zero here)
    _, o0 = run_oracle(c, steps)
    assert np.abs(o0[1] - o[1]).max() > 0


def test_unew_coupling_f64_batch_matches_oracle(lbm):
    c = CASES["walls_d3q27"]()
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    B = lbm.Batch(c.lattice, "f64")
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f64", coupling_unew=1, **prm)
    L.init_fields(c.phi0, c.P0, c.u0)
    B.add(L, 20)
    B.step(20)
    g = L.read_fields()
    _, o = run_oracle(c, 20, coupling_unew=1)
    for x, y in zip(g, o):
        assert np.array_equal(x, y)
    B.close()


@pytest.mark.parametrize("case", ["droplet_2d", "walls_d3q27"])
def test_unew_coupling_f32_short_horizon(lbm, case):
    """FP32 arithmetic takes the omega-term from the pair stencil's
    divergence (sum_i w_i c_i . u(x - c_i) = -T div u, the same wall rule):
    the oracle's sum up to rounding."""
    c = CASES[case]()
    _, g = run_gpu(lbm, c, 5, "f32", coupling_unew=1)
    _, o = run_oracle(c, 5, coupling_unew=1)
    d = 2 if c.lattice == "D2Q9" else 3
    (f1, P1, u1), (f2, P2, u2) = g, o
    assert np.abs(f1 - f2).max() <= 1e-5
    assert np.abs(u1[:d] - u2[:d]).max() <= 1e-5 * np.abs(u2[:d]).max()
    assert np.abs(P1 - P2).max() <= 1e-5 * np.abs(P2).max()


def test_unew_coupling_other_forms_refused(lbm):
    c = small_3d("D3Q27", nx=64, ny=8, nz=9)
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f32", coupling_unew=1, **prm)
    for variant in (1, 2, 4, 5):
        with pytest.raises(lbm.LbmError) as e:
            L.set_tuning(variant, 0)
        assert e.value.code == 5
    L.set_tuning(3, 0)
