"""The seeded workloads against the numbers the paper prints (host only).

The rising bubble (Sec. III.D) must carry the table's densities,
viscosities and surface tension, the stated geometry and gravity; its Re and
We then follow as the table gives them."""
import json
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.json")


@pytest.mark.parametrize("case", [1, 2])
def test_rising_bubble_carries_the_table(case):
    g = json.load(open(GOLDEN))[f"bubble_case{case}"]
    c = W.rising_bubble_2d(case)
    p = c.params
    assert c.lattice == "D2Q9" and c.shape == (200, 400, 1)
    assert p["rho_w"] == pytest.approx(g["rho1"]) and p["rho_a"] == pytest.approx(0.22)
    assert p["nu_w"] * p["rho_w"] == pytest.approx(g["mu1"], rel=1e-12)
    assert p["sigma"] == pytest.approx(g["sigma"])
    assert p["g_ext"][0] == 0.0 and p["g_ext"][1] == pytest.approx(-g["g"])
    assert p["M"] == pytest.approx(0.166) and p["W"] == pytest.approx(4.0)
    # Re and We of the table from the workload's own parameters
    Ug = np.sqrt(2 * g["R"] * -p["g_ext"][1])
    Re = p["rho_w"] * Ug * 2 * g["R"] / (p["nu_w"] * p["rho_w"])
    We = p["rho_w"] * Ug ** 2 * 2 * g["R"] / p["sigma"]
    assert Re == pytest.approx(g["Re"], rel=0.01)
    assert We == pytest.approx(g["We"], rel=0.01)


@pytest.mark.parametrize("case", [1, 2])
def test_rising_bubble_geometry(case):
    """Bubble of radius 50 at (100, 100): phi = 1/2 at distance R from the
    centre, light inside, liquid outside; solid rows at y = 0 and 399."""
    c = W.rising_bubble_2d(case)
    phi = c.phi0[0]
    assert phi[100, 100] < 1e-12 and phi[300, 100] > 1 - 1e-12
    # along x through the centre the phi = 1/2 crossings lie at 100 -+ 50
    row = phi[100, :]
    left = np.where(row[:100] > 0.5)[0].max()
    right = np.where(row[100:] > 0.5)[0].min() + 100
    assert left in (49, 50) and right in (150, 151)
    assert c.solid[0, 0].all() and c.solid[0, -1].all() and c.solid[0, 1:-1].sum() == 0
    assert c.periodic == (1, 0, 1)
    # the phase mass deficit is the disc's area, pi R^2, up to the interface profile's symmetry
    deficit = float((1 - phi)[1:-1].sum())
    assert deficit == pytest.approx(np.pi * 50.0 ** 2, rel=2e-3)
