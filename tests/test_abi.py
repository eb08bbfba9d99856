"""The C-ABI library builds, loads and exports every symbol include/lbm.h
declares; argument checks and the no-device path need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2512_01027_gb300 as lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lbm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_read_fields", "lbm_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    L = lbm.lib()
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(L, n), f"missing export {n}"
    # the binding marshals every declared function
    assert set(names) == set(lbm.SIGNATURES)


def test_default_params_are_the_papers():
    p = lbm.default_params()
    assert p.struct_size == ctypes.sizeof(lbm.Params)
    assert (p.gamma, p.phi_n, p.phi_m, p.D, p.eps) == (-22.5, 0.8, 0.2, 1e-4, 1e-10)
    assert p.lambda_b == 1.0 / 6.0 and p.M == 0.166 and p.W == 4.0
    assert p.rho_w / p.rho_a == pytest.approx(1000.0)
    assert p.storage == lbm.F32 and p.filter_full_trace == 0 and p.clamp_phi_props == 1


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_direction_tables_agree_by_convention(lat):
    """Library and oracle write their own tables; both follow rest-first, (c, -c) pairs."""
    d1, q1, c1, w1 = lbm.lattice_info(lat)
    d2, q2, c2, w2 = oracle.lattice_info(lat)
    assert (d1, q1) == (d2, q2)
    assert np.array_equal(c1, c2)
    assert np.array_equal(w1, w2)


def _create(**kw):
    g = lbm.Grid()
    g.nx, g.ny, g.nz = kw.pop("shape", (8, 8, 1))
    for a in range(3):
        g.periodic[a] = 1
    p = lbm.default_params(**kw.pop("params", {}))
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    rc = lbm.lib().lbm_create(ctypes.byref(g), kw.get("lattice", lbm.D2Q9), ctypes.byref(p), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("bad", [dict(rho_a=0.0), dict(rho_w=1e-4), dict(nu_w=0.0), dict(M=-1.0),
                                 dict(W=0.0), dict(storage=9), dict(struct_size=8)])
def test_create_rejects_bad_parameters(bad):
    rc, h = _create(**bad)
    assert rc == lbm.LBM_ERR_INVALID_ARG
    assert not h.value
    assert lbm.lib().lbm_last_error(None)


def test_create_rejects_bad_grids():
    rc, _ = _create(shape=(0, 8, 1))
    assert rc == lbm.LBM_ERR_INVALID_ARG
    rc, _ = _create(shape=(8, 8, 2))          # 2D lattice with nz > 1
    assert rc == lbm.LBM_ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly():
    L = lbm.lib()
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_destroy(None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_check(None) == lbm.LBM_ERR_INVALID_ARG


def test_no_cpu_fallback_without_a_device():
    """On a machine without a CUDA device the library refuses (LBM_ERR_CUDA)."""
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a CUDA device is present")
    rc, h = _create()
    assert rc == lbm.LBM_ERR_CUDA
    assert b"CUDA" in lbm.lib().lbm_last_error(None) or b"device" in lbm.lib().lbm_last_error(None)


def test_footprint_estimate_needs_no_device():
    """Admission control sizes a lattice before creating it: populations
    (2 sets in place, 4 ping-pong), P, u (two each), phi; with FP32
    arithmetic the packed (u, P) words (two), the packed (u, phi) words and
    the six second moments of g; with BF16 storage the odd part of g (two);
    scratch, mask."""
    N = 32 ** 3
    scratch = 8 * (1024 * 8 + 64) + 256
    packed = (2 * 16 + 16 + 4 * 6) * N + 4 * (2 + 32)
    got = lbm.estimate_footprint("D3Q27", (32, 32, 32), storage="f16", inplace=1)
    assert got == 2 * 27 * N * 2 + 9 * N * 4 + packed + scratch
    got = lbm.estimate_footprint("D3Q27", (32, 32, 32), storage="bf16", inplace=1)
    assert got == 2 * 27 * N * 2 + 9 * N * 4 + packed + 2 * 16 * N + scratch
    got = lbm.estimate_footprint("D3Q27", (32, 32, 32), periodic=(1, 1, 0), storage="f32")
    assert got == 4 * 27 * N * 4 + 9 * N * 4 + packed + scratch + 4 * N
    got = lbm.estimate_footprint("D2Q9", (16, 8, 1), storage="f64")
    assert got == 4 * 9 * 128 * 8 + 7 * 128 * 8 + scratch
    solid = np.zeros((1, 8, 16), np.uint8)
    solid[0, 3, 3] = 1
    assert lbm.estimate_footprint("D2Q9", (16, 8, 1), solid=solid, storage="f64") == got + 4 * 128
    with pytest.raises(lbm.LbmError):
        lbm.estimate_footprint("D2Q9", (16, 8, 2))


def test_batch_calls_without_a_batch_fail_cleanly():
    L = lbm.lib()
    assert L.lbm_batch_step(None, 1, None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_batch_destroy(None) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_batch_add(None, None, 1) == lbm.LBM_ERR_INVALID_ARG
    assert L.lbm_autotune(None, 1, None, None, None) == lbm.LBM_ERR_INVALID_ARG
    out = ctypes.c_void_p()
    assert L.lbm_batch_create(7, 1, ctypes.byref(out)) == lbm.LBM_ERR_INVALID_ARG
