"""The allocation-free reduction entry point (lbm_reduce_fields_noalloc).

It serves callers that cannot allocate device memory at the point of the
call (real-time loops that must not block in an allocator, hosts whose
device memory belongs to a pool they do not own): inputs and outputs are the
caller's device arrays and the partial sums live in a fixed array inside the
library.  This test checks it against the
handle's own reduction (lbm_reduce) on two calls in a row, through the C
ABI.  Kept in a file of its own that sorts last, so a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_lbm_reduce(lbm):
    torch = pytest.importorskip("torch")
    c = W.poiseuille_2d(nx=40, ny=34, g=1e-6)          # walls: solid rows are skipped by both
    prm = {k: v for k, v in c.params.items() if k != "g_ext"}
    L = lbm.Lattice(c.lattice, c.shape, periodic=c.periodic, solid=c.solid, storage="f64",
                    g_ext=c.params["g_ext"], **prm)
    L.init_fields(c.phi0, c.P0, c.u0)
    N = L.N
    d_phi = torch.empty(N, dtype=torch.float64, device="cuda")
    d_P = torch.empty(N, dtype=torch.float64, device="cuda")
    d_u = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    d_solid = torch.from_numpy(np.ascontiguousarray(c.solid.reshape(-1))).to("cuda")
    d_out = torch.empty(5, dtype=torch.float64, device="cuda")
    lib = lbm.lib()
    for call in range(2):
        L.step(37)
        L.read_fields_device(d_phi, d_P, d_u)
        torch.cuda.synchronize()
        rc = lib.lbm_reduce_fields_noalloc(d_phi.data_ptr(), d_u.data_ptr(), d_solid.data_ptr(), N,
                                           L.params.rho_w, L.params.rho_a, L.params.clamp_phi_props,
                                           d_out.data_ptr(), None)
        assert rc == lbm.LBM_OK
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        want = L.reduce()
        ref = np.array([want["mass"], *want["momentum"], want["fluid_sites"]])
        assert got[4] == ref[4] == (34 - 2) * 40
        scale = np.maximum(np.abs(ref), 1e-300)
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (call, got, ref)


def test_noalloc_rejects_bad_sizes(lbm):
    torch = pytest.importorskip("torch")
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    lib = lbm.lib()
    for n in (0, -1, 2 ** 31):
        rc = lib.lbm_reduce_fields_noalloc(d.data_ptr(), d.data_ptr(), None, n, 1.0, 1e-3, 1,
                                           d.data_ptr(), None)
        assert rc == lbm.LBM_ERR_INVALID_ARG
    # densities must satisfy rho_w > rho_a > 0; device pointers must be given
    for rho_w, rho_a in ((1e-3, 1e-3), (1e-3, 1.0), (1.0, 0.0), (1.0, -1e-3)):
        rc = lib.lbm_reduce_fields_noalloc(d.data_ptr(), d.data_ptr(), None, 8, rho_w, rho_a, 1,
                                           d.data_ptr(), None)
        assert rc == lbm.LBM_ERR_INVALID_ARG
    for ptrs in ((d.data_ptr(), d.data_ptr(), None), (None, d.data_ptr(), d.data_ptr()),
                 (d.data_ptr(), None, d.data_ptr())):
        rc = lib.lbm_reduce_fields_noalloc(ptrs[0], ptrs[1], None, 8, 1.0, 1e-3, 1, ptrs[2], None)
        assert rc == lbm.LBM_ERR_INVALID_ARG
