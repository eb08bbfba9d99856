"""FP64 CPU oracle of the coupled phase-field / pressure-velocity LB step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_2512_01027_gb300``) never imports it and shares no code
with it.

The arithmetic lives in ``lbm_oracle.c`` (plain per-site loops, FP64, built
with ``-ffp-contract=off`` so no fused multiply-adds reorder the rounding);
this module only compiles it and marshals numpy arrays through ctypes.
``crosscheck_np`` holds an independent NumPy restatement of the D2Q9 periodic
case that pins the C oracle against a second transcription of Sec. II.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19, D3Q27 = 0, 1, 2
LATTICE_IDS = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into a shared library (gcc, FP64, no FP contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of orc_params (lbm_oracle.c)."""

    _fields_ = [(n, ctypes.c_double) for n in (
        "rho_w", "rho_a", "nu_w", "nu_a", "sigma", "M", "W", "lambda_b",
        "gamma", "phi_n", "phi_m", "D", "eps")] + [
        ("g_ext", ctypes.c_double * 3),
        ("clamp_phi_props", ctypes.c_int32),
        ("filter_full_trace", ctypes.c_int32),
        ("coupling_unew", ctypes.c_int32),
    ]


def make_params(**kw) -> Params:
    """Parameter block with the paper's defaults (Sec. II, Sec. III):
    lambda_b = 1/6, gamma = -22.5, phi_n = 0.8, phi_m = 0.2, D = 1e-4,
    eps = 1e-10, M = 0.166, W = 4."""
    d = dict(rho_w=1.0, rho_a=1e-3, nu_w=0.0167, nu_a=0.167, sigma=1e-3,
             M=0.166, W=4.0, lambda_b=1.0 / 6.0, gamma=-22.5, phi_n=0.8,
             phi_m=0.2, D=1e-4, eps=1e-10, g_ext=(0.0, 0.0, 0.0),
             clamp_phi_props=1)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k == "g_ext":
            for a in range(3):
                p.g_ext[a] = float(v[a]) if a < len(v) else 0.0
        else:
            setattr(p, k, v)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            vp = ctypes.c_void_p
            L.orc_create.restype = vp
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                     ctypes.POINTER(Params)]
            L.orc_destroy.argtypes = [vp]
            L.orc_init.argtypes = [vp, dp, dp, dp, ctypes.c_int]
            L.orc_step.argtypes = [vp, ctypes.c_long]
            L.orc_fields.argtypes = [vp, dp, dp, dp]
            L.orc_get_state.argtypes = [vp, dp, dp, dp, dp]
            L.orc_set_state.argtypes = [vp, dp, dp, dp, dp]
            L.orc_steps_done.argtypes = [vp]
            L.orc_steps_done.restype = ctypes.c_long
            L.orc_grad_lap.argtypes = [vp, dp, ctypes.c_int, dp, dp]
            L.orc_k_terms.argtypes = [vp, dp, dp, dp, dp, dp]
            L.orc_h_eq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_double, dp]
            L.orc_g_eq.argtypes = [ctypes.c_int, ctypes.POINTER(Params), ctypes.c_double,
                                   ctypes.c_double, dp, dp, ctypes.c_double, ctypes.c_double,
                                   dp, dp, dp]
            L.orc_filter.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, ctypes.c_int]
            L.orc_delta_theta.argtypes = [ctypes.POINTER(Params), ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double]
            L.orc_delta_theta.restype = ctypes.c_double
            L.orc_lattice_info.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), dp]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def lattice_info(lattice):
    """(d, Q, c [Q,3] int, w [Q]) of the oracle's own lattice table."""
    lid = LATTICE_IDS.get(lattice, lattice)
    d = ctypes.c_int()
    Q = ctypes.c_int()
    c = (ctypes.c_int * 81)()
    w = np.zeros(27)
    if lib().orc_lattice_info(lid, ctypes.byref(d), ctypes.byref(Q), c, _dp(w)) != 0:
        raise ValueError(lattice)
    q = Q.value
    return d.value, q, np.array(c[: 3 * q], dtype=np.int64).reshape(q, 3), w[:q].copy()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Oracle:
    """One lattice state advanced by the FP64 oracle.

    shape = (nx, ny, nz); arrays are returned as [nz, ny, nx] (x fastest),
    vector fields as [3, nz, ny, nx]."""

    def __init__(self, lattice, shape, params: Params | None = None, periodic=(1, 1, 1),
                 solid=None):
        self.lattice = LATTICE_IDS.get(lattice, lattice)
        self.d, self.Q, self.c, self.w = lattice_info(self.lattice)
        nx, ny, nz = (tuple(shape) + (1, 1))[:3]
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.params = params if params is not None else make_params()
        per = (ctypes.c_int32 * 3)(*[int(v) for v in periodic])
        self._solid = None
        sp = None
        if solid is not None:
            self._solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
            if self._solid.size != self.N:
                raise ValueError("solid mask size")
            sp = self._solid.ctypes.data_as(ctypes.c_void_p)
        self._h = lib().orc_create(self.lattice, nx, ny, nz, per, sp, ctypes.byref(self.params))
        if not self._h:
            raise ValueError("orc_create failed (bad lattice/shape)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def _grid(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def init(self, phi0, P0, u0):
        phi0 = _f64(phi0, self.N)
        P0 = _f64(P0, self.N)
        u0 = _f64(u0)
        ncomp = u0.size // self.N
        if u0.size != ncomp * self.N or ncomp not in (2, 3):
            raise ValueError("u0 must hold 2 or 3 component planes")
        if lib().orc_init(self._h, _dp(phi0), _dp(P0), _dp(u0), ncomp) != 0:
            raise ValueError("orc_init failed")

    def step(self, n: int = 1):
        if lib().orc_step(self._h, int(n)) != 0:
            raise ValueError("orc_step failed")

    @property
    def steps_done(self) -> int:
        return int(lib().orc_steps_done(self._h))

    def fields(self):
        phi = np.zeros(self.N)
        P = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        lib().orc_fields(self._h, _dp(phi), _dp(P), _dp(u))
        g = self._grid()
        return phi.reshape(g), P.reshape(g), u.reshape((3,) + g)

    def get_state(self):
        h = np.zeros(self.Q * self.N)
        g = np.zeros(self.Q * self.N)
        P = np.zeros(self.N)
        u = np.zeros(3 * self.N)
        lib().orc_get_state(self._h, _dp(h), _dp(g), _dp(P), _dp(u))
        gr = self._grid()
        return (h.reshape((self.Q,) + gr), g.reshape((self.Q,) + gr), P.reshape(gr),
                u.reshape((3,) + gr))

    def set_state(self, h, g, P, u):
        h = _f64(h, self.Q * self.N)
        g = _f64(g, self.Q * self.N)
        P = _f64(P, self.N)
        u = _f64(u, 3 * self.N)
        lib().orc_set_state(self._h, _dp(h), _dp(g), _dp(P), _dp(u))

    def grad_lap(self, f, solid_value_zero: bool = False):
        f = _f64(f, self.N)
        grad = np.zeros(3 * self.N)
        lap = np.zeros(self.N)
        lib().orc_grad_lap(self._h, _dp(f), 1 if solid_value_zero else 0, _dp(grad), _dp(lap))
        gr = self._grid()
        return grad.reshape((3,) + gr), lap.reshape(gr)

    def k_terms(self, P, rho, u):
        P = _f64(P, self.N)
        rho = _f64(rho, self.N)
        u = _f64(u, 3 * self.N)
        K = np.zeros(self.Q * self.N)
        wcu = np.zeros(self.N)
        lib().orc_k_terms(self._h, _dp(P), _dp(rho), _dp(u), _dp(K), _dp(wcu))
        gr = self._grid()
        return K.reshape((self.Q,) + gr), wcu.reshape(gr)


def h_eq(lattice, phi, u, n, theta_tot):
    lid = LATTICE_IDS.get(lattice, lattice)
    out = np.zeros(27)
    lib().orc_h_eq(lid, float(phi), _dp(_f64(u, 3)), _dp(_f64(n, 3)), float(theta_tot), _dp(out))
    return out[: lattice_info(lid)[1]].copy()


def g_eq(lattice, params, P, rho, u, F, B, div, sigma, grad_rho):
    lid = LATTICE_IDS.get(lattice, lattice)
    out = np.zeros(27)
    lib().orc_g_eq(lid, ctypes.byref(params), float(P), float(rho), _dp(_f64(u, 3)),
                   _dp(_f64(F, 3)), float(B), float(div), _dp(_f64(sigma, 9)),
                   _dp(_f64(grad_rho, 3)), _dp(out))
    return out[: lattice_info(lid)[1]].copy()


def filter_collision(lattice, tau, g, geq, full_trace: bool = False):
    lid = LATTICE_IDS.get(lattice, lattice)
    q = lattice_info(lid)[1]
    g = _f64(g, q)
    geq = _f64(geq, q)
    out = np.zeros(q)
    lib().orc_filter(lid, float(tau), _dp(g), _dp(geq), _dp(out), 1 if full_trace else 0)
    return out


def delta_theta(params, phi, grad_norm, lap):
    return float(lib().orc_delta_theta(ctypes.byref(params), float(phi), float(grad_norm),
                                       float(lap)))


def run(lattice, shape, params, phi0, P0, u0, nsteps, periodic=(1, 1, 1), solid=None):
    """Convenience: init from fields, advance nsteps, return (phi, P, u)."""
    o = Oracle(lattice, shape, params, periodic=periodic, solid=solid)
    o.init(phi0, P0, u0)
    o.step(nsteps)
    return o.fields()
