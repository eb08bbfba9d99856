"""Python binding of the GB300 coupled multiphase LB step library.

Thin ctypes marshalling over the C ABI in ``include/lbm.h``; every step of
the method runs in the CUDA kernels of ``csrc/``.  There is no CPU path: if
the shared library cannot be built or loaded, or no CUDA device is present,
the calls raise.

PyTorch is used only as plumbing: the current torch CUDA stream can be handed
to a lattice (``set_stream``), device arrays may be torch tensors, and
``use_torch_allocator()`` routes the library's device allocations through
torch's caching allocator.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Lattice", "Batch", "estimate_footprint", "lib", "build", "default_params", "lattice_info", "LbmError",
           "D2Q9", "D3Q19", "D3Q27", "F64", "F32", "F16DEV", "BF16DEV"]

D2Q9, D3Q19, D3Q27 = 0, 1, 2
F64, F32, F16DEV, BF16DEV = 0, 1, 2, 3
LATTICES = {"D2Q9": D2Q9, "D3Q19": D3Q19, "D3Q27": D3Q27}
STORAGES = {"f64": F64, "f32": F32, "f16": F16DEV, "bf16": BF16DEV}

(LBM_OK, LBM_ERR_INVALID_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_UNSUPPORTED,
 LBM_ERR_TIMEOUT) = range(7)
_ERR_NAMES = {1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "NONFINITE", 5: "UNSUPPORTED", 6: "TIMEOUT"}


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"LBM_ERR_{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3), ("solid", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint64)] + [(n, ctypes.c_double) for n in (
        "rho_w", "rho_a", "nu_w", "nu_a", "sigma", "M", "W", "lambda_b", "gamma", "phi_n",
        "phi_m", "D", "eps")] + [("g_ext", ctypes.c_double * 3),
                                ("clamp_phi_props", ctypes.c_int32),
                                ("filter_full_trace", ctypes.c_int32),
                                ("storage", ctypes.c_int32), ("inplace", ctypes.c_int32),
                                ("coupling_unew", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None

# every exported symbol of include/lbm.h with (restype, argtypes)
_vp, _dp, _i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
SIGNATURES = {
    "lbm_default_params": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "lbm_lattice_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Params),
                                  ctypes.POINTER(_vp)]),
    "lbm_destroy": (ctypes.c_int, [_vp]),
    "lbm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbm_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _vp]),
    "lbm_init_fields": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_init_fields_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_step": (ctypes.c_int, [_vp, _i64]),
    "lbm_read_fields": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "lbm_read_fields_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "lbm_steps_done": (ctypes.c_int, [_vp, ctypes.POINTER(_i64)]),
    "lbm_check": (ctypes.c_int, [_vp]),
    "lbm_reduce": (ctypes.c_int, [_vp, _dp]),
    "lbm_pressure_jump": (ctypes.c_int, [_vp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
    "lbm_get_state": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "lbm_probe": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(_i64), _dp, _dp, _dp, _dp]),
    "lbm_state_bytes": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_save_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "lbm_load_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "lbm_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_set_cluster": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_footprint": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_reduce_fields_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int32, _vp, _vp]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
    "lbm_debug_stall": (ctypes.c_int, [_vp, ctypes.c_int]),
    "lbm_estimate_footprint": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Params),
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    _dp]),
    "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    "lbm_batch_destroy": (ctypes.c_int, [_vp]),
    "lbm_batch_set_stream": (ctypes.c_int, [_vp, _vp]),
    "lbm_batch_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_set_shape": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "lbm_batch_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]),
    "lbm_batch_add": (ctypes.c_int, [_vp, _vp, _i64]),
    "lbm_batch_remove": (ctypes.c_int, [_vp, _vp]),
    "lbm_batch_step": (ctypes.c_int, [_vp, _i64, ctypes.POINTER(ctypes.c_int)]),
    "lbm_batch_remaining": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_i64)]),
    "lbm_batch_pause": (ctypes.c_int, [_vp, _vp, ctypes.c_int32]),
    "lbm_batch_info": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64)]),
    "lbm_batch_last_error": (ctypes.c_char_p, [_vp]),
}


def build(force: bool = False) -> str:
    return _build.build(force=force)


def lib():
    """Load (building first if needed) the CUDA library.  Raises on failure."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc, handle=None):
    if rc != LBM_OK:
        msg = lib().lbm_last_error(handle)
        raise LbmError(rc, msg.decode() if msg else "")


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def default_params(**kw) -> Params:
    p = Params()
    _check(lib().lbm_default_params(ctypes.byref(p)))
    for k, v in kw.items():
        if k == "g_ext":
            for a in range(3):
                p.g_ext[a] = float(v[a]) if a < len(v) else 0.0
        elif k == "storage":
            p.storage = STORAGES.get(v, v)
        else:
            setattr(p, k, v)
    return p


def lattice_info(lattice):
    """(d, Q, c [Q,3], w [Q]) of the library's direction table."""
    lid = LATTICES.get(lattice, lattice)
    d = ctypes.c_int()
    Q = ctypes.c_int()
    c = (ctypes.c_int * 81)()
    w = np.zeros(27)
    _check(lib().lbm_lattice_info(lid, ctypes.byref(d), ctypes.byref(Q), c, _d(w)))
    q = Q.value
    return d.value, q, np.array(c[: 3 * q]).reshape(q, 3), w[:q].copy()


_torch_hooks = None


def estimate_footprint(lattice, shape, periodic=(1, 1, 1), solid=None, storage="f32", inplace=0) -> int:
    """Device bytes a Lattice of this description would hold (no device
    needed, nothing allocated)."""
    nx, ny, nz = (tuple(shape) + (1, 1))[:3]
    g = Grid()
    g.nx, g.ny, g.nz = nx, ny, nz
    for a in range(3):
        g.periodic[a] = int(periodic[a])
    keep = None
    if solid is not None:
        keep = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
        g.solid = keep.ctypes.data
    p = default_params(storage=storage, inplace=int(inplace))
    out = ctypes.c_size_t()
    _check(lib().lbm_estimate_footprint(ctypes.byref(g), LATTICES.get(lattice, lattice), ctypes.byref(p),
                                        ctypes.byref(out)))
    return out.value


def use_torch_allocator(enable: bool = True) -> None:
    """Route device allocations of later Lattice() calls through torch's
    caching allocator (current device, current stream)."""
    global _torch_hooks
    import torch

    if not enable:
        _check(lib().lbm_set_allocator(ALLOC_FN(), FREE_FN(), None))
        _torch_hooks = None
        return

    def _alloc(nbytes, _ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
        except Exception:
            return None

    def _free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().lbm_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


class Lattice:
    """One lattice state on the current CUDA device.

    shape = (nx, ny, nz); host fields are numpy arrays [nz, ny, nx] (x fastest),
    vector fields [3, nz, ny, nx]."""

    def __init__(self, lattice, shape, params: Params | None = None, periodic=(1, 1, 1), solid=None,
                 storage=None, **param_kw):
        self.lattice = LATTICES.get(lattice, lattice)
        nx, ny, nz = (tuple(shape) + (1, 1))[:3]
        self.shape = (nx, ny, nz)
        self.N = nx * ny * nz
        self.d, self.Q, self.c, self.w = lattice_info(self.lattice)
        p = params if params is not None else default_params(**param_kw)
        if storage is not None:
            p.storage = STORAGES.get(storage, storage)
        self.params = p
        g = Grid()
        g.nx, g.ny, g.nz = nx, ny, nz
        for a in range(3):
            g.periodic[a] = int(periodic[a])
        self._solid = None
        if solid is not None:
            self._solid = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
            if self._solid.size != self.N:
                raise ValueError("solid mask size")
            g.solid = self._solid.ctypes.data
        self._h = _vp()
        rc = lib().lbm_create(ctypes.byref(g), self.lattice, ctypes.byref(p), ctypes.byref(self._h))
        _check(rc, None)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    def _grid(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    # -- streams
    def set_stream(self, stream=None):
        """stream: a torch.cuda.Stream, an int handle, or None (legacy default)."""
        ptr = None
        if stream is not None:
            ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib().lbm_set_stream(self._h, ptr), self._h)

    # -- fields
    def init_fields(self, phi, P, u):
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1)
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1)
        u = np.asarray(u, dtype=np.float64).reshape(-1, self.N)
        if phi.size != self.N or P.size != self.N or u.shape[0] not in (2, 3):
            raise ValueError("field sizes")
        u3 = np.zeros((3, self.N))
        u3[: u.shape[0]] = u
        _check(lib().lbm_init_fields(self._h, _d(phi), _d(P), _d(u3)), self._h)

    def init_fields_device(self, phi, P, u):
        """phi, P: float64 CUDA tensors [N]; u: float64 CUDA tensor [3, N]."""
        _check(lib().lbm_init_fields_device(self._h, phi.data_ptr(), P.data_ptr(), u.data_ptr()), self._h)

    def step(self, n: int = 1):
        _check(lib().lbm_step(self._h, int(n)), self._h)

    def read_fields(self):
        phi = np.empty(self.N)
        P = np.empty(self.N)
        u = np.empty(3 * self.N)
        _check(lib().lbm_read_fields(self._h, _d(phi), _d(P), _d(u)), self._h)
        g = self._grid()
        return phi.reshape(g), P.reshape(g), u.reshape((3,) + g)

    def read_fields_device(self, phi, P, u):
        _check(lib().lbm_read_fields_device(self._h, phi.data_ptr() if phi is not None else None,
                                            P.data_ptr() if P is not None else None,
                                            u.data_ptr() if u is not None else None), self._h)

    @property
    def steps_done(self) -> int:
        s = ctypes.c_int64()
        _check(lib().lbm_steps_done(self._h, ctypes.byref(s)), self._h)
        return s.value

    def check(self):
        _check(lib().lbm_check(self._h), self._h)

    def reduce(self):
        out = np.zeros(5)
        _check(lib().lbm_reduce(self._h, _d(out)), self._h)
        return dict(mass=out[0], momentum=out[1:4].copy(), fluid_sites=out[4])

    def pressure_jump(self, center, r_in, r_out) -> float:
        c = np.ascontiguousarray(center, dtype=np.float64)
        dP = ctypes.c_double()
        _check(lib().lbm_pressure_jump(self._h, _d(c), float(r_in), float(r_out), ctypes.byref(dP)), self._h)
        return dP.value

    def get_state(self):
        h = np.empty(self.Q * self.N)
        g = np.empty(self.Q * self.N)
        P = np.empty(self.N)
        u = np.empty(3 * self.N)
        _check(lib().lbm_get_state(self._h, _d(h), _d(g), _d(P), _d(u)), self._h)
        gr = self._grid()
        return (h.reshape((self.Q,) + gr), g.reshape((self.Q,) + gr), P.reshape(gr), u.reshape((3,) + gr))

    def probe(self, sites):
        """Decoded state at linear site indices: (h [n,Q], g [n,Q], P [n], u [n,3])."""
        s = np.ascontiguousarray(sites, dtype=np.int64).reshape(-1)
        n = s.size
        h = np.empty((n, self.Q))
        g = np.empty((n, self.Q))
        P = np.empty(n)
        u = np.empty((n, 3))
        _check(lib().lbm_probe(self._h, n, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _d(h), _d(g),
                               _d(P), _d(u)), self._h)
        return h, g, P, u

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        _check(lib().lbm_state_bytes(self._h, ctypes.byref(n)), self._h)
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().lbm_save_state(self._h, buf, n.value), self._h)
        return buf.raw

    def load_state(self, data: bytes):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib().lbm_load_state(self._h, buf, len(data)), self._h)

    def set_tuning(self, variant: int = 0, zchunk: int = 0):
        """variant 0 auto, 1 fused plane-synchronous, 2 fused pipelined, 3 split form,
        4 persistent split form, 5 cluster step; zchunk 0 = auto."""
        _check(lib().lbm_set_tuning(self._h, int(variant), int(zchunk)), self._h)

    def set_cluster(self, rows: int = 0, staged: int = -1):
        """Cluster step shape: CTAs (rows) per cluster (0 = auto) and whether the
        pulled rows are staged by bulk copies (-1 = default, no; 0 = no; 1 = yes)."""
        _check(lib().lbm_set_cluster(self._h, int(rows), int(staged)), self._h)

    def debug_stall(self, plane: int):
        """Testing aid of the persistent step's failure path (see lbm.h)."""
        _check(lib().lbm_debug_stall(self._h, int(plane)), self._h)

    def autotune(self, trial_steps: int = 5):
        """Time every launch form on this lattice's state, keep the fastest,
        restore the state.  Returns (variant, zchunk, ms_per_step)."""
        v, z, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().lbm_autotune(self._h, int(trial_steps), ctypes.byref(v), ctypes.byref(z), ctypes.byref(ms)),
               self._h)
        return v.value, z.value, ms.value

    def footprint(self):
        dev = ctypes.c_size_t()
        step = ctypes.c_size_t()
        _check(lib().lbm_footprint(self._h, ctypes.byref(dev), ctypes.byref(step)), self._h)
        return dev.value, step.value


def _bcheck(rc, b):
    if rc != LBM_OK:
        msg = lib().lbm_batch_last_error(b)
        raise LbmError(rc, msg.decode() if msg else "")


class Batch:
    """Lattices of one DdQq and storage stepped together: two kernel launches
    per time step for the whole set, chunks of steps replayed as CUDA graphs.
    Members are Lattice objects with a step budget each."""

    def __init__(self, lattice="D3Q27", storage="f32"):
        self._b = _vp()
        self.members = []
        _check(lib().lbm_batch_create(LATTICES.get(lattice, lattice), STORAGES.get(storage, storage),
                                      ctypes.byref(self._b)))

    def close(self):
        if getattr(self, "_b", None):
            lib().lbm_batch_destroy(self._b)
            self._b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        ptr = None
        if stream is not None:
            ptr = stream if isinstance(stream, int) else stream.cuda_stream
        _bcheck(lib().lbm_batch_set_stream(self._b, ptr), self._b)

    def set_tuning(self, chunk: int = 16, use_graph: bool = True):
        _bcheck(lib().lbm_batch_set_tuning(self._b, int(chunk), int(bool(use_graph))), self._b)

    def set_shape(self, span: int = 1, blocks_per_sm: int = 0):
        """Work item span (blocks of 128 sites) and persistent blocks per SM (0 = all that fit)."""
        _bcheck(lib().lbm_batch_set_shape(self._b, int(span), int(blocks_per_sm)), self._b)

    def autotune(self, trial_steps: int = 32):
        """Time the launch shapes on the current members, keep the fastest,
        restore every member's state and budget.  Returns (chunk, span,
        blocks_per_sm, ms_per_step)."""
        K, sp, bps, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _bcheck(lib().lbm_batch_autotune(self._b, int(trial_steps), ctypes.byref(K), ctypes.byref(sp),
                                         ctypes.byref(bps), ctypes.byref(ms)), self._b)
        return K.value, sp.value, bps.value, ms.value

    def add(self, lat: "Lattice", steps: int):
        _bcheck(lib().lbm_batch_add(self._b, lat.handle, int(steps)), self._b)
        self.members.append(lat)

    def remove(self, lat: "Lattice"):
        _bcheck(lib().lbm_batch_remove(self._b, lat.handle), self._b)
        self.members.remove(lat)

    def pause(self, lat: "Lattice", paused: bool = True):
        """A paused member takes no steps (budget, state and memory kept)."""
        _bcheck(lib().lbm_batch_pause(self._b, lat.handle, int(bool(paused))), self._b)

    def step(self, n: int) -> int:
        """Advance every unpaused member by min(n, its remaining budget);
        returns the number of members whose budget is spent."""
        f = ctypes.c_int()
        _bcheck(lib().lbm_batch_step(self._b, int(n), ctypes.byref(f)), self._b)
        return f.value

    def remaining(self, lat: "Lattice") -> int:
        r = _i64()
        _bcheck(lib().lbm_batch_remaining(self._b, lat.handle, ctypes.byref(r)), self._b)
        return r.value

    def info(self):
        m, n = ctypes.c_int(), _i64()
        _bcheck(lib().lbm_batch_info(self._b, ctypes.byref(m), ctypes.byref(n)), self._b)
        return m.value, n.value
