"""ctypes binding of the C ABI in ``include/lbm.h`` (same names, argument marshalling only).

Every step of the scheme runs in the CUDA library ``_build/liblbmch.so``; if that library is
missing this module raises on import — there is no CPU fallback.  PyTorch supplies device memory
(the population buffers are one ``torch.uint8`` CUDA tensor handed to ``lbm_init``) and the stream
(``torch.cuda.current_stream()``).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

LBM_OK, LBM_ERR_PARAM, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S = 0, 1, 2, 3
LBM_PERIODIC, LBM_WALLS_Y = 0, 1
LBM_OMEGA_LINEAR, LBM_TAU_LINEAR = 0, 1
LBM_K8_PROJECTED, LBM_K8_PRINTED = 0, 1
LBM_COLLIDE_CM, LBM_COLLIDE_BGK = 0, 1
LBM_FORCE_UNIFORM, LBM_FORCE_PHASE_L = 0, 1
LBM_ROUND_NEAREST, LBM_ROUND_STOCHASTIC = 0, 1
LBM_KERNEL_AUTO, LBM_KERNEL_GENERIC, LBM_KERNEL_STAGED, LBM_KERNEL_GENERIC_WIDE, LBM_KERNEL_PAIR = 0, 1, 2, 3, 4
LBM_KERNEL_PAIR_STAGED = 5

PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau_l", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("M", ctypes.c_double), ("Gamma", ctypes.c_double),
        ("gamma", ctypes.c_double), ("a", ctypes.c_double),
        ("omega3", ctypes.c_double),
        ("k8_form", ctypes.c_int), ("visc", ctypes.c_int), ("bc", ctypes.c_int),
        ("u_top", ctypes.c_double), ("u_bottom", ctypes.c_double),
        ("prec", ctypes.c_int), ("collision", ctypes.c_int),
        ("wet_bottom", ctypes.c_double), ("wet_top", ctypes.c_double),
        ("force_x", ctypes.c_double), ("force_y", ctypes.c_double), ("force_mode", ctypes.c_int),
        ("rounding", ctypes.c_int), ("seed", ctypes.c_uint),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is not built; run paper_1803_11345_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, dp, i, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_size_t
    pp = ctypes.POINTER(lbm_params)
    lib.lbm_default_params.argtypes = [pp]
    lib.lbm_default_params.restype = None
    lib.lbm_wall_gradient.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.lbm_wall_gradient.restype = ctypes.c_double
    lib.lbm_state_bytes.argtypes = [pp, ctypes.POINTER(sz)]
    lib.lbm_state_bytes.restype = i
    lib.lbm_init.argtypes = [pp, dp, dp, dp, dp, vp, sz, vp, ctypes.POINTER(vp)]
    lib.lbm_init.restype = i
    lib.lbm_step.argtypes = [vp, i]
    lib.lbm_step.restype = i
    lib.lbm_fields.argtypes = [vp, dp, dp, dp, dp]
    lib.lbm_fields.restype = i
    lib.lbm_conservation.argtypes = [vp, dp, dp, dp]
    lib.lbm_conservation.restype = i
    lib.lbm_get_populations.argtypes = [vp, dp, dp]
    lib.lbm_get_populations.restype = i
    lib.lbm_set_populations.argtypes = [vp, dp, dp]
    lib.lbm_set_populations.restype = i
    lib.lbm_check.argtypes = [vp]
    lib.lbm_check.restype = i
    lib.lbm_set_wait_limit.argtypes = [vp, i]
    lib.lbm_set_wait_limit.restype = i
    lib.lbm_set_kernel.argtypes = [vp, i, i, i, i, i]
    lib.lbm_set_kernel.restype = i
    ip = ctypes.POINTER(ctypes.c_int)
    lib.lbm_get_kernel.argtypes = [vp, ip, ip, ip, ip, ip]
    lib.lbm_get_kernel.restype = i
    lib.lbm_autotune.argtypes = [vp, i, dp]
    lib.lbm_autotune.restype = i
    bp = ctypes.POINTER(ctypes.c_void_p)
    lib.lbm_batch_state_bytes.argtypes = [pp, i, ctypes.POINTER(sz)]
    lib.lbm_batch_state_bytes.restype = i
    lib.lbm_batch_init.argtypes = [pp, i, ctypes.POINTER(dp), vp, sz, vp, bp]
    lib.lbm_batch_init.restype = i
    lib.lbm_batch_step.argtypes = [vp, i]
    lib.lbm_batch_step.restype = i
    lib.lbm_batch_fields.argtypes = [vp, i, dp, dp, dp, dp]
    lib.lbm_batch_fields.restype = i
    lib.lbm_batch_get_populations.argtypes = [vp, i, dp, dp]
    lib.lbm_batch_get_populations.restype = i
    lib.lbm_batch_set_state.argtypes = [vp, i, vp]
    lib.lbm_batch_set_state.restype = i
    lib.lbm_batch_get_state.argtypes = [vp, i, vp]
    lib.lbm_batch_get_state.restype = i
    lib.lbm_batch_check.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.lbm_batch_check.restype = i
    lib.lbm_batch_set_tile.argtypes = [vp, i, i, i]
    lib.lbm_batch_set_tile.restype = i
    lib.lbm_batch_get_tile.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 5
    lib.lbm_batch_get_tile.restype = i
    lib.lbm_batch_set_kernel.argtypes = [vp, i, i]
    lib.lbm_batch_set_kernel.restype = i
    lib.lbm_batch_get_kernel.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.lbm_batch_get_kernel.restype = i
    lib.lbm_batch_autotune.argtypes = [vp, i, dp]
    lib.lbm_batch_autotune.restype = i
    lib.lbm_batch_time.argtypes = [vp]
    lib.lbm_batch_time.restype = ctypes.c_longlong
    lib.lbm_batch_last_error.argtypes = [vp]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    lib.lbm_batch_free.argtypes = [vp]
    lib.lbm_batch_free.restype = None
    lib.lbm_totals_noalloc.argtypes = [vp, i, i, i, dp, vp]
    lib.lbm_totals_noalloc.restype = i
    lib.lbm_time.argtypes = [vp]
    lib.lbm_time.restype = ctypes.c_longlong
    lib.lbm_last_error.argtypes = [vp]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_free.argtypes = [vp]
    lib.lbm_free.restype = None
    return lib


_lib = _load()


def declared_functions(header: str = HEADER):
    """Names of the functions declared in include/lbm.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M)))


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _check(status: int, h=None):
    if status != LBM_OK:
        msg = _lib.lbm_last_error(h).decode(errors="replace")
        raise LbmError(status, msg)


# ------------------------------------------------------------------------------------------
# Same-name wrappers of the C entry points.

def lbm_default_params(**overrides) -> lbm_params:
    p = lbm_params()
    _lib.lbm_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if k == "prec" and isinstance(v, str):
            v = PRECISIONS[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def lbm_wall_gradient(theta: float, a: float, gamma: float) -> float:
    """Eq. 18: wall gradient of phi along the outward normal for contact angle theta (radians)."""
    return _lib.lbm_wall_gradient(float(theta), float(a), float(gamma))


def lbm_state_bytes(p: lbm_params) -> int:
    n = ctypes.c_size_t(0)
    _check(_lib.lbm_state_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def lbm_init(p: lbm_params, phi0, ux0=None, uy0=None, rho0=None, device_buffer: int = 0,
             buffer_bytes: int = 0, stream: int = 0) -> int:
    n = p.nx * p.ny
    arrs = [_f64(phi0, n), _f64(ux0, n), _f64(uy0, n), _f64(rho0, n)]
    h = ctypes.c_void_p()
    st = _lib.lbm_init(ctypes.byref(p), *(_dptr(a) for a in arrs), ctypes.c_void_p(device_buffer or None),
                       buffer_bytes, ctypes.c_void_p(stream or None), ctypes.byref(h))
    _check(st, None)
    return h.value


def lbm_step(h: int, n: int) -> None:
    _check(_lib.lbm_step(h, int(n)), h)


def lbm_fields(h: int, rho=None, ux=None, uy=None, phi=None) -> int:
    """Fill the given float64 arrays; returns the status (NONFINITE is returned, not raised)."""
    st = _lib.lbm_fields(h, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(phi))
    if st not in (LBM_OK, LBM_ERR_NONFINITE):
        _check(st, h)
    return st


def lbm_conservation(h: int):
    sp, sr = ctypes.c_double(), ctypes.c_double()
    mom = (ctypes.c_double * 2)()
    _check(_lib.lbm_conservation(h, ctypes.byref(sp), ctypes.byref(sr), mom), h)
    return sp.value, sr.value, mom[0], mom[1]


def lbm_get_populations(h: int, f, g) -> None:
    _check(_lib.lbm_get_populations(h, _dptr(f), _dptr(g)), h)


def lbm_set_populations(h: int, f, g) -> None:
    _check(_lib.lbm_set_populations(h, _dptr(f), _dptr(g)), h)


def lbm_check(h: int) -> int:
    return _lib.lbm_check(h)


def lbm_set_wait_limit(h: int, probes: int) -> None:
    _check(_lib.lbm_set_wait_limit(h, int(probes)), h)


def lbm_set_kernel(h: int, variant: int, bx: int = 0, by: int = 0, depth: int = 0, rows: int = 0) -> None:
    _check(_lib.lbm_set_kernel(h, variant, bx, by, depth, rows), h)


def lbm_get_kernel(h: int):
    """(variant, bx, by, depth, rows) of the fused-step kernel in use."""
    v = [ctypes.c_int() for _ in range(5)]
    _check(_lib.lbm_get_kernel(h, *(ctypes.byref(x) for x in v)), h)
    return tuple(x.value for x in v)


def lbm_totals_noalloc(state: int, nx: int, ny: int, prec: int, stream: int = 0):
    """Totals (sum phi, sum rho, sum rho vx, sum rho vy) of a device population state; see
    include/lbm.h for the layout.  Allocates no device memory."""
    out = (ctypes.c_double * 4)()
    _check(_lib.lbm_totals_noalloc(ctypes.c_void_p(state), nx, ny, prec,
                                   ctypes.cast(out, ctypes.POINTER(ctypes.c_double)),
                                   ctypes.c_void_p(stream or None)), None)
    return tuple(out)


def lbm_autotune(h: int, trial_steps: int = 5) -> float:
    """Pick the fastest kernel/tile for this lattice (state unchanged); returns ms per step."""
    ms = ctypes.c_double()
    _check(_lib.lbm_autotune(h, trial_steps, ctypes.byref(ms)), h)
    return ms.value


def _bcheck(status: int, b=None):
    if status != LBM_OK:
        raise LbmError(status, _lib.lbm_batch_last_error(b).decode(errors="replace"))


def lbm_batch_state_bytes(params) -> int:
    arr = (lbm_params * len(params))(*params)
    n = ctypes.c_size_t()
    _bcheck(_lib.lbm_batch_state_bytes(arr, len(params), ctypes.byref(n)))
    return n.value


def lbm_batch_init(params, phi0s, device_buffer: int = 0, buffer_bytes: int = 0, stream: int = 0) -> int:
    arr = (lbm_params * len(params))(*params)
    keep = [_f64(p0, p.nx * p.ny) for p, p0 in zip(params, phi0s)]
    ptrs = (ctypes.POINTER(ctypes.c_double) * len(keep))(*[_dptr(a) for a in keep])
    b = ctypes.c_void_p()
    _bcheck(_lib.lbm_batch_init(arr, len(params), ptrs, ctypes.c_void_p(device_buffer or None), buffer_bytes,
                                ctypes.c_void_p(stream or None), ctypes.byref(b)))
    return b.value


def lbm_batch_step(b: int, n: int) -> None:
    _bcheck(_lib.lbm_batch_step(b, int(n)), b)


def lbm_batch_fields(b: int, member: int, rho=None, ux=None, uy=None, phi=None) -> None:
    _bcheck(_lib.lbm_batch_fields(b, member, _dptr(rho), _dptr(ux), _dptr(uy), _dptr(phi)), b)


def lbm_batch_get_populations(b: int, member: int, f, g) -> None:
    _bcheck(_lib.lbm_batch_get_populations(b, member, _dptr(f), _dptr(g)), b)


def lbm_batch_set_state(b: int, member: int, state: int) -> None:
    """Restart a member from a device array of nx*ny x (phi, ux, uy) FP32 (asynchronous)."""
    _bcheck(_lib.lbm_batch_set_state(b, member, ctypes.c_void_p(state)), b)


def lbm_batch_get_state(b: int, member: int, state: int) -> None:
    """Write a member's (phi, ux, uy) into a device array of nx*ny x 3 FP32 (asynchronous)."""
    _bcheck(_lib.lbm_batch_get_state(b, member, ctypes.c_void_p(state)), b)


def lbm_batch_check(b: int, count: int):
    """(status, per-member non-finite flags)."""
    flags = (ctypes.c_int * count)()
    st = _lib.lbm_batch_check(b, flags)
    if st not in (LBM_OK, LBM_ERR_NONFINITE):
        _bcheck(st, b)
    return st, list(flags)


def lbm_batch_set_tile(b: int, bx: int, by: int, target_nodes: int) -> None:
    _bcheck(_lib.lbm_batch_set_tile(b, bx, by, target_nodes), b)


def lbm_batch_get_tile(b: int):
    """(bx, by, target_nodes, items, grid)."""
    v = [ctypes.c_int() for _ in range(5)]
    _bcheck(_lib.lbm_batch_get_tile(b, *(ctypes.byref(x) for x in v)), b)
    return tuple(x.value for x in v)


def lbm_batch_set_kernel(b: int, variant: int, target_nodes: int = 4096) -> None:
    _bcheck(_lib.lbm_batch_set_kernel(b, variant, target_nodes), b)


def lbm_batch_get_kernel(b: int) -> int:
    v = ctypes.c_int()
    _bcheck(_lib.lbm_batch_get_kernel(b, ctypes.byref(v)), b)
    return v.value


def lbm_batch_autotune(b: int, trial_steps: int = 5) -> float:
    ms = ctypes.c_double()
    _bcheck(_lib.lbm_batch_autotune(b, trial_steps, ctypes.byref(ms)), b)
    return ms.value


def lbm_batch_time(b: int) -> int:
    return _lib.lbm_batch_time(b)


def lbm_batch_last_error(b: int | None = None) -> str:
    return _lib.lbm_batch_last_error(b).decode(errors="replace")


def lbm_batch_free(b: int) -> None:
    _lib.lbm_batch_free(b)


def state_copy_bytes(p: lbm_params) -> int:
    """Bytes of one population copy inside a caller-supplied lbm_init buffer."""
    return (lbm_state_bytes(p) - 256) // 2


def lbm_time(h: int) -> int:
    return _lib.lbm_time(h)


def lbm_last_error(h: int | None = None) -> str:
    return _lib.lbm_last_error(h).decode(errors="replace")


def lbm_free(h: int) -> None:
    _lib.lbm_free(h)


# ------------------------------------------------------------------------------------------
# Convenience object: torch owns the device buffer and the stream.

class Lattice:
    """One lattice on the current CUDA device.  ``params`` are lbm_params field names."""

    def __init__(self, phi0, ux0=None, uy0=None, rho0=None, stream=None, **params):
        import torch
        phi0 = np.asarray(phi0, dtype=np.float64)
        self.ny, self.nx = phi0.shape
        self.params = lbm_default_params(nx=self.nx, ny=self.ny, **params)
        nbytes = lbm_state_bytes(self.params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.stream.device)
        self.h = lbm_init(self.params, phi0, ux0, uy0, rho0, self.buffer.data_ptr(), nbytes,
                          self.stream.cuda_stream)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def fields(self):
        """(rho, ux, uy, phi) as (ny, nx) float64 arrays; raises LbmError on a non-finite state."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        st = lbm_fields(self.h, *out)
        if st == LBM_ERR_NONFINITE:
            raise LbmError(st, lbm_last_error(self.h))
        return tuple(out)

    def conservation(self):
        return lbm_conservation(self.h)

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        lbm_get_populations(self.h, f, g)
        return f, g

    def set_populations(self, f, g):
        lbm_set_populations(self.h, np.ascontiguousarray(f, dtype=np.float64),
                            np.ascontiguousarray(g, dtype=np.float64))

    def autotune(self, trial_steps: int = 5) -> float:
        return lbm_autotune(self.h, trial_steps)

    def set_kernel(self, variant: int, bx: int = 0, by: int = 0, depth: int = 0, rows: int = 0):
        lbm_set_kernel(self.h, variant, bx, by, depth, rows)

    def set_wait_limit(self, probes: int):
        lbm_set_wait_limit(self.h, probes)

    @property
    def state_ptr(self) -> int:
        """Device address of the current population copy (inside self.buffer)."""
        return self.buffer.data_ptr() + (self.time % 2) * state_copy_bytes(self.params)

    @property
    def kernel(self):
        return lbm_get_kernel(self.h)

    @property
    def time(self) -> int:
        return lbm_time(self.h)

    def close(self):
        if getattr(self, "h", None):
            lbm_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent lattices advanced together on the current CUDA device.  ``members`` is a
    list of (phi0, params) with params as lbm_params field names; all share ``prec``."""

    def __init__(self, members, prec="fp32", stream=None):
        import torch
        self.params, phis = [], []
        for phi0, kw in members:
            phi0 = np.asarray(phi0, dtype=np.float64)
            ny, nx = phi0.shape
            self.params.append(lbm_default_params(nx=nx, ny=ny, prec=prec, **kw))
            phis.append(phi0)
        self.count = len(self.params)
        nbytes = lbm_batch_state_bytes(self.params)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.buffer = torch.empty(nbytes, dtype=torch.uint8, device=self.stream.device)
        self.b = lbm_batch_init(self.params, phis, self.buffer.data_ptr(), nbytes, self.stream.cuda_stream)

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n)

    def fields(self, member: int):
        p = self.params[member]
        out = [np.empty((p.ny, p.nx)) for _ in range(4)]
        lbm_batch_fields(self.b, member, *out)
        return tuple(out)

    def populations(self, member: int):
        p = self.params[member]
        f = np.empty((9, p.ny, p.nx))
        g = np.empty((9, p.ny, p.nx))
        lbm_batch_get_populations(self.b, member, f, g)
        return f, g

    def check(self):
        return lbm_batch_check(self.b, self.count)

    def set_state(self, member: int, state_ptr: int):
        lbm_batch_set_state(self.b, member, state_ptr)

    def get_state(self, member: int, state_ptr: int):
        lbm_batch_get_state(self.b, member, state_ptr)

    def set_tile(self, bx: int, by: int, target_nodes: int):
        lbm_batch_set_tile(self.b, bx, by, target_nodes)

    @property
    def tile(self):
        return lbm_batch_get_tile(self.b)

    def set_kernel(self, variant: int, target_nodes: int = 4096):
        lbm_batch_set_kernel(self.b, variant, target_nodes)

    @property
    def kernel(self) -> int:
        return lbm_batch_get_kernel(self.b)

    def autotune(self, trial_steps: int = 5) -> float:
        return lbm_batch_autotune(self.b, trial_steps)

    @property
    def time(self) -> int:
        return lbm_batch_time(self.b)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
