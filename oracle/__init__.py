"""FP64 CPU oracle for the hybrid central-moment / BGK lattice Boltzmann scheme of
De Rosis, Saito, Kaneko & Abe (arXiv:1803.11345) — ctypes wrapper around ``lbm_oracle.cpp``.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import this package.  It shares no code with the CUDA
path (``paper_1803_11345_gb300``) and never imports it.

The C++ file is compiled with ``-ffp-contract=off`` so that x86 and Arm hosts round the
same way (no fused multiply-adds are introduced by the compiler).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

CS2 = 1.0 / 3.0


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau_l", ctypes.c_double), ("tau_g", ctypes.c_double),
        ("M", ctypes.c_double), ("Gamma", ctypes.c_double),
        ("gamma", ctypes.c_double), ("a", ctypes.c_double),
        ("omega3", ctypes.c_double),
        ("omega6", ctypes.c_double), ("omega7", ctypes.c_double), ("omega8", ctypes.c_double),
        ("visc_interp", ctypes.c_int), ("k8_form", ctypes.c_int),
        ("collision", ctypes.c_int), ("walls", ctypes.c_int),
        ("u_top", ctypes.c_double), ("u_bottom", ctypes.c_double),
        ("wet_bottom", ctypes.c_double), ("wet_top", ctypes.c_double),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double), ("force_mode", ctypes.c_int),
    ]


_DEFAULTS = dict(tau_l=1.0, tau_g=1.0, M=0.1, Gamma=1.0, gamma=0.04, a=0.04, omega3=1.0,
                 omega6=1.0, omega7=1.0, omega8=1.0, visc_interp=0, k8_form=0, collision=0,
                 walls=0, u_top=0.0, u_bottom=0.0, wet_bottom=0.0, wet_top=0.0, Fx=0.0, Fy=0.0,
                 force_mode=0)


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.cpp`` into ``oracle/_build/liblbm_oracle.so``."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(_Params)
    lib.orc_feq.argtypes = [d, d, d, d, d, d, d, dp]
    lib.orc_geq.argtypes = [d, d, d, d, d, dp]
    lib.orc_basis.argtypes = [d, d, dp]
    lib.orc_keq_printed.argtypes = [d, d, d, d, d, d, d, d, dp]
    lib.orc_solve.argtypes = [i, dp, dp, dp]
    lib.orc_solve.restype = i
    lib.orc_omega_rho.argtypes = [pp, d]
    lib.orc_omega_rho.restype = d
    lib.orc_omega_phi.argtypes = [pp]
    lib.orc_omega_phi.restype = d
    lib.orc_collide_f.argtypes = [pp, dp, d, d, d, d, dp]
    lib.orc_collide_g.argtypes = [pp, dp, d, d, d, d, d, dp]
    lib.orc_stencils.argtypes = [i, i, i, d, d, dp, dp, dp, dp]
    lib.orc_wall_gradient.argtypes = [d, d, d]
    lib.orc_wall_gradient.restype = d
    lib.orc_force.argtypes = [pp, d, dp]
    lib.orc_guo_source.argtypes = [d, d, d, d, dp]
    lib.orc_velocity.argtypes = [pp, dp, d, dp]
    lib.orc_create.argtypes = [pp, dp, dp, dp, dp]
    lib.orc_create.restype = p
    lib.orc_step.argtypes = [p, i]
    lib.orc_fields.argtypes = [p, dp, dp, dp, dp]
    lib.orc_get_populations.argtypes = [p, dp, dp]
    lib.orc_set_populations.argtypes = [p, dp, dp]
    lib.orc_sums.argtypes = [p, dp]
    lib.orc_free.argtypes = [p]
    lib.orc_node_update.argtypes = [pp, dp, dp, i, i, dp, dp]
    lib.orc_set_threads.argtypes = [i]
    lib.orc_set_threads.restype = i
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def make_params(nx: int, ny: int, **kw) -> _Params:
    """Oracle parameter block; unknown keys raise."""
    vals = dict(_DEFAULTS)
    for k, v in kw.items():
        if k not in vals:
            raise KeyError(f"unknown oracle parameter {k!r}")
        vals[k] = v
    return _Params(nx=nx, ny=ny, **vals)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave unchanged); returns the count in use."""
    return _load().orc_set_threads(int(n))


# --------------------------------------------------------------------------------------
# Node-level functions (used by the pins).

def feq(rho, ux, uy, pt, gx, gy, gamma):
    out = np.zeros(9)
    _load().orc_feq(rho, ux, uy, pt, gx, gy, gamma, _ptr(out))
    return out


def geq(phi, ux, uy, mu, Gamma):
    out = np.zeros(9)
    _load().orc_geq(phi, ux, uy, mu, Gamma, _ptr(out))
    return out


def basis(ux, uy):
    out = np.zeros(81)
    _load().orc_basis(ux, uy, _ptr(out))
    return out.reshape(9, 9)


def keq_printed(rho, ux, uy, pt, gx, gy, lap, gamma):
    out = np.zeros(9)
    _load().orc_keq_printed(rho, ux, uy, pt, gx, gy, lap, gamma, _ptr(out))
    return out


def solve(A, b):
    A = _f64(A)
    b = _f64(b)
    x = np.zeros(len(b))
    rc = _load().orc_solve(len(b), _ptr(A), _ptr(b), _ptr(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def omega_rho(params: _Params, phi: float) -> float:
    return _load().orc_omega_rho(ctypes.byref(params), phi)


def omega_phi(params: _Params) -> float:
    return _load().orc_omega_phi(ctypes.byref(params))


def collide_f(params: _Params, f, phi, gx, gy, lap):
    f = _f64(f)
    out = np.zeros(9)
    _load().orc_collide_f(ctypes.byref(params), _ptr(f), phi, gx, gy, lap, _ptr(out))
    return out


def collide_g(params: _Params, g, ux, uy, gx, gy, lap):
    g = _f64(g)
    out = np.zeros(9)
    _load().orc_collide_g(ctypes.byref(params), _ptr(g), ux, uy, gx, gy, lap, _ptr(out))
    return out


def stencils(phi, walls: bool = False, wet_bottom: float = 0.0, wet_top: float = 0.0):
    """(d/dx, d/dy, Laplacian) of a (ny, nx) array with the isotropic stencils; with walls the
    ghost rows are the adjacent rows plus the wall gradients wet_bottom / wet_top."""
    phi = _f64(phi)
    ny, nx = phi.shape
    gx, gy, lap = (np.zeros_like(phi) for _ in range(3))
    _load().orc_stencils(nx, ny, int(walls), float(wet_bottom), float(wet_top), _ptr(phi), _ptr(gx), _ptr(gy),
                         _ptr(lap))
    return gx, gy, lap


def wall_gradient(theta, a, gamma):
    """Wall gradient of phi along the outward normal for contact angle theta (radians), Eq. 18."""
    return _load().orc_wall_gradient(float(theta), float(a), float(gamma))


def force(params: _Params, phi):
    out = np.zeros(2)
    _load().orc_force(ctypes.byref(params), float(phi), _ptr(out))
    return out


def guo_source(ux, uy, Fx, Fy):
    out = np.zeros(9)
    _load().orc_guo_source(ux, uy, Fx, Fy, _ptr(out))
    return out


def velocity(params: _Params, f, phi):
    """(sum f c + F/2) / rho of one node's populations f."""
    f = _f64(f)
    out = np.zeros(2)
    _load().orc_velocity(ctypes.byref(params), _ptr(f), float(phi), _ptr(out))
    return out


def node_update(params: _Params, f, g, x: int, y: int):
    """Post-collision (f, g) of node (x, y) one step after the full-lattice post-collision
    state f, g ((9, ny, nx) arrays), from that node's neighbourhood only."""
    f = _f64(f)
    g = _f64(g)
    fo, go = np.zeros(9), np.zeros(9)
    _load().orc_node_update(ctypes.byref(params), _ptr(f), _ptr(g), int(x), int(y), _ptr(fo), _ptr(go))
    return fo, go


# --------------------------------------------------------------------------------------
# Whole-lattice simulation.

class Oracle:
    """FP64 lattice of post-collision populations, advanced step by step on the host."""

    def __init__(self, phi0, ux0=None, uy0=None, rho0=None, **params):
        phi0 = _f64(phi0)
        self.ny, self.nx = phi0.shape
        self.params = make_params(self.nx, self.ny, **params)
        self._keep = [phi0, _f64(ux0), _f64(uy0), _f64(rho0)]
        self._h = _load().orc_create(ctypes.byref(self.params), *(_ptr(a) for a in self._keep))

    def step(self, n: int = 1):
        _load().orc_step(self._h, int(n))

    def fields(self):
        """Return (rho, ux, uy, phi) as (ny, nx) FP64 arrays."""
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        _load().orc_fields(self._h, *(_ptr(a) for a in out))
        return tuple(out)

    def populations(self):
        """Return (f, g) as (9, ny, nx) FP64 arrays."""
        f = np.zeros((9, self.ny, self.nx))
        g = np.zeros((9, self.ny, self.nx))
        _load().orc_get_populations(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_populations(self, f, g):
        f = _f64(f)
        g = _f64(g)
        _load().orc_set_populations(self._h, _ptr(f), _ptr(g))

    def sums(self):
        """Compensated sums: (sum phi, sum rho, sum rho*ux, sum rho*uy)."""
        out = np.zeros(4)
        _load().orc_sums(self._h, _ptr(out))
        return tuple(out)

    def close(self):
        if self._h:
            _load().orc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tau_from_nu(nu: float) -> float:
    """tau = nu / c_s^2 + 1/2 (paragraph after Eq. 14)."""
    return nu / CS2 + 0.5
