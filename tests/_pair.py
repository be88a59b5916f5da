"""Helpers that run the CUDA path and the CPU oracle on the same seeded inputs."""
import numpy as np

# Parameter names of the C ABI that the oracle spells differently.
_TO_ORACLE = {"visc": "visc_interp", "bc": "walls", "force_x": "Fx", "force_y": "Fy"}
_GPU_ONLY = {"prec"}


def oracle_kwargs(kw):
    out = {}
    for k, v in kw.items():
        if k in _GPU_ONLY:
            continue
        out[_TO_ORACLE.get(k, k)] = v
    return out


def rel_err(a, b):
    """max |a - b| / max |b|."""
    scale = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / (scale if scale > 0 else 1.0)


def abs_err(a, b):
    return float(np.abs(a - b).max())
