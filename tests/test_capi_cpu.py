"""The C ABI library loads without a GPU, exports every function include/lbm.h declares, and
rejects invalid parameters before touching the device."""
import ctypes
import math
import re

import pytest


@pytest.fixture(scope="module")
def lbm():
    from paper_1803_11345_gb300 import build
    build.build()
    from paper_1803_11345_gb300 import lbm as mod
    return mod


def test_exports_every_declared_symbol(lbm):
    names = lbm.declared_functions()
    assert {"lbm_init", "lbm_step", "lbm_fields", "lbm_free", "lbm_conservation",
            "lbm_get_populations", "lbm_set_populations", "lbm_last_error"} <= set(names)
    lib = ctypes.CDLL(lbm._build.LIB)
    for n in names:
        assert hasattr(lib, n), n


def test_surrogate_header_exported_and_wrapped(lbm):
    """Every function include/surrogate.h declares is exported and has a same-name wrapper."""
    import os
    import re
    from paper_1803_11345_gb300 import surrogate
    hdr = os.path.join(os.path.dirname(lbm.HEADER), "surrogate.h")
    text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(sur_\w+)\s*\(", text)))
    assert {"sur_conv3x3", "sur_conv3x3_up_add", "sur_conv3x3_wgrad_up", "sur_adam"} <= set(names)
    lib = ctypes.CDLL(lbm._build.LIB)
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(surrogate, n), f"binding lacks {n}"


def test_header_declares_what_the_binding_wraps(lbm):
    for n in lbm.declared_functions():
        assert hasattr(lbm, n), f"binding lacks {n}"


def test_defaults_follow_the_paper(lbm):
    p = lbm.lbm_default_params()
    assert (p.M, p.Gamma, p.gamma, p.a) == (0.1, 1.0, 0.04, 0.04)
    assert p.tau_l == pytest.approx(0.8) and p.omega3 == 1.0
    assert p.prec == lbm.LBM_FP32 and p.collision == lbm.LBM_COLLIDE_CM
    assert p.rounding == lbm.LBM_ROUND_NEAREST and p.seed == 0


@pytest.mark.parametrize("bad", [
    dict(nx=2), dict(ny=0), dict(tau_l=0.5), dict(tau_g=0.2), dict(M=0.0), dict(Gamma=-1.0),
    dict(gamma=-0.1), dict(omega3=2.0), dict(prec=7), dict(bc=3), dict(visc=5), dict(k8_form=2),
    dict(collision=9), dict(u_top=float("nan")), dict(nx=70000, ny=70000), dict(force_mode=2),
    dict(force_x=float("inf")), dict(wet_bottom=0.1), dict(bc=1, wet_top=float("nan")), dict(rounding=2),
    dict(rounding=1), dict(rounding=1, prec=0)])
def test_invalid_parameters_rejected(lbm, bad):
    kw = dict(nx=16, ny=16)
    kw.update(bad)
    p = lbm.lbm_default_params(**kw)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_state_bytes(p)
    assert ei.value.status == lbm.LBM_ERR_PARAM
    assert lbm.lbm_last_error(None)


def test_state_bytes_scale_with_precision(lbm):
    sizes = {}
    for name, prec in lbm.PRECISIONS.items():
        sizes[name] = lbm.lbm_state_bytes(lbm.lbm_default_params(nx=256, ny=256, prec=prec))
    N = 256 * 256
    assert sizes["fp64"] >= 2 * 18 * 8 * N
    assert sizes["fp32"] >= 2 * 18 * 4 * N
    assert sizes["fp16s"] >= 2 * (16 * 2 + 2 * 4) * N
    assert sizes["fp16s"] < sizes["fp32"] < sizes["fp64"]


def test_init_rejects_nonfinite_and_missing_input(lbm):
    import numpy as np
    p = lbm.lbm_default_params(nx=8, ny=8)
    phi = np.zeros(64)
    phi[5] = np.nan
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_init(p, phi)
    assert ei.value.status == lbm.LBM_ERR_PARAM and "non-finite" in str(ei.value)


def test_wall_gradient_matches_the_oracle(lbm, orc):
    """Eq. 18 on the host side of the library equals the oracle's, and is odd about 90 degrees."""
    for ratio in (1.0, 4.0):
        for deg in (10, 45, 60, 90, 120, 170):
            th = math.radians(deg)
            want = orc.wall_gradient(th, 0.04, 0.04 * ratio)
            assert math.isclose(lbm.lbm_wall_gradient(th, 0.04, 0.04 * ratio), want, rel_tol=1e-14, abs_tol=1e-16)
            assert math.isclose(lbm.lbm_wall_gradient(math.pi - th, 0.04, 0.04 * ratio), -want, rel_tol=1e-14,
                                abs_tol=1e-16)
    assert math.isnan(lbm.lbm_wall_gradient(1.0, 0.04, 0.0))


def test_stochastic_rounding_only_for_16bit_storage(lbm):
    """Stochastic rounding is accepted for FP16S / BF16S storage, for single lattices and batches
    (whose step keys come from a device-side step counter), and refused for FP32 / FP64 (no 16-bit
    rounding to randomise)."""
    for prec in (lbm.LBM_FP16S, lbm.LBM_BF16S):
        p = lbm.lbm_default_params(nx=16, ny=16, prec=prec, rounding=1, seed=7)
        assert lbm.lbm_state_bytes(p) > 0
        assert lbm.lbm_batch_state_bytes([p, p]) > 0
    for prec in (lbm.LBM_FP32, lbm.LBM_FP64):
        p = lbm.lbm_default_params(nx=16, ny=16, prec=prec, rounding=1)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_batch_state_bytes([p, p])
        assert ei.value.status == lbm.LBM_ERR_PARAM


def test_tcgen05_conv_planner_host_side(lbm):
    """The tcgen05 convolution's tiling rules, answered on the host without a GPU: rows of 128
    pixels or a multiple (row mode), or a power-of-two width from 2 to 64 dividing 128 (copy mode:
    whole rows per tile, weights by tensor-map boxes, so every stage lands on 128-byte
    boundaries); heights a multiple of the tile's rows; channels multiples of 16; more than 128
    output channels only in whole 128-channel tiles; even sizes when upsampled."""
    from paper_1803_11345_gb300 import surrogate as S
    ok = [(16, 256, 256, 16, 32, 0), (16, 128, 128, 64, 64, 0), (16, 64, 64, 128, 128, 0),
          (16, 32, 32, 256, 256, 0), (2, 8, 256, 48, 96, 0), (1, 16, 32, 16, 16, 0), (2, 64, 2, 16, 16, 0),
          (16, 256, 256, 64, 32, 1), (16, 64, 64, 256, 128, 1)]
    bad = [(1, 16, 96, 32, 32, 0),    # width neither a multiple of 128 nor a power of two below it
           (1, 6, 32, 32, 32, 0),     # height not a multiple of the 4 rows a 32-wide tile holds
           (1, 16, 32, 24, 32, 0),    # input channels not a multiple of 16
           (1, 16, 32, 32, 160, 0),   # 160 output channels: not a whole number of 128-channel tiles
           (1, 256, 1, 16, 16, 0),    # width 1: a stage would not end on a 128-byte boundary
           (1, 15, 256, 32, 32, 1)]   # odd height through the 2x upsampling
    for shape in ok:
        assert S.sur_conv3x3_tc_supported(*shape), shape
    for shape in bad:
        assert not S.sur_conv3x3_tc_supported(*shape), shape
