"""The allocation-free totals entry point (lbm_totals_noalloc), through the C ABI.

It serves callers that cannot allocate device memory and hold a population state in memory of
their own: its reduction scratch is a static array inside the library.  Its totals must equal
those of lbm_conservation (same kernels, same order) on the same state, call after call.
This file is collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_1803_11345_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_11345_gb300 import build
    build.build()
    from paper_1803_11345_gb300 import lbm as mod
    return mod


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s"])
def test_noalloc_totals_match_conservation_twice(lbm, prec):
    nx, ny = 136, 77
    lat = lbm.Lattice(W.spinodal(nx, ny, seed=31), prec=prec, tau_l=0.8, tau_g=0.55)
    p = lbm.PRECISIONS[prec]
    for k in range(2):  # two calls in a row, the state advancing between them
        lat.step(7 + k)
        want = np.array(lat.conservation())
        got = np.array(lbm.lbm_totals_noalloc(lat.state_ptr, nx, ny, p, lat.stream.cuda_stream))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-9), (k, got, want)
        again = np.array(lbm.lbm_totals_noalloc(lat.state_ptr, nx, ny, p, lat.stream.cuda_stream))
        assert np.array_equal(again, got)


def test_noalloc_rejects_bad_arguments(lbm):
    lat = lbm.Lattice(W.spinodal(64, 32, seed=1), prec="fp32")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_totals_noalloc(lat.state_ptr, 2, 32, lbm.LBM_FP32)
    assert ei.value.status == lbm.LBM_ERR_PARAM and "nx and ny" in str(ei.value)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_totals_noalloc(lat.state_ptr, 64, 32, 9)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_totals_noalloc(lat.state_ptr, 70000, 70000, lbm.LBM_FP32)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_totals_noalloc(0, 64, 32, lbm.LBM_FP32)
