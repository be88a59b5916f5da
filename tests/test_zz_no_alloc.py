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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16s", "bf16s"])
def test_noalloc_totals_match_conservation_twice(lbm, prec):
    """Bit-identical to lbm_conservation on the same state, on two calls in a row (the state
    advancing between them), and a repeated call on the same state gives the same bits."""
    nx, ny = 136, 77
    lat = lbm.Lattice(W.spinodal(nx, ny, seed=31), prec=prec, tau_l=0.8, tau_g=0.55)
    p = lbm.PRECISIONS[prec]
    for k in range(2):
        lat.step(7 + k)
        want = np.array(lat.conservation())
        got = np.array(lbm.lbm_totals_noalloc(lat.state_ptr, nx, ny, p, lat.stream.cuda_stream))
        assert np.array_equal(got, want), (k, got, want)
        again = np.array(lbm.lbm_totals_noalloc(lat.state_ptr, nx, ny, p, lat.stream.cuda_stream))
        assert np.array_equal(again, got)


def test_noalloc_call_allocates_nothing(lbm):
    """Free device memory is the same before and after a call on a lattice the entry point has
    not seen (after one earlier call has loaded the library's static array on this device)."""
    import torch
    first = lbm.Lattice(W.spinodal(64, 40, seed=2), prec="fp32")
    lbm.lbm_totals_noalloc(first.state_ptr, 64, 40, lbm.LBM_FP32, first.stream.cuda_stream)
    lat = lbm.Lattice(W.spinodal(520, 260, seed=3), prec="fp32")
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    got = lbm.lbm_totals_noalloc(lat.state_ptr, 520, 260, lbm.LBM_FP32, lat.stream.cuda_stream)
    torch.cuda.synchronize()
    after = torch.cuda.mem_get_info()[0]
    assert after == before, (before, after)
    assert np.array_equal(np.array(got), np.array(lat.conservation()))


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
