"""Batched stepping (many independent lattices in one persistent launch per step, CUDA-graph
replays, autotuned tiles) against single-lattice runs and the oracle."""
import numpy as np
import pytest

from _pair import abs_err, oracle_kwargs, rel_err
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


def _members():
    """Uneven sizes, both boundaries, different viscosity ratios and surface tensions."""
    return [
        (W.droplet(64, 64, 16, gamma=0.02, a=0.04), dict(tau_l=1.0, tau_g=1.0, gamma=0.02, a=0.04)),
        (W.spinodal(128, 64, seed=5), dict(tau_l=0.8, tau_g=0.53, visc=1)),
        (W.droplet(96, 40, 12, gamma=0.04, a=0.04), dict(tau_l=0.9, tau_g=0.6, bc=1, u_top=0.01, u_bottom=-0.01)),
        (W.droplet(67, 45, 14, gamma=0.04, a=0.04), dict(tau_l=0.7, tau_g=0.51, omega3=1.3)),
        (W.spinodal(3, 3, seed=1), dict()),
        (W.spinodal(512, 256, seed=8), dict(tau_l=0.8, tau_g=0.503)),
    ]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-5)])
def test_batch_members_equal_single_lattices(lbm, prec, tol):
    """The batch runs the single-lattice tile code over a work list, so every member follows a
    single lattice stepped with the same tile shape, through graph replays and odd step counts.
    The batch kernel is a separate compilation of that code and the compiler may contract a
    multiply-add into an FMA in one kernel and not the other, so the two agree to rounding:
    FP64 within 1e-13 of the population scale after 61 steps (measured: 2e-15), FP32 within 1e-5
    (1-ulp differences at a few nodes, amplified in the near-unstable tau_g = 0.51 member to
    3e-7).  Bit-identity across tile shapes of one compiled kernel is checked below."""
    mem = _members()
    bat = lbm.Batch(mem, prec=prec)
    bx, by = bat.tile[:2]
    singles = [lbm.Lattice(phi0, prec=prec, **kw) for phi0, kw in mem]
    for s in singles:
        s.set_kernel(lbm.LBM_KERNEL_GENERIC, bx, by, 0, 0)
    for n in (5, 37, 16, 3):
        bat.step(n)
        for s in singles:
            s.step(n)
    assert bat.time == 61
    for m, s in enumerate(singles):
        fb, gb = bat.populations(m)
        fs, gs = s.populations()
        assert rel_err(fb, fs) <= tol and abs_err(gb, gs) <= tol * max(1.0, float(np.abs(gs).max())), m


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_batch_stochastic_rounding_follows_single_lattices(lbm, prec):
    """Batches round stochastically too: the key of a step is derived on the device from the
    batch's step counter (two parity slots, so graph replays advance it) by the function a single
    lattice uses on the host, so a member draws the single lattice's random stream.  One step from
    the same state stores the same values as a single lattice of the same seed and tile, except
    where the two separately compiled kernels' FP32 results straddle a rounding decision (at most
    1% of the moving populations, by one 16-bit unit); over 61 steps, through graph replays, phi
    stays within 1e-3 of the single lattice's, and the rounding does change with the step (the
    batch differs from the same batch rounded to nearest)."""
    mem = [(phi0, dict(kw, rounding=lbm.LBM_ROUND_STOCHASTIC, seed=7 + k))
           for k, (phi0, kw) in enumerate(_members()) if phi0.shape[0] >= 40]
    bat = lbm.Batch(mem, prec=prec)
    near = lbm.Batch([(p0, dict(kw, rounding=lbm.LBM_ROUND_NEAREST)) for p0, kw in mem], prec=prec)
    bx, by = bat.tile[:2]
    singles = [lbm.Lattice(phi0, prec=prec, **kw) for phi0, kw in mem]
    for s in singles:
        s.set_kernel(lbm.LBM_KERNEL_GENERIC, bx, by, 0, 0)
    bat.step(1)
    for s in singles:
        s.step(1)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    rel = 2.0 ** -10 if prec == "fp16s" else 2.0 ** -7
    for m, s in enumerate(singles):
        fb, gb = bat.populations(m)
        fs, gs = s.populations()
        for k, (a, b) in enumerate(((fb[1:] - w[1:], fs[1:] - w[1:]), (gb[1:], gs[1:]))):
            d = np.abs(a - b)
            assert np.mean(d > 0) <= 0.01, (m, k, np.mean(d > 0))
            assert np.all(d <= rel * np.maximum(np.maximum(np.abs(a), np.abs(b)), 2.0 ** -14) * 1.0001), (m, k)
    for n in (36, 16, 8):
        bat.step(n)
        near.step(n + (1 if n == 36 else 0))
        for s in singles:
            s.step(n)
    assert bat.time == 61 and near.time == 61
    differs = False
    for m, s in enumerate(singles):
        pb = bat.fields(m)[3]
        assert abs_err(pb, s.fields()[3]) <= 1e-3, m
        differs |= not np.array_equal(pb, near.fields(m)[3])
    assert differs
    assert bat.check()[0] == lbm.LBM_OK


def _pair_members():
    """Periodic members with even nx: a full 256-column strip, ragged strips (326 = 256 + 70,
    70 < 256), a narrow lattice (8 columns), different viscosity ratios and surface tensions."""
    return [
        (W.spinodal(326, 90, seed=4), dict(tau_l=0.8, tau_g=0.53, visc=1)),
        (W.droplet(256, 64, 16, gamma=0.02, a=0.04), dict(tau_l=1.0, tau_g=0.6, gamma=0.02, a=0.04)),
        (W.spinodal(70, 33, seed=9), dict(tau_l=0.7, tau_g=0.55, omega3=1.3)),
        (W.spinodal(8, 16, seed=2), dict()),
        (W.droplet(512, 128, 30, gamma=0.04, a=0.04), dict(tau_l=0.9, tau_g=0.503)),
    ]


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
def test_paired_batch_members_equal_single_lattices(lbm, prec, rounding):
    """The paired 16-bit tile in the batch work list: each work item is stepped by the paired
    kernel's tile code with its member's geometry and physics, and stochastic-rounding keys come
    from the batch's device step counter by the function single lattices use, so every member's
    state equals, bit for bit, a single lattice stepped with LBM_KERNEL_PAIR, through graph
    replays and odd step counts, whatever the item size."""
    mem = _pair_members()
    if rounding == "stochastic":
        mem = [(p0, dict(kw, rounding=lbm.LBM_ROUND_STOCHASTIC, seed=5 + k)) for k, (p0, kw) in enumerate(mem)]
    singles = [lbm.Lattice(phi0, prec=prec, **kw) for phi0, kw in mem]
    for s in singles:
        s.set_kernel(lbm.LBM_KERNEL_PAIR, 128, 1)
    for target in (2048, 16384):
        bat = lbm.Batch(mem, prec=prec)
        bat.set_kernel(lbm.LBM_KERNEL_PAIR, target)
        assert bat.kernel == lbm.LBM_KERNEL_PAIR and bat.tile[:2] == (128, 1)
        for n in (5, 37, 16, 3):
            bat.step(n)
        assert bat.time == 61 and bat.check()[0] == lbm.LBM_OK
        if target == 2048:
            for n in (5, 37, 16, 3):
                for s in singles:
                    s.step(n)
        for m, s in enumerate(singles):
            fb, gb = bat.populations(m)
            fs, gs = s.populations()
            assert np.array_equal(fb, fs) and np.array_equal(gb, gs), (target, m, abs_err(fb, fs))
        bat.close()


def test_paired_batch_refused_where_it_cannot_serve(lbm):
    """LBM_KERNEL_PAIR needs every member periodic with even nx and 16-bit storage; otherwise
    lbm_batch_set_kernel refuses and the batch keeps its tile, and a new batch never starts with
    it, even when the autotuner chose it for a batch of the same sizes without walls."""
    for mem, prec in (([(W.spinodal(64, 32, seed=1), dict()), (W.spinodal(65, 32, seed=2), dict())], "fp16s"),
                      ([(W.spinodal(64, 32, seed=1), dict()), (W.spinodal(64, 32, seed=2), dict(bc=1))], "fp16s"),
                      ([(W.spinodal(64, 32, seed=1), dict())], "fp32")):
        bat = lbm.Batch(mem, prec=prec)
        before = bat.tile
        with pytest.raises(lbm.LbmError):
            bat.set_kernel(lbm.LBM_KERNEL_PAIR)
        assert bat.kernel == lbm.LBM_KERNEL_GENERIC and bat.tile == before
        bat.close()
    # The autotuner's cached winner for a periodic batch is not handed to a walled batch of the
    # same sizes: the paired tile would step its walls as periodic rows.
    sizes = [(96, 48), (64, 32)]
    per = lbm.Batch([(W.spinodal(nx, ny, seed=nx), dict()) for nx, ny in sizes], prec="fp16s")
    per.set_kernel(lbm.LBM_KERNEL_PAIR)
    per.autotune(trial_steps=2)
    per.close()
    walled = lbm.Batch([(W.spinodal(nx, ny, seed=nx), dict(bc=1)) for nx, ny in sizes], prec="fp16s")
    assert walled.kernel == lbm.LBM_KERNEL_GENERIC
    walled.close()


def test_batch_fp64_member_matches_oracle(lbm, orc):
    mem = _members()[:4]
    bat = lbm.Batch(mem, prec="fp64")
    bat.step(40)
    for m, (phi0, kw) in enumerate(mem):
        o = orc.Oracle(phi0, **oracle_kwargs(kw))
        o.step(40)
        _, _, _, pg = bat.fields(m)
        _, _, _, po = o.fields()
        assert rel_err(pg, po) <= 1e-12, m


def test_batch_tiles_and_autotune_keep_state(lbm):
    mem = _members()
    bat = lbm.Batch(mem, prec="fp32")
    ref = lbm.Batch(mem, prec="fp32")
    bat.step(7)
    ref.step(7)
    before = [bat.populations(m) for m in range(len(mem))]
    ms = bat.autotune(trial_steps=2)
    assert ms > 0 and bat.time == 7
    for m in range(len(mem)):
        f, g = bat.populations(m)
        assert np.array_equal(f, before[m][0]) and np.array_equal(g, before[m][1])
    # Other tile shapes are other compiled kernels (multiply-add contraction may differ by an
    # ulp), so the states follow each other to FP32 rounding.
    for bx, by, tgt in [(32, 4, 2048), (128, 1, 16384), (256, 1, 4096)]:
        bat.set_tile(bx, by, tgt)
        assert bat.tile[:3] == (bx, by, tgt)
        bat.step(16)
        ref.step(16)
    for m in range(len(mem)):
        f, g = bat.populations(m)
        fr, gr = ref.populations(m)
        assert rel_err(f, fr) <= 1e-5 and abs_err(g, gr) <= 1e-5, m
    with pytest.raises(lbm.LbmError):
        bat.set_tile(48, 4, 4096)


def test_batch_flags_only_the_unstable_member(lbm):
    """A member with omega_phi = 1.74 (Gamma = 2, M = 0.05) goes non-finite; only its flag rises."""
    mem = _members()[:3] + [(W.droplet(48, 40, 12, gamma=0.04, a=0.04), dict(tau_l=0.9, tau_g=0.6, Gamma=2.0, M=0.05))]
    bat = lbm.Batch(mem, prec="fp32")
    bat.step(300)
    st, flags = bat.check()
    assert st == lbm.LBM_ERR_NONFINITE and flags == [0, 0, 0, 1]
    st, flags = bat.check()
    assert st == lbm.LBM_OK


def test_single_lattice_autotune_keeps_state(lbm):
    lat = lbm.Lattice(W.spinodal(256, 128, seed=3), prec="fp32", tau_l=0.8, tau_g=0.53)
    first = lat.kernel
    lat.step(3)
    f0, g0 = lat.populations()
    ms = lat.autotune(trial_steps=2)
    assert ms > 0 and lat.time == 3
    f1, g1 = lat.populations()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    # The same kernels in the same order (the first default for 3 steps, then the autotuned one):
    # bit for bit.  A lattice of the same shape created now starts with the cached winner, so
    # the first kernel is set explicitly.
    ref = lbm.Lattice(W.spinodal(256, 128, seed=3), prec="fp32", tau_l=0.8, tau_g=0.53)
    ref.set_kernel(*first)
    ref.step(3)
    ref.set_kernel(*lat.kernel)
    lat.step(10)
    ref.step(10)
    fa, ga = lat.populations()
    fb, gb = ref.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
