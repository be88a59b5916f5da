"""Reduced-precision storage on the paper's two-phase workloads: errors against the FP64 oracle at
full size, and the statistics the paper's experiments report.

Measured here (the tests print them):
* Sheared-droplet channel, 1024 x 512, walls at +-0.01, droplet R = 64, nu_l = 0.2, viscosity
  contrasts 1 to 1000, 1000 steps, max |phi - phi_oracle|: FP64 ~7e-14, FP32 2.7e-6 to 5.4e-6,
  FP16 9.8e-4 to 1.8e-3 (3.4e-4 to 6.5e-4 rounded stochastically), BF16 8.7e-3 to 1.4e-2 (3.2e-3
  to 5.2e-3 stochastically).  FP32 and FP16 meet the contract (1e-5, 2e-3); BF16 does not.
* Laplace droplet (64^2, R = 16, a = 0.04, gamma = 0.02, tau = 1), converged pressure jump
  against the oracle's: FP32 +0.009%, FP16 +0.18%, BF16 -0.03%.
* Taylor deformation in shear (the paper's set-up, 2H = 200, R = 30, Ca 0.05 to 0.25) against
  the FP64 run: FP32 within 0.4%; rounded stochastically FP16 within 0.27% and BF16 within 0.79%.
  Rounded to nearest the 16-bit forms do not resolve this flow (FP16 +2.7% to +9.0%, BF16 -27% to
  +48%): the wall speed is 2.2e-3, the shear changes a moving population's deviation by ~7e-6 per
  lattice row, and the stored deviations (~7e-4) have a rounding unit of 4.8e-7 in FP16 (15 units
  per row) and 3.8e-6 in BF16 (under 2): the viscous stress the flow runs on is quantised, and
  rounding to nearest quantises it the same way at neighbouring nodes.  Stochastic rounding
  (unbiased rounding of every stored value) removes that bias.
"""
import json
import math
import os

import numpy as np
import pytest

from _pair import abs_err, oracle_kwargs, rel_err
from paper_1803_11345_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PRECS = ("fp64", "fp32", "fp16s", "bf16s")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1803_11345_gb300 import build
    build.build()
    from paper_1803_11345_gb300 import lbm as mod
    return mod


def tau(nu):
    return 3.0 * nu + 0.5


ZETAS = (1, 10, 100, 1000)
CHANNEL_FORMS = ("fp64", "fp32", "fp16s", "fp16s+sr", "bf16s", "bf16s+sr")
# The contract on phi after 1000 steps: FP32 1e-5, 16-bit storage 2e-3 (absolute; phi's bulk
# values are +-1).  BF16 does not meet it (see test_sheared_channel_bf16_contract); its errors are
# held at the measured level only so that a regression shows.
CONTRACT = {"fp32": 1e-5, "fp16s": 2e-3, "fp16s+sr": 2e-3}
BF16_GUARD = {"bf16s": 2e-2, "bf16s+sr": 6e-3}


def channel_kw(zeta):
    """The sheared-droplet channel: 1024 x 512, walls moving at +-0.01, nu_l = 0.2 (the paper's
    shear set-up), nu_g = nu_l / zeta, gamma = a = 0.04, M = 0.1, Gamma = 1."""
    return dict(tau_l=tau(0.2), tau_g=tau(0.2 / zeta), gamma=0.04, a=0.04, M=0.1, Gamma=1.0, bc=1,
                u_top=0.01, u_bottom=-0.01)


@pytest.fixture(scope="module")
def channel(orc):
    """Oracle fields of the channel after 1000 steps, one run per contrast (about 30 s each on
    the host's cores), cached for the module."""
    cache = {}

    def run(zeta):
        if zeta not in cache:
            phi0 = W.droplet(1024, 512, 64, gamma=0.04, a=0.04)
            o = orc.Oracle(phi0, **oracle_kwargs(channel_kw(zeta)))
            o.step(1000)
            cache[zeta] = (phi0, o.fields())
            o.close()
        return cache[zeta]
    return run


def channel_form(lbm, phi0, zeta, form, steps=1000):
    prec = form.split("+")[0]
    kw = dict(channel_kw(zeta), prec=prec)
    if form.endswith("+sr"):
        kw.update(rounding=lbm.LBM_ROUND_STOCHASTIC, seed=7)
    lat = lbm.Lattice(phi0, **kw)
    s0 = lat.conservation()
    lat.step(steps)
    out = lat.fields()
    s1 = lat.conservation()
    lat.close()
    return out, s0, s1


@pytest.mark.parametrize("zeta", ZETAS)
def test_sheared_channel_contrast_sweep(lbm, channel, zeta):
    """The sheared-droplet channel at full size (1024 x 512, R = 64) for viscosity contrasts
    1, 10, 100 and 1000, 1000 steps, every storage form against the FP64 oracle.  FP64 matches to
    1e-12 (relative); FP32 and FP16 (rounded to nearest or stochastically) meet the contract on
    phi, 1e-5 and 2e-3.  Measured max |phi - phi_oracle|: FP32 2.7e-6 to 5.4e-6, FP16 9.8e-4 to
    1.8e-3, FP16 stochastic 3.4e-4 to 6.5e-4; BF16 8.7e-3 to 1.4e-2 and 3.2e-3 to 5.2e-3 stochastic
    (above the contract: see test_sheared_channel_bf16_contract).  16-bit storage keeps sum rho and
    sum phi exactly (bit for bit)."""
    phi0, (ro, uxo, uyo, po) = channel(zeta)
    errs = {}
    for form in CHANNEL_FORMS:
        (rg, uxg, uyg, pg), s0, s1 = channel_form(lbm, phi0, zeta, form)
        errs[form] = abs_err(pg, po)
        if form == "fp64":
            assert rel_err(pg, po) <= 1e-12 and rel_err(rg, ro) <= 1e-12
            assert abs_err(uxg, uxo) <= 1e-12 and abs_err(uyg, uyo) <= 1e-12
        if form.startswith(("fp16s", "bf16s")):
            assert s1[0] == s0[0] and s1[1] == s0[1], (form, s0, s1)
    print(f"zeta {zeta}: max |phi - phi_oracle| after 1000 steps:", errs)
    for form, bound in CONTRACT.items():
        assert errs[form] <= bound, (form, errs)
    for form, guard in BF16_GUARD.items():
        assert errs[form] <= guard, (form, errs)


@pytest.mark.xfail(strict=True, reason="BF16 storage misses the 2e-3 bound on phi: its 8-bit significand rounds "
                                       "the stored deviations (~3e-3) to ~1e-5 each step; measured 8.7e-3 to 1.4e-2 "
                                       "(nearest) and 3.2e-3 to 5.2e-3 (stochastic) over contrasts 1 to 1000")
def test_sheared_channel_bf16_contract(lbm, channel):
    """The 16-bit contract (2e-3 on phi after 1000 steps) applied to BF16 storage at contrast 100,
    rounded to nearest and stochastically.  Expected to fail, strictly: should BF16 ever meet it,
    this test fails and the statement of the miss must be revised."""
    phi0, (_, _, _, po) = channel(100)
    for form in ("bf16s", "bf16s+sr"):
        (_, _, _, pg), _, _ = channel_form(lbm, phi0, 100, form)
        assert abs_err(pg, po) <= 2e-3, (form, abs_err(pg, po))


def laplace_jump(rho, phi, a):
    """Bulk-pressure jump (Eq. 13) between the droplet centre and the far corner."""
    p0 = rho / 3 + a * (-0.5 * phi ** 2 + 0.75 * phi ** 4)
    c = phi.shape[0] // 2
    return p0[c - 1:c + 1, c - 1:c + 1].mean() - p0[0, 0]


def test_laplace_jump_across_precisions(lbm, orc):
    """64^2 periodic droplet, R = 16, tanh profile, a = 0.04, gamma = 0.02, M = 0.1, Gamma = 1,
    tau = 1 in both phases, 5000 steps (converged: the jump moves by < 0.2% from 5000 to 40000
    steps).  FP64 equals the oracle's jump; it is 0.846 sigma/R, for both, and the oracle gives
    the same ratio for R = 32 on 128^2 once converged (0.841 after 32000 steps): a deficit that
    does not depend on R, i.e. the discrete interface of width sqrt(gamma/a) = 0.71 carries ~16%
    less tension than the continuum sigma (the sweep at gamma = a lands within 3% of sigma).  Every
    storage form is within the 1% the statistics are held to: measured FP32 +0.009%, FP16 +0.18%,
    BF16 -0.03% (BF16 was 1.2% low while the order-one rest population g_0 took several FP32
    roundings per step and the 16-bit closures were inexact)."""
    a, ga = 0.04, 0.02
    phi0 = W.droplet(64, 64, 16, gamma=ga, a=a)
    kw = dict(tau_l=1.0, tau_g=1.0, gamma=ga, a=a, M=0.1, Gamma=1.0)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(5000)
    ro, _, _, po = o.fields()
    ref = laplace_jump(ro, po, a)
    jumps = {}
    for prec in PRECS:
        lat = lbm.Lattice(phi0, prec=prec, **kw)
        lat.step(5000)
        rho, _, _, phi = lat.fields()
        jumps[prec] = laplace_jump(rho, phi, a)
        lat.close()
    print("Laplace pressure jump (oracle %.6e):" % ref, jumps)
    sigma = math.sqrt(8 * ga * a / 9)
    assert abs(jumps["fp64"] / ref - 1) <= 1e-9
    assert abs(ref / (sigma / 16) - 0.846) < 0.01
    for prec in ("fp32", "fp16s", "bf16s"):
        assert abs(jumps[prec] / ref - 1) <= 0.01, (prec, jumps)


def deformation(phi):
    """D_f = (A - B)/(A + B) with A, B the axes of the ellipse with the same second moments as
    the region phi > 0 (the paper's statistic, as in the Taylor test of the paper suite)."""
    ny, nx = phi.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    w = (phi > 0).astype(float)
    area = w.sum()
    cx, cy = (w * x).sum() / area, (w * y).sum() / area
    ixx = (w * (x - cx) ** 2).sum() / area
    iyy = (w * (y - cy) ** 2).sum() / area
    ixy = (w * (x - cx) * (y - cy)).sum() / area
    lo, hi = np.linalg.eigvalsh(np.array([[ixx, ixy], [ixy, iyy]]))
    A, B = math.sqrt(hi), math.sqrt(lo)
    return (A - B) / (A + B)


def test_taylor_deformation_across_precisions(lbm):
    """The paper's droplet-in-shear set-up (2H = 200, R = 30, nu = 0.2, Re = 0.1, Ca 0.05 to
    0.25, 150000 steps, one batch per precision), the deformation D_f against the FP64 run, which
    itself follows 35/32 Ca within 5%.  The contract holds statistics within 1%: FP32 storage
    (measured within 0.4%) and both 16-bit forms rounded stochastically (FP16 0.27%, BF16 0.79%
    as single lattices; here batched) meet it.  Rounded to nearest the 16-bit forms do not resolve this slow shear (FP16 +2.7% to
    +9.0%, BF16 -27% to +48%; see the module notes): the test checks that they miss, so that the
    statement of the miss is revised should they ever meet it."""
    gold = json.load(open(GOLDEN))["taylor"]
    n, R, nu, Re = 200, 30, 0.2, 0.1
    H = n / 2
    vw = Re * H * nu / R ** 2
    cas = [0.05, 0.1, 0.15, 0.2, 0.25]
    members = []
    for ca in cas:
        sigma = vw * R * nu / (H * ca)
        ga = 3 * sigma / math.sqrt(8)
        members.append((W.droplet(n, n, R, gamma=ga, a=ga),
                        dict(tau_l=tau(nu), tau_g=tau(nu), gamma=ga, a=ga, M=0.1, bc=1, u_top=vw, u_bottom=-vw)))
    d = {}
    for prec in PRECS:
        bat = lbm.Batch(members, prec=prec)
        bat.step(150000)
        st, flags = bat.check()
        assert st == lbm.LBM_OK and not any(flags), (prec, st, flags)
        d[prec] = np.array([deformation(bat.fields(m)[3]) for m in range(len(cas))])
        bat.close()
    # 16-bit storage rounded stochastically, also one batch per precision (the batch derives each
    # step's key on the device)
    for prec in ("fp16s", "bf16s"):
        bat = lbm.Batch([(p0, dict(kw, rounding=1, seed=1 + k)) for k, (p0, kw) in enumerate(members)], prec=prec)
        bat.step(150000)
        st, flags = bat.check()
        assert st == lbm.LBM_OK and not any(flags), (prec, st, flags)
        d[prec + "+sr"] = np.array([deformation(bat.fields(m)[3]) for m in range(len(cas))])
        bat.close()
    print("Taylor deformation by Ca", cas, {k: v.tolist() for k, v in d.items()})
    slope = np.polyfit(np.array(cas), d["fp64"], 1)[0]
    assert abs(slope / gold["slope_theory"] - 1) < 0.05, (slope, d["fp64"])
    for prec in ("fp32", "fp16s+sr", "bf16s+sr"):
        assert np.all(np.abs(d[prec] / d["fp64"] - 1) <= 0.01), (prec, d[prec], d["fp64"])
    for prec in ("fp16s", "bf16s"):  # rounded to nearest: a known miss, checked as such
        assert np.max(np.abs(d[prec] / d["fp64"] - 1)) > 0.01, (prec, d[prec], d["fp64"])


# -------------------------------------------------------------------------------------------
# Stochastic rounding of the 16-bit storage (lbm_params.rounding = LBM_ROUND_STOCHASTIC).

W1 = {1: 1.0 / 9.0, 5: 1.0 / 36.0}  # weights of one axis and one diagonal direction


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("kernel", ["one-node", "paired"])
def test_stochastic_rounding_is_unbiased(lbm, prec, kernel):
    """A uniform lattice at rest (phi = 0, rho = 1 + delta, tau = 1 in both phases, so that one
    collision returns the equilibrium exactly): after one step every node stores the same FP32
    value d_i = w_i (rho - 1).  Rounded to nearest, all nodes hold one 16-bit value; rounded
    stochastically they hold the two neighbouring 16-bit values in the proportion that makes the
    mean equal d_i: within 1% of the 16-bit unit over 65536 nodes (the standard error of that mean
    is at most 0.2% of the unit).  The diagonal value (w = 1/36, ~2.8e-5) lies in FP16's subnormal
    range, the axis value (~1.1e-4) in its normal range."""
    n, delta = 256, 1.0e-3 * math.pi
    phi0 = np.zeros((n, n))
    rho0 = np.full((n, n), 1.0 + delta)
    for rounding in (0, 1):
        lat = lbm.Lattice(phi0, None, None, rho0, prec=prec, tau_l=1.0, tau_g=1.0, rounding=rounding, seed=11)
        if kernel == "paired":
            lat.set_kernel(lbm.LBM_KERNEL_PAIR, 128, 1)
            assert lat.kernel[0] == lbm.LBM_KERNEL_PAIR
        f0, _ = lat.populations()
        drho = float(f0[:, 0, 0].sum() - 1.0)  # the stored state's rho - 1 (identical at every node)
        lat.step(1)
        f1, _ = lat.populations()
        lat.close()
        for i, w in W1.items():
            d = f1[i] - w  # exact in FP64: the stored value is a 16-bit number
            levels = np.unique(d)
            v = w * drho
            if rounding == 0:
                assert len(levels) == 1, (i, levels)
                continue
            assert len(levels) == 2, (prec, kernel, i, levels)
            unit = levels[1] - levels[0]
            assert levels[0] < v < levels[1]
            assert abs(d.mean() - v) <= 0.01 * unit, (prec, kernel, i, d.mean(), v, unit)


def test_stochastic_rounding_is_reproducible(lbm):
    """The random bits are a counter-based stream of (seed, step, node): the same seed gives the
    same state bit for bit, another seed another state."""
    phi0 = W.spinodal(128, 64, seed=5)
    kw = dict(prec="fp16s", tau_l=0.8, tau_g=0.53, rounding=1)
    runs = []
    for seed in (3, 3, 4):
        lat = lbm.Lattice(phi0, seed=seed, **kw)
        lat.step(20)
        runs.append(lat.populations())
        lat.close()
    assert all(np.array_equal(a, b) for a, b in zip(runs[0], runs[1]))
    assert not np.array_equal(runs[0][0], runs[2][0])


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_stochastic_rounding_paired_follows_one_node(lbm, prec, bc):
    """Both 16-bit kernels draw the same random stream for a node, so one stochastically rounded
    step from the same non-uniform state stores the same values, except where the two kernels'
    FP32 results (their multiply-adds are fused at different places) straddle a rounding decision:
    at most 1% of the moving populations, each by one 16-bit unit.  A mix-up of the pair's lanes
    would move values by the node-to-node differences of the field instead.  Periodic, and between
    moving walls (the paired kernel's walled variant and its edge-row launch)."""
    phi0 = W.spinodal(256, 64, seed=8)
    walls = dict(bc=1, u_top=0.01, u_bottom=-0.01) if bc else {}
    out = []
    for variant, bx in ((lbm.LBM_KERNEL_GENERIC, 256), (lbm.LBM_KERNEL_PAIR, 128)):
        lat = lbm.Lattice(phi0, prec=prec, tau_l=0.8, tau_g=0.53, rounding=1, seed=5, **walls)
        lat.set_kernel(variant, bx, 1)
        lat.step(1)
        out.append(lat.populations())
        lat.close()
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    rel = 2.0 ** -10 if prec == "fp16s" else 2.0 ** -7  # a unit relative to the stored value
    for k in (0, 1):  # f as stored (deviations f_i - w_i), g as is
        va, vb = out[0][k][1:], out[1][k][1:]
        if k == 0:
            va, vb = va - w[1:], vb - w[1:]
        d = np.abs(va - vb)
        assert np.mean(d > 0) <= 0.01, (k, np.mean(d > 0))
        assert np.all(d <= rel * np.maximum(np.maximum(np.abs(va), np.abs(vb)), 2.0 ** -14) * 1.0001), (k, float(d.max()))


def test_staged_kernel_refused_with_stochastic_rounding(lbm):
    """The staged kernel stores from shared memory without the node index the rounding stream is
    keyed on, so a lattice with stochastic rounding refuses it and lbm_autotune leaves it out."""
    lat = lbm.Lattice(W.spinodal(128, 64, seed=2), prec="fp16s", rounding=1)
    with pytest.raises(lbm.LbmError) as ei:
        lat.set_kernel(lbm.LBM_KERNEL_STAGED, 64, 4)
    assert ei.value.status == lbm.LBM_ERR_PARAM
    lat.autotune(trial_steps=2)
    assert lat.kernel[0] != lbm.LBM_KERNEL_STAGED
    lat.close()


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_sheared_droplet_stochastic_rounding_against_oracle(lbm, orc, prec):
    """The parity suite's sheared droplet (128 x 64, walls at +-0.01, R = 16, nu_l = 0.2, contrast
    10) after 1000 steps against the FP64 oracle, with the 16-bit storage rounded stochastically.
    FP16: 3.5e-4 (1.5e-4 rounded to nearest), within the 2e-3 contract.  BF16: 3.7e-3 (1.25e-3 to
    nearest): the maximum difference is then set by BF16's own rounding noise (a unit of ~1.5e-5
    on every stored deviation each step), not by a bias; held at 5e-3 as a regression guard."""
    phi0 = W.droplet(128, 64, 16, gamma=0.04, a=0.04)
    kw = dict(tau_l=tau(0.2), tau_g=tau(0.02), bc=1, u_top=0.01, u_bottom=-0.01)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(1000)
    po = o.fields()[3]
    errs = {}
    for rounding in (0, 1):
        lat = lbm.Lattice(phi0, prec=prec, rounding=rounding, seed=9, **kw)
        lat.step(1000)
        errs[rounding] = abs_err(lat.fields()[3], po)
        lat.close()
    print(prec, "max |phi - phi_oracle| after 1000 steps, nearest / stochastic:", errs)
    assert errs[1] <= (2e-3 if prec == "fp16s" else 5e-3), errs
