"""The paper's experiments, run on the GPU path, against what the paper prints or states."""
import json
import math
import os

import numpy as np
import pytest

from paper_1803_11345_gb300 import workloads as W

pytestmark = pytest.mark.gpu
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


def test_laplace_law_sweep(lbm):
    """Laplace paragraph after Eq. 17: 200^2 periodic bubbles, gamma = a = 0.04, nu_l = 0.1,
    nu_g = nu_l / zeta, zeta in {2, 10, 100, 1000}, M = 0.1, Gamma = 1.  The bulk-pressure jump
    falls on a line in 1/R whose slope is sigma = sqrt(8 gamma a / 9) = 0.03771 (paper's fit
    0.03717, 1.43% off) and does not depend on zeta.  All 24 runs advance as one batch."""
    gold = json.load(open(GOLDEN))["laplace"]
    n, ga = 200, gold["gamma"]
    radii, zetas = [10, 15, 20, 25, 30, 40], [2, 10, 100, 1000]
    members = [(W.droplet(n, n, R, gamma=ga, a=ga),
                dict(tau_l=tau(0.1), tau_g=tau(0.1 / z), gamma=ga, a=ga, M=0.1, Gamma=1.0))
               for z in zetas for R in radii]
    bat = lbm.Batch(members, prec="fp32")
    bat.step(30000)
    st, flags = bat.check()
    assert st == lbm.LBM_OK and not any(flags)
    slopes = []
    for k, z in enumerate(zetas):
        dps = []
        for j, R in enumerate(radii):
            rho, _, _, phi = bat.fields(k * len(radii) + j)
            p0 = rho / 3 + ga * (-0.5 * phi ** 2 + 0.75 * phi ** 4)  # Eq. 13
            c = n // 2
            dps.append(p0[c - 1:c + 1, c - 1:c + 1].mean() - p0[0, 0])
        inv = 1.0 / np.array(radii, dtype=float)
        slope, _ = np.polyfit(inv, np.array(dps), 1)
        slopes.append(slope)
    sigma = math.sqrt(8 * ga * ga / 9)
    assert round(sigma, 5) == gold["slope_theory"]
    for s in slopes:
        assert abs(s / sigma - 1) < 0.03, slopes
    assert (max(slopes) - min(slopes)) / sigma < 0.03, slopes


def _bubble_run(lbm, steps, **kw):
    n, ga = 200, 0.04
    lat = lbm.Lattice(W.droplet(n, n, 40, gamma=ga, a=ga), prec="fp64", gamma=ga, a=ga, M=0.1, **kw)
    lat.step(steps)
    rho, ux, uy, phi = (np.empty(n * n) for _ in range(4))
    st = lbm.lbm_fields(lat.h, rho, ux, uy, phi)
    return st, float(np.max(np.hypot(ux, uy))) if st == lbm.LBM_OK else float("nan")


def test_double_bgk_unstable_central_moments_stable(lbm):
    """Stability paragraph (after Eq. 14) and the figure after it: on the 200^2 bubble with
    nu_l = 0.1, double-BGK (Eq. 6) blows up at zeta = 3, while the central-moment scheme runs
    smoothly at zeta = 100 (and at zeta = 3)."""
    st, _ = _bubble_run(lbm, 2000, collision=1, tau_l=tau(0.1), tau_g=tau(0.1 / 3))
    assert st == lbm.LBM_ERR_NONFINITE
    st, umax = _bubble_run(lbm, 2000, collision=1, tau_l=tau(0.1), tau_g=tau(0.1 / 2))
    assert st == lbm.LBM_OK and umax < 1e-2
    for z in (3, 100):
        st, umax = _bubble_run(lbm, 20000, tau_l=tau(0.1), tau_g=tau(0.1 / z))
        assert st == lbm.LBM_OK and umax < 1e-2, (z, umax)


def _deformation(phi):
    """D_f = (A - B)/(A + B) with A, B the axes of the ellipse with the same second moments as
    the region phi > 0."""
    ny, nx = phi.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    w = (phi > 0).astype(float)
    area = w.sum()
    cx, cy = (w * x).sum() / area, (w * y).sum() / area
    ixx = (w * (x - cx) ** 2).sum() / area
    iyy = (w * (y - cy) ** 2).sum() / area
    ixy = (w * (x - cx) * (y - cy)).sum() / area
    lo, hi = np.linalg.eigvalsh(np.array([[ixx, ixy], [ixy, iyy]]))
    a, b = math.sqrt(hi), math.sqrt(lo)
    return (a - b) / (a + b)


def test_taylor_deformation_in_shear(lbm):
    """Droplet-in-shear paragraph: 2H = 200, R = 30, nu_l = nu_g = 0.2, Re = v_w R^2 / (H nu)
    = 0.1, walls moving at +-v_w; D_f grows linearly with Ca = v_w R nu / (H sigma) with slope
    35/32 (paper's fit 1.09536).  The paper leaves gamma/a and the measurement of the axes
    unstated: here gamma = a (interface width 1) and the axes come from the second moments of
    phi > 0; the fitted slope lands within 5% of 35/32."""
    gold = json.load(open(GOLDEN))["taylor"]
    n, R, nu, Re = 200, 30, 0.2, 0.1
    H = n / 2
    vw = Re * H * nu / R ** 2
    cas = [0.05, 0.1, 0.15, 0.2, 0.25]
    members = []
    for ca in cas:
        sigma = vw * R * nu / (H * ca)
        ga = 3 * sigma / math.sqrt(8)  # sigma = sqrt(8 gamma a / 9) with gamma = a
        members.append((W.droplet(n, n, R, gamma=ga, a=ga),
                        dict(tau_l=tau(nu), tau_g=tau(nu), gamma=ga, a=ga, M=0.1, bc=1, u_top=vw, u_bottom=-vw)))
    bat = lbm.Batch(members, prec="fp32")
    bat.step(150000)
    assert bat.check()[0] == lbm.LBM_OK
    d = np.array([_deformation(bat.fields(m)[3]) for m in range(len(cas))])
    slope, icpt = np.polyfit(np.array(cas), d, 1)
    assert abs(slope / gold["slope_theory"] - 1) < 0.05, (slope, d)
    assert abs(icpt) < 0.02
    assert np.all(np.diff(d) > 0)


def test_interface_width_sweep_laplace(lbm):
    """Laplace paragraph after Eq. 17 at three interface widths xi = sqrt(gamma/a) in {1, sqrt 2, 2}
    with sigma = sqrt(8 gamma a / 9) held at the paper's 0.03771: bubbles of R = 15..40 on 200^2,
    zeta = 10, 30000 steps.  At gamma = a the fitted slope is close to sigma but the jump times R
    falls from 0.92 to 0.81 of sigma as R grows; at xi = sqrt 2 and 2 every bubble's jump times R
    is within 5% of sigma, and all three slopes lie within 3% of it."""
    n, radii, ratios = 200, [15, 20, 25, 30, 40], (1, 2, 4)
    sigma = math.sqrt(8 * 0.04 * 0.04 / 9)
    members = []
    for r in ratios:
        a = 3 * sigma / math.sqrt(8 * r)
        members += [(W.droplet(n, n, R, gamma=r * a, a=a),
                     dict(tau_l=tau(0.1), tau_g=tau(0.01), gamma=r * a, a=a, M=0.1, Gamma=1.0)) for R in radii]
    bat = lbm.Batch(members, prec="fp32")
    bat.step(30000)
    assert bat.check()[0] == lbm.LBM_OK
    c = n // 2
    for k, r in enumerate(ratios):
        a = 3 * sigma / math.sqrt(8 * r)
        dps = []
        for j in range(len(radii)):
            rho, _, _, phi = bat.fields(k * len(radii) + j)
            p0 = rho / 3 + a * (-0.5 * phi ** 2 + 0.75 * phi ** 4)  # Eq. 13
            dps.append(p0[c - 1:c + 1, c - 1:c + 1].mean() - p0[0, 0])
        jump = np.array(dps) * np.array(radii) / sigma
        slope = np.polyfit(1.0 / np.array(radii, dtype=float), np.array(dps), 1)[0]
        print(f"gamma/a={r}: slope/sigma-1={slope / sigma - 1:+.4f}  jump*R/sigma={np.round(jump, 3)}")
        assert abs(slope / sigma - 1) < 0.03
        if r > 1:
            assert np.all(np.abs(jump - 1) < 0.05), jump


def test_interface_width_sweep_taylor(lbm):
    """Droplet-in-shear paragraph at interface widths xi = sqrt(gamma/a) in {1, sqrt 2, 2}, run to
    600000 steps (12 wall-driven viscous times H^2 / nu): the phase field settles on a time set by
    M a, which is small at these surface tensions, so D_f still drifts by a few percent after the
    150000 steps of the gamma = a test.  With xi = sqrt 2 the slope of D_f against Ca meets 35/32
    within 1% (the paper's fit is 0.15% off); at gamma = a it overshoots and at xi = 2 (xi/R = 1/15)
    it undershoots, both within 5%."""
    gold = json.load(open(GOLDEN))["taylor"]
    n, R, nu, Re = 200, 30, 0.2, 0.1
    H = n / 2
    vw = Re * H * nu / R ** 2
    cas, ratios = [0.05, 0.1, 0.15, 0.2, 0.25], (1, 2, 4)
    members = []
    for r in ratios:
        for ca in cas:
            sigma = vw * R * nu / (H * ca)
            a = 3 * sigma / math.sqrt(8 * r)  # sigma = sqrt(8 gamma a / 9) with gamma = r a
            members.append((W.droplet(n, n, R, gamma=r * a, a=a),
                            dict(tau_l=tau(nu), tau_g=tau(nu), gamma=r * a, a=a, M=0.1, bc=1, u_top=vw,
                                 u_bottom=-vw)))
    bat = lbm.Batch(members, prec="fp32")
    bat.step(600000)
    assert bat.check()[0] == lbm.LBM_OK
    rel = {}
    for k, r in enumerate(ratios):
        d = np.array([_deformation(bat.fields(k * len(cas) + j)[3]) for j in range(len(cas))])
        slope = np.polyfit(np.array(cas), d, 1)[0]
        rel[r] = slope / gold["slope_theory"] - 1
        print(f"gamma/a={r}: slope={slope:.4f} ({rel[r]:+.4f})  D_f={np.round(d, 4)}")
        assert np.all(np.diff(d) > 0)
    assert abs(rel[2]) < 0.01, rel
    assert 0 < rel[1] < 0.05 and -0.05 < rel[4] < 0, rel


# -------------------------------------------------------------------------------------------
# Contact angles (Eq. 18 and the paragraph after it) and layered channel flow.

def _contour_points(phi):
    """Points where phi changes sign along grid rows and columns (linear interpolation)."""
    pts = []
    ny, nx = phi.shape
    for x in range(nx):
        c = phi[:, x]
        idx = np.nonzero((c[:-1] > 0) != (c[1:] > 0))[0]
        pts += [(x, y + c[y] / (c[y] - c[y + 1])) for y in idx]
    for y in range(ny):
        r = phi[y]
        idx = np.nonzero((r[:-1] > 0) != (r[1:] > 0))[0]
        pts += [(x + r[x] / (r[x] - r[x + 1]), y) for x in idx]
    return np.array(pts)


def contact_angle(phi, skip=4.0):
    """Angle (degrees, inside phi > 0) between the bottom wall (y = -1/2) and the circle fitted
    by least squares to the phi = 0 contour above y = skip - 1/2: cos(theta) = -d / R with d the
    height of the circle's centre above the wall."""
    p = _contour_points(phi)
    p = p[p[:, 1] > skip - 0.5]
    A = np.c_[2 * p[:, 0], 2 * p[:, 1], np.ones(len(p))]
    c = np.linalg.lstsq(A, (p ** 2).sum(1), rcond=None)[0]
    R = math.sqrt(c[2] + c[0] ** 2 + c[1] ** 2)
    return math.degrees(math.acos(max(-1.0, min(1.0, -(c[1] + 0.5) / R))))


def test_contact_angles_follow_eq18(lbm):
    """Sessile droplets (radius 25, started as half discs on the bottom wall) with the paper's
    contact-angle parameters gamma = a = 0.04, nu_l = 0.1, zeta = 2, and the Eq. 18 wall gradient
    for 45..135 degrees settle to angles that rise monotonically with theta, lie within 3 degrees
    of theta for 75..105 and within 8 degrees for 45..135, with errors that grow with the wall
    gradient (the trend the paper reports for its scheme).  All seven run as one batch."""
    thetas = [45, 60, 75, 90, 105, 120, 135]
    ga = 0.04
    members = [(W.droplet(200, 100, 25, gamma=ga, a=ga, cy=-0.5),
                dict(tau_l=tau(0.1), tau_g=tau(0.05), gamma=ga, a=ga, bc=lbm.LBM_WALLS_Y,
                     wet_bottom=lbm.lbm_wall_gradient(math.radians(t), ga, ga)))
               for t in thetas]
    bat = lbm.Batch(members, prec="fp32")
    bat.step(60000)
    got = [contact_angle(bat.fields(m)[3]) for m in range(len(thetas))]
    bat.close()
    err = [g - t for g, t in zip(got, thetas)]
    assert all(b > a for a, b in zip(got, got[1:])), got
    assert all(abs(e) <= 3.0 for t, e in zip(thetas, err) if 75 <= t <= 105), err
    assert all(abs(e) <= 8.0 for e in err), err
    assert abs(err[0]) > abs(err[2]) and abs(err[-1]) > abs(err[-3]), err


def test_contact_angle_paper_setup_with_force(lbm):
    """The paper's set-up: 100 x 100, droplet of radius 20 at the centre, walls at top and bottom,
    gamma = a = 0.04, nu_l = 0.1, zeta = 2 and a downward force 1e-5 on the droplet phase, which
    falls onto the bottom wall and spreads there.  sum phi is conserved to FP32 rounding (below
    1e-8 per node and step: each step rounds the nine g values of every node to 2^-24 relative)
    and the settled angle is within 10 degrees of Eq. 18 for 60 and 90 degrees (the force
    flattens the droplet: Bond number F R^2 / sigma = 0.1)."""
    ga = 0.04
    for theta in (60, 90):
        phi0 = W.droplet(100, 100, 20, gamma=ga, a=ga)
        lat = lbm.Lattice(phi0, prec="fp32", tau_l=tau(0.1), tau_g=tau(0.05), gamma=ga, a=ga,
                          bc=lbm.LBM_WALLS_Y, wet_bottom=lbm.lbm_wall_gradient(math.radians(theta), ga, ga),
                          force_y=-1e-5, force_mode=lbm.LBM_FORCE_PHASE_L)
        s0 = lat.conservation()[0]
        lat.step(60000)
        _, _, _, phi = lat.fields()
        assert abs(lat.conservation()[0] - s0) < 1e-8 * phi.size * 60000
        assert phi[0].max() > 0.5  # it reached the wall
        assert abs(contact_angle(phi) - theta) <= 10.0, (theta, contact_angle(phi))
        lat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_layered_two_viscosity_poiseuille(lbm, prec):
    """Two layers (phase l, nu = 0.1, above a flat interface; phase g, nu = 0.01, below) between walls
    driven by a uniform force: the velocity equals the exact shear-stress balance
    rho nu(y) u' = -F (y - y*) integrated with the run's own nu(phi(y)) (omega linear in phi),
    within 3e-3 of the peak speed, in FP64 and in FP32 storage (measured 1.5e-3 in FP32), with
    |u_y| at rounding level (FP64 1e-9, FP32 2e-8).  A force of 1e-6 changes each population by
    about 1e-7 per step: FP32 resolves that because it stores and computes the deviations
    f_i - w_i (rounding unit ~1e-10 here); full values f ~ 0.4 (unit 3e-8) left it 2-3% off."""
    nx, ny, F = 4, 48, 1e-6
    tl, tg = tau(0.1), tau(0.01)
    y = np.arange(ny)
    prof = np.tanh((y - (ny / 2 - 0.5)) / math.sqrt(2.0))
    lat = lbm.Lattice(np.repeat(prof[:, None], nx, axis=1), prec=prec, tau_l=tl, tau_g=tg,
                      bc=lbm.LBM_WALLS_Y, force_x=F)
    lat.step(150000)
    rho, ux, uy, phi = lat.fields()
    p, r = phi[:, 0], rho[:, 0]
    om = 1 / tg + 0.5 * (p + 1) * (1 / tl - 1 / tg)
    inv = 1.0 / (r * (1 / om - 0.5) / 3)
    yf = np.linspace(-0.5, ny - 0.5, 100001)
    fi = np.interp(yf, y, inv)
    dy = np.diff(yf)
    A = np.concatenate([[0], np.cumsum(0.5 * (fi[1:] + fi[:-1]) * dy)])
    B = np.concatenate([[0], np.cumsum(0.5 * (yf[1:] * fi[1:] + yf[:-1] * fi[:-1]) * dy)])
    want = np.interp(y, yf, -F * (B - (B[-1] / A[-1]) * A))
    print(prec, "layered Poiseuille max error / peak:", abs(ux[:, 0] - want).max() / want.max())
    assert abs(ux[:, 0] - want).max() < 3e-3 * want.max(), abs(ux[:, 0] - want).max() / want.max()
    assert abs(uy).max() < (1e-9 if prec == "fp64" else 2e-8)
    lat.close()


# -------------------------------------------------------------------------------------------
# Droplet breakup in shear (the breakup paragraph after the Taylor test).

def _components(phi):
    """Connected regions of phi > 0 on a lattice periodic in x (4-neighbour connectivity)."""
    from scipy import ndimage
    m = phi > 0
    nx = m.shape[1]
    lab, _ = ndimage.label(np.concatenate([m, m], axis=1))
    parent = {}

    def find(a):
        while parent.setdefault(a, a) != a:
            a = parent[a]
        return a
    for y, x in zip(*np.nonzero(m)):  # a region seen in both copies of the strip is one region
        parent[find(lab[y, x])] = find(lab[y, x + nx])
    return len({find(lab[y, x]) for y, x in zip(*np.nonzero(m))})


def test_droplet_breakup_in_shear(lbm):
    """240 x 60 between walls moving at +-v_w, droplet radius 15 at the centre, H = 30, the shear
    test's nu_l = nu_g = 0.2 and Re = v_w R^2 / (H nu) = 0.1, t_dag = H / v_w.  The paper shows
    the droplet stretching as one body until about 20 t_dag, its ends separating near 25 t_dag
    and satellite droplets after, but gives no capillary number; at Ca = 1.5 (gamma = a) the
    droplet is one body at 20 t_dag and three or more drops at 30 t_dag, while at Ca = 1.0 it
    only stretches.  Both run as one batch."""
    pytest.importorskip("scipy")
    nx, ny, R, nu, Re = 240, 60, 15, 0.2, 0.1
    H = ny / 2
    vw = Re * H * nu / R ** 2
    tdag = H / vw
    mem = []
    for ca in (1.5, 1.0):
        sigma = vw * R * nu / (H * ca)
        ga = 3 * sigma / math.sqrt(8)  # sigma = sqrt(8 gamma a / 9) with gamma = a
        mem.append((W.droplet(nx, ny, R, gamma=ga, a=ga),
                    dict(tau_l=tau(nu), tau_g=tau(nu), gamma=ga, a=ga, M=0.1, bc=lbm.LBM_WALLS_Y, u_top=vw,
                         u_bottom=-vw)))
    bat = lbm.Batch(mem, prec="fp32")
    s0 = [float(m[0].sum()) for m in mem]
    bat.step(int(20 * tdag))
    assert [_components(bat.fields(m)[3]) for m in range(2)] == [1, 1]
    bat.step(int(10 * tdag))
    assert bat.check()[0] == lbm.LBM_OK
    n_break, n_keep = (_components(bat.fields(m)[3]) for m in range(2))
    assert n_break >= 3 and n_keep == 1, (n_break, n_keep)
    for m in range(2):
        # sum phi to FP32 rounding over 3.4e5 steps of 14 400 nodes
        assert abs(bat.fields(m)[3].sum() - s0[m]) < 1e-8 * nx * ny * 30 * tdag
    bat.close()
