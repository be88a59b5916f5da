"""Wetting walls (Eq. 18 ghost rows) and the body force (Guo's source in central-moment form) on
the CUDA path against the FP64 oracle, called through the C ABI.

Tolerances as for the rest of the scheme: FP64 storage 1e-12 (relative to the field's maximum;
absolute for velocities), FP32 storage 1e-5 on phi, 16-bit storage 2e-3 on phi (FP16).
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


def _pair(lbm, orc, phi0, steps, **kw):
    lat = lbm.Lattice(phi0, **kw)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    lat.step(steps)
    o.step(steps)
    return lat, o


def _fp64_parity(lat, o, tol=1e-12):
    rg, uxg, uyg, pg = lat.fields()
    ro, uxo, uyo, po = o.fields()
    assert rel_err(pg, po) <= tol, rel_err(pg, po)
    assert rel_err(rg, ro) <= tol, rel_err(rg, ro)
    assert abs_err(uxg, uxo) <= tol and abs_err(uyg, uyo) <= tol, (abs_err(uxg, uxo), abs_err(uyg, uyo))
    fg, gg = lat.populations()
    fo, go = o.populations()
    assert rel_err(fg, fo) <= tol, rel_err(fg, fo)
    assert rel_err(gg, go) <= tol, rel_err(gg, go)


def _sessile(nx, ny, R, gamma=0.04, a=0.04):
    """Droplet of radius R whose centre sits R - 2 above the bottom wall (it already touches)."""
    return W.droplet(nx, ny, R, gamma=gamma, a=a, cy=R - 2.0)


@pytest.mark.parametrize("theta_deg,mode", [(60, 1), (120, 1), (45, 0)])
def test_sessile_droplet_wetting_and_force_fp64(lbm, orc, theta_deg, mode):
    """Contact-angle set-up (walls, Eq. 18 gradient on the bottom wall, downward force on the
    droplet phase or everywhere), ragged 70 x 45 lattice, CM collision, 400 steps."""
    h = orc.wall_gradient(math.radians(theta_deg), 0.04, 0.04)
    phi0 = _sessile(70, 45, 12)
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.8, tau_g=0.65, bc=lbm.LBM_WALLS_Y, wet_bottom=h, force_y=-1e-4,
              force_mode=mode)
    lat, o = _pair(lbm, orc, phi0, 400, **kw)
    _fp64_parity(lat, o)


def test_both_walls_wet_moving_and_bgk_fp64(lbm, orc):
    """Different gradients on the two walls, moving walls and a sideways force, with both
    collisions."""
    phi0 = W.layers(48, 30, 6.0, 22.0, 0.04, 0.04)
    for coll in (0, 1):
        kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.7, bc=lbm.LBM_WALLS_Y, wet_bottom=0.2, wet_top=-0.15,
                  u_top=0.01, u_bottom=-0.005, force_x=2e-5, force_y=-1e-5, collision=coll)
        lat, o = _pair(lbm, orc, phi0, 300, **kw)
        _fp64_parity(lat, o)
        lat.close()


@pytest.mark.parametrize("nx,ny", [(67, 45), (3, 3)])
def test_periodic_force_fp64(lbm, orc, nx, ny):
    """Uniform force on a periodic ragged / minimal lattice with random initial velocities."""
    phi0 = W.droplet(nx, ny, min(nx, ny) / 3, gamma=0.04, a=0.04)
    rng = np.random.default_rng(nx + ny)
    ux0 = 0.01 * rng.standard_normal((ny, nx))
    uy0 = 0.01 * rng.standard_normal((ny, nx))
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.6, force_x=3e-5, force_y=1e-5)
    lat = lbm.Lattice(phi0, ux0, uy0, **kw)
    o = orc.Oracle(phi0, ux0, uy0, **oracle_kwargs(kw))
    lat.step(150)
    o.step(150)
    _fp64_parity(lat, o)


GENERIC_TILES = [(32, 4), (32, 8), (64, 2), (64, 4), (128, 1), (128, 2), (256, 1)]
STAGED_TILES = [(32, 4, 1), (32, 8, 1), (64, 2, 1), (64, 4, 1), (64, 4, 2), (128, 2, 1), (128, 1, 2)]


def test_every_tile_with_wetting_and_force_fp64(lbm, orc):
    """Each compiled tile of both kernels applies the ghost rows and the force (nx = 136: a
    ragged multiple of every tile width; rows = 7 puts segment edges next to the walls)."""
    nx, ny = 136, 45
    phi0 = _sessile(nx, ny, 14)
    kw = dict(prec=lbm.LBM_FP64, tau_l=0.9, tau_g=0.55, bc=lbm.LBM_WALLS_Y, wet_bottom=0.25, wet_top=-0.1,
              force_y=-5e-5, force_mode=1)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(40)
    variants = [(lbm.LBM_KERNEL_GENERIC, bx, by, 0) for bx, by in GENERIC_TILES]
    variants += [(lbm.LBM_KERNEL_STAGED, bx, by, d) for bx, by, d in STAGED_TILES]
    variants += [(lbm.LBM_KERNEL_GENERIC_WIDE, bx, by, 0) for bx, by in GENERIC_TILES]
    for var, bx, by, d in variants:
        for rows in (0, 7):
            lat = lbm.Lattice(phi0, **kw)
            lat.set_kernel(var, bx, by, d, rows)
            lat.step(40)
            _fp64_parity(lat, o)
            lat.close()


@pytest.fixture(scope="module")
def contact_angle_setup(orc):
    """The contact-angle set-up (a droplet falling under a force of 1e-5 onto a wall with the
    60-degree gradient of Eq. 18) and the oracle's fields after 1000 steps."""
    h = orc.wall_gradient(math.radians(60), 0.04, 0.04)
    phi0 = W.droplet(100, 100, 20, gamma=0.04, a=0.04, cy=30.0)
    kw = dict(tau_l=orc.tau_from_nu(0.1), tau_g=orc.tau_from_nu(0.05), bc=1, wet_bottom=h,
              force_y=-1e-5, force_mode=1)
    o = orc.Oracle(phi0, **oracle_kwargs(kw))
    o.step(1000)
    return phi0, kw, o.fields()


@pytest.mark.parametrize("prec,bound", [
    ("fp32", 1e-5), ("fp16s", 2e-3),
    pytest.param("bf16s", 2e-3, marks=pytest.mark.xfail(
        strict=True, reason="BF16 storage does not resolve the 1e-5 body force: the per-step momentum it adds "
                            "(~3e-6 per population) is below BF16's rounding unit of the stored deviations; "
                            "measured 4.5e-2 on phi"))])
def test_contact_angle_setup_reduced_precision(lbm, contact_angle_setup, prec, bound):
    """The contact-angle set-up after 1000 steps against the FP64 oracle: the contract on phi,
    1e-5 for FP32 storage (measured 5.3e-7) and 2e-3 for 16-bit storage (FP16 3.4e-4); velocities
    within twice those."""
    phi0, kw, (_, uxo, uyo, po) = contact_angle_setup
    lat = lbm.Lattice(phi0, prec=prec, **kw)
    lat.step(1000)
    _, uxg, uyg, pg = lat.fields()
    lat.close()
    print(prec, "contact-angle set-up, max |phi - phi_oracle|:", abs_err(pg, po),
          "max |u - u_oracle|:", max(abs_err(uxg, uxo), abs_err(uyg, uyo)))
    assert abs_err(pg, po) <= bound, (prec, abs_err(pg, po))
    assert abs_err(uxg, uxo) <= 2 * bound and abs_err(uyg, uyo) <= 2 * bound, prec


def test_batch_members_with_wetting_and_force_fp64(lbm, orc):
    """A batch mixing a wetting/forced member with a plain periodic one matches the oracle."""
    h = orc.wall_gradient(math.radians(120), 0.04, 0.04)
    members = [
        (_sessile(64, 40, 10), dict(tau_l=0.8, tau_g=0.6, bc=lbm.LBM_WALLS_Y, wet_bottom=h, force_y=-1e-4,
                                    force_mode=1)),
        (W.spinodal(48, 48, seed=5), dict(tau_l=0.8, tau_g=0.6, force_x=1e-5)),
    ]
    bat = lbm.Batch(members, prec="fp64")
    bat.step(200)
    for m, (phi0, params) in enumerate(members):
        o = orc.Oracle(phi0, **oracle_kwargs(params))
        o.step(200)
        rg, uxg, uyg, pg = bat.fields(m)
        ro, uxo, uyo, po = o.fields()
        assert rel_err(pg, po) <= 1e-12 and rel_err(rg, ro) <= 1e-12, m
        assert abs_err(uxg, uxo) <= 1e-12 and abs_err(uyg, uyo) <= 1e-12, m
        o.close()
    bat.close()


def test_momentum_grows_by_the_force_on_gpu(lbm):
    """Device totals: on a periodic lattice sum phi is conserved and the momentum grows by
    F sum (1 + phi)/2 per step for a force on phase l (FP64 storage)."""
    phi0 = W.droplet(96, 64, 18, gamma=0.04, a=0.04)
    F = (2e-5, -1e-5)
    lat = lbm.Lattice(phi0, prec=lbm.LBM_FP64, force_x=F[0], force_y=F[1], force_mode=lbm.LBM_FORCE_PHASE_L)
    s0 = lat.conservation()
    lat.step(500)
    s1 = lat.conservation()
    w = ((1 + phi0) / 2).sum()
    assert abs(s1[0] - s0[0]) < 1e-12 * phi0.size
    np.testing.assert_allclose(np.array(s1[2:4]) - np.array(s0[2:4]), 500 * np.array(F) * w, rtol=1e-9)
    lat.close()
