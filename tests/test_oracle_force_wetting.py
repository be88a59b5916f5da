"""Pins of the oracle's wetting walls and body force (the contact-angle test of arXiv:1803.11345,
Eq. 18 and the paragraph around it, which applies a force but prints no forcing scheme).

The force follows Guo, Zheng & Shi, Phys. Rev. E 65, 046308 (2002); its central-moment form is
pinned by the reduction to the forced BGK collision, the moments of the source term, momentum
bookkeeping and textbook Poiseuille flows.  The wall gradient is pinned against Young's law
evaluated from the paper's free energy, and the wall profile against the continuum first
integral of that free energy.
"""
import math

import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


# ---------------------------------------------------------------------------------------
# Eq. 18 against Young's law.

def _young_angle(h, a, gamma):
    """Contact angle (degrees) that a wall gradient h of phi along the outward normal gives,
    from Young's law cos(theta) = (sigma_w- - sigma_w+) / sigma with the free energy
    psi = a(-phi^2/2 + phi^4/4) + (gamma/2)|grad phi|^2 and a linear wall energy: for each bulk
    phase +-1 the wall value phi_s follows from the first integral gamma phi'^2 = 2 (psi -
    psi_bulk) = (a/2)(1 - phi^2)^2 and phi'(wall) = -h, the wall tension is the wall energy plus
    the profile energy int_{phi_s}^{+-1} sqrt(a gamma / 2) |1 - phi^2| dphi, and
    sigma = sqrt(8 gamma a / 9)."""
    k = math.sqrt(a / (2 * gamma))
    s = math.sqrt(a * gamma / 2)
    g = -h  # derivative into the fluid
    prim = lambda p: p - p ** 3 / 3  # noqa: E731
    # wall values for bulk +1 (monotone profile, phi' = k(1 - phi^2)) and bulk -1
    sp, sm = math.sqrt(1 - g / k), -math.sqrt(1 + g / k)
    wall_p = gamma * g * sp + s * abs(prim(1.0) - prim(sp))
    wall_m = gamma * g * sm + s * abs(prim(-1.0) - prim(sm))
    sigma = math.sqrt(8 * gamma * a / 9)
    return math.degrees(math.acos((wall_m - wall_p) / sigma))


@pytest.mark.parametrize("ratio", [1.0, 4.0])
def test_wall_gradient_reproduces_youngs_law(orc, ratio):
    """Eq. 18 (square root over the whole product, sign(90 deg - theta)) inverts Young's law of
    the paper's free energy exactly, for hydrophilic and hydrophobic angles."""
    a = 0.04
    gamma = a * ratio
    for theta in (5, 20, 45, 60, 80, 90, 100, 120, 150, 175):
        h = orc.wall_gradient(math.radians(theta), a, gamma)
        assert math.isclose(_young_angle(h, a, gamma), theta, abs_tol=1e-8), theta
        assert (h > 0) == (theta < 90) and (h < 0) == (theta > 90)
    assert orc.wall_gradient(math.pi / 2, a, gamma) == 0.0


# ---------------------------------------------------------------------------------------
# Forcing.

def test_guo_source_moments(orc):
    """Guo's term has zero mass, momentum F and second moments u F + F u (Guo et al. 2002)."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        ux, uy, fx, fy = 0.1 * rng.standard_normal(4)
        S = orc.guo_source(ux, uy, fx, fy)
        assert abs(S.sum()) < 1e-15 * abs(S).max()
        assert math.isclose((S * CX).sum(), fx, rel_tol=1e-13, abs_tol=1e-18)
        assert math.isclose((S * CY).sum(), fy, rel_tol=1e-13, abs_tol=1e-18)
        assert math.isclose((S * CX * CX).sum(), 2 * ux * fx, rel_tol=1e-12, abs_tol=1e-18)
        assert math.isclose((S * CY * CY).sum(), 2 * uy * fy, rel_tol=1e-12, abs_tol=1e-18)
        assert math.isclose((S * CX * CY).sum(), ux * fy + uy * fx, rel_tol=1e-12, abs_tol=1e-18)


def _rand_f(rng, orc):
    f = orc.feq(1 + 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(), 0.05 * rng.standard_normal(),
                0.35, 0.2 * rng.standard_normal(), 0.2 * rng.standard_normal(), 0.04)
    return f + 0.01 * rng.standard_normal(9)


def test_forced_equal_rates_reduce_to_forced_bgk(orc):
    """With every rate equal to omega_rho, the forced central-moment collision (source projected
    with (1 - omega/2) on each moment, k*_1,2 = F/2) equals Guo's forced BGK collision."""
    rng = np.random.default_rng(4)
    for tau in (0.6, 1.0, 1.4):
        om = 1 / tau
        for mode in (0, 1):
            kw = dict(tau_l=tau, tau_g=tau, Fx=2e-3, Fy=-3e-3, force_mode=mode)
            cm = orc.make_params(4, 4, omega3=om, omega6=om, omega7=om, omega8=om, **kw)
            bgk = orc.make_params(4, 4, collision=1, **kw)
            for _ in range(8):
                f = _rand_f(rng, orc)
                args = (rng.uniform(-1, 1), 0.2 * rng.standard_normal(), 0.2 * rng.standard_normal(),
                        0.05 * rng.standard_normal())
                np.testing.assert_allclose(orc.collide_f(cm, f, *args), orc.collide_f(bgk, f, *args),
                                           rtol=0, atol=1e-14)


def test_collision_adds_the_force(orc):
    """Both collisions conserve mass and add exactly F(phi) to the momentum; F acts on phase l
    only with weight (1 + phi)/2 in force_mode 1."""
    rng = np.random.default_rng(5)
    for extra in (dict(), dict(collision=1)):
        for mode in (0, 1):
            P = orc.make_params(4, 4, tau_l=0.9, tau_g=0.6, Fx=1e-3, Fy=2e-3, force_mode=mode, **extra)
            for phi in (-1.0, -0.3, 0.4, 1.0):
                f = _rand_f(rng, orc)
                fs = orc.collide_f(P, f, phi, 0.1, -0.2, 0.03)
                w = 1.0 if mode == 0 else (1 + phi) / 2
                np.testing.assert_allclose(orc.force(P, phi), [1e-3 * w, 2e-3 * w], rtol=1e-15, atol=0)
                assert math.isclose(fs.sum(), f.sum(), abs_tol=1e-15)
                assert math.isclose((fs * CX).sum() - (f * CX).sum(), 1e-3 * w, abs_tol=1e-15)
                assert math.isclose((fs * CY).sum() - (f * CY).sum(), 2e-3 * w, abs_tol=1e-15)


def test_velocity_is_half_force_corrected(orc):
    """A uniform lattice at rest under a uniform force: the initial collision adds F, each step
    adds F, and the reported velocity is that of the last collision, (n + 1/2) F / rho."""
    F = 1e-5
    o = orc.Oracle(np.full((4, 5), 0.3), Fx=F, Fy=-2 * F, tau_l=0.9, tau_g=0.7)
    for n in (0, 7):
        if n:
            o.step(n)
        rho, ux, uy, _ = o.fields()
        np.testing.assert_allclose(ux, (n + 0.5) * F / rho, rtol=1e-10)
        np.testing.assert_allclose(uy, -2 * (n + 0.5) * F / rho, rtol=1e-10)
    o.close()


def test_periodic_momentum_grows_by_the_total_force(orc):
    """On a periodic two-phase lattice the total momentum grows by sum_x F(phi) per step: N F
    for a uniform force, F sum (1 + phi)/2 (exact, as sum phi is conserved) on phase l only."""
    ny, nx = 12, 14
    y, x = np.mgrid[0:ny, 0:nx]
    phi = np.tanh(4 - np.hypot(x - 6.5, y - 5.5) / 1.2)
    F = np.array([3e-5, -1e-5])
    for mode in (0, 1):
        o = orc.Oracle(phi, tau_l=0.8, tau_g=0.6, Fx=F[0], Fy=F[1], force_mode=mode)
        s0 = np.array(o.sums())
        o.step(200)
        s1 = np.array(o.sums())
        wsum = phi.size if mode == 0 else ((1 + phi) / 2).sum()
        np.testing.assert_allclose(s1[2:] - s0[2:], 200 * F * wsum, rtol=1e-10)
        assert abs(s1[0] - s0[0]) < 1e-12 * phi.size
        o.close()


def _poiseuille_exact(F, nu_of_y, rho_of_y, ny):
    """Steady channel flow between halfway walls at y = -1/2 and ny - 1/2 for force F: the shear
    stress rho nu u' = -F (y - y*) is linear, y* from u = 0 on both walls; 1/(rho nu) is taken
    piecewise linear between nodes and constant from the last nodes to the walls."""
    y = np.arange(ny)
    yf = np.linspace(-0.5, ny - 0.5, 100001)
    inv = np.interp(yf, y, 1.0 / (rho_of_y * nu_of_y))
    dy = np.diff(yf)
    A = np.concatenate([[0], np.cumsum(0.5 * (inv[1:] + inv[:-1]) * dy)])
    B = np.concatenate([[0], np.cumsum(0.5 * (yf[1:] * inv[1:] + yf[:-1] * inv[:-1]) * dy)])
    ystar = B[-1] / A[-1]
    return np.interp(y, yf, -F * (B - ystar * A))


@pytest.mark.parametrize("tau", [0.8, 1.0])
def test_single_phase_poiseuille(orc, tau):
    """One phase between no-slip walls driven by a uniform force: the parabola
    u = F (y + 1/2)(ny - 1/2 - y) / (2 rho nu), nu = (tau - 1/2)/3, within 1e-3 (the
    halfway-bounce-back slip of this collision is a few 1e-4)."""
    nx, ny, F = 3, 24, 1e-6
    o = orc.Oracle(np.full((ny, nx), -1.0), walls=1, tau_l=tau, tau_g=tau, Fx=F)
    o.step(12000)
    rho, ux, uy, _ = o.fields()
    nu = (tau - 0.5) / 3
    yy = np.arange(ny)
    want = F * (yy + 0.5) * (ny - 0.5 - yy) / (2 * nu)
    assert abs(ux[:, 0] - want).max() < 1e-3 * want.max()
    assert abs(uy).max() < 1e-12
    o.close()


def test_layered_two_viscosity_poiseuille(orc):
    """Two layers (viscosity ratio 10) separated by a flat interface parallel to the walls: the
    exact shear-stress balance evaluated with the oracle's own nu(phi(y)) (omega linear in phi),
    within 3e-3 of the peak speed."""
    nx, ny, F = 3, 48, 1e-6
    tau_l = 0.8
    nu_l = (tau_l - 0.5) / 3
    tau_g = 3 * nu_l / 10 + 0.5
    y = np.arange(ny)
    prof = np.tanh((y - (ny / 2 - 0.5)) / math.sqrt(2))
    o = orc.Oracle(np.repeat(prof[:, None], nx, axis=1), walls=1, tau_l=tau_l, tau_g=tau_g, Fx=F)
    o.step(50000)
    rho, ux, _, phi = o.fields()
    p = phi[:, 0]
    om = 1 / tau_g + 0.5 * (p + 1) * (1 / tau_l - 1 / tau_g)
    want = _poiseuille_exact(F, (1 / om - 0.5) / 3, rho[:, 0], ny)
    assert abs(ux[:, 0] - want).max() < 3e-3 * want.max()
    o.close()


# ---------------------------------------------------------------------------------------
# Wetting walls.

def test_stencil_wall_ghost_rows(orc):
    """The ghost rows are the adjacent rows plus the wall gradients: a linear profile
    phi = s y whose ghosts continue it (wet_bottom = -s, wet_top = +s) has the exact stencil
    values at the wall rows."""
    ny, nx, s = 6, 5, 0.3
    phi = np.repeat((s * np.arange(ny))[:, None], nx, axis=1)
    gx, gy, lap = orc.stencils(phi, walls=True, wet_bottom=-s, wet_top=s)
    np.testing.assert_allclose(gy, s, atol=1e-15)
    np.testing.assert_allclose(lap, 0, atol=1e-15)
    np.testing.assert_allclose(gx, 0, atol=1e-15)


def test_wetting_walls_conserve_phi(orc):
    """Bounce-back returns every g population, so sum phi stays exact with wetting walls."""
    ny, nx = 14, 12
    y, x = np.mgrid[0:ny, 0:nx]
    phi = np.tanh(3 - np.hypot(x - 5.5, y - 2.0) / 1.5)
    o = orc.Oracle(phi, walls=1, wet_bottom=0.2, wet_top=-0.1, Fy=-1e-5, force_mode=1)
    s0 = o.sums()
    o.step(300)
    s1 = o.sums()
    assert abs(s1[0] - s0[0]) < 1e-12 * phi.size
    assert abs(s1[1] - s0[1]) < 1e-12 * phi.size
    o.close()


def _wall_profile(pb, h, a, gamma, zs):
    """Continuum steady profile next to a wall with gradient h along the outward normal and
    bulk value pb far away: gamma phi'^2 = 2 [psi(phi) - psi(pb) - mu(pb)(phi - pb)] (first
    integral of mu = const), wall value from phi'^2 = h^2, integrated from the wall."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq
    psi = lambda p: a * (-p * p / 2 + p ** 4 / 4)  # noqa: E731
    mub = a * (pb ** 3 - pb)
    V = lambda p: (2 / gamma) * (psi(p) - psi(pb) - mub * (p - pb))  # noqa: E731
    if h > 0:
        ps = brentq(lambda p: V(p) - h * h, pb + 1e-12, 0.0)
    else:
        ps = brentq(lambda p: V(p) - h * h, -3.0, pb - 1e-12)
    sgn = -1.0 if h > 0 else 1.0
    sol = solve_ivp(lambda z, y: [sgn * math.sqrt(max(V(y[0]), 0.0))], (0, max(zs)), [ps], t_eval=zs,
                    rtol=1e-11, atol=1e-13)
    return sol.y[0]


def test_wetting_wall_profile_matches_the_free_energy(orc):
    """A single bulk phase next to a wall with the Eq. 18 gradient for 60 and 120 degrees relaxes
    to the continuum wall profile of the free energy (nodes at distance 1/2, 3/2, ... from the
    wall); the error falls as the interface widens (second-order stencils)."""
    pytest.importorskip("scipy")
    ny, nx, a = 24, 1, 0.04
    nthreads = orc.set_threads(0)
    orc.set_threads(1)  # 24 nodes: threads cost more than they save
    errs = {}
    for ratio, theta in ((1, 60), (4, 60), (4, 120)):
        gamma = a * ratio
        h = orc.wall_gradient(math.radians(theta), a, gamma)
        o = orc.Oracle(np.full((ny, nx), -1.0), walls=1, gamma=gamma, a=a, wet_bottom=h)
        o.step(150000)
        _, ux, _, phi = o.fields()
        p = phi[:, 0]
        want = _wall_profile(p[ny // 2], h, a, gamma, np.arange(6) + 0.5)
        errs[(ratio, theta)] = abs(p[:6] - want).max()
        assert abs(ux).max() < 1e-12
        o.close()
    orc.set_threads(nthreads)
    assert errs[(4, 60)] < 1.5e-3 and errs[(4, 120)] < 3e-3, errs
    assert errs[(4, 60)] < 0.5 * errs[(1, 60)], errs
