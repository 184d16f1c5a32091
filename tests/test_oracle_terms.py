"""Term-by-term pins of the oracle's step against closed forms of Eqs. 2-4.

Each background is chosen so that one coefficient of Eq. 3 (dmu/dt) or Eq. 4
(dp/dt) has a closed form; a dropped term, a wrong sign or a transposed
velocity-gradient index changes one of these numbers.
"""
import math

import numpy as np
import pytest

from fte_inputs.configs import Params
from fte_inputs.grid import GridSpec
from oracle import oracle as O

P0 = 0.0146          # ~100 keV proton
NODIFF = dict(dmumu="iso", lambda_par=1e300)


def _particle(x, y, z, mu, p=P0, pid=3):
    P = O.make_particles(1, x, y, z, mu, p)
    P["id"] = pid
    return P[0]


@pytest.mark.parametrize("mu", [-0.9, -0.2, 0.0, 0.5, 1.0])
def test_hubble_flow_momentum_rate(mu):
    """V = alpha x: grad V = alpha I, so Eq. 4 gives dp/dt = -alpha p for every mu and Eq. 3 gives 0."""
    a = 2e-5
    bg = O.analytic_background("hubble", [a, 5.0])
    prm = Params(dvdt_term=0, dt=10.0, **NODIFF)
    t = O.step_terms(bg, prm, _particle(0.3, -0.2, 0.5, mu), 0)
    assert t["divv"] == pytest.approx(3 * a, rel=1e-14)
    assert t["bbgv"] == pytest.approx(a, rel=1e-14)
    assert t["pdot_p"] == pytest.approx(-a, rel=1e-12)
    assert abs(t["mudot"]) < 1e-12 * a
    assert t["p1"] == pytest.approx(P0 * math.exp(-a * 10.0), rel=1e-14)


def test_hubble_flow_fluid_acceleration_term():
    """With the b.dV/dt term on: dV/dt = (V.grad)V = alpha^2 x, b = z_hat."""
    a = 2e-5
    bg = O.analytic_background("hubble", [a, 5.0])
    prm = Params(dvdt_term=1, dt=10.0, **NODIFF)
    x, y, z, mu = 0.3, -0.2, 0.5, 0.4
    t = O.step_terms(bg, prm, _particle(x, y, z, mu), 0)
    v = t["v"]
    assert t["bdvdt"] == pytest.approx(a * a * z, rel=1e-13)
    assert t["pdot_p"] == pytest.approx(-a - mu / v * a * a * z, rel=1e-12)
    assert t["mudot"] == pytest.approx(0.5 * (1 - mu * mu) * (-2 / v * a * a * z), rel=1e-9)


@pytest.mark.parametrize("mu", [-0.7, 0.0, 0.35, 0.9])
def test_monopole_focusing(mu):
    """|B| ~ r^-2: div b = -b.grad|B|/|B| = 2/r, so dmu/dt = (1-mu^2) v / r."""
    bg = O.analytic_background("monopole", [5.0])
    prm = Params(dt=1.0, **NODIFF)
    x, y, z = 0.2, 0.3, -0.4
    r = math.sqrt(x * x + y * y + z * z)
    t = O.step_terms(bg, prm, _particle(x, y, z, mu), 0)
    assert t["divb"] == pytest.approx(2 / r, rel=1e-13)
    assert t["mudot"] == pytest.approx((1 - mu * mu) * t["v"] / r, rel=1e-12)
    assert t["pdot_p"] == 0.0


@pytest.mark.parametrize("mu", [-0.8, -0.1, 0.3, 0.95])
def test_parallel_compression(mu):
    """V = V(x) x_hat, B || x_hat: bb:grad V = div V = V'; b.dV/dt = V V'."""
    V1, V2, w = 4e-6, 1e-6, 0.01
    bg = O.analytic_background("planar_shock", [V1, V2, w, 5.0, 0.0])
    prm = Params(dt=1.0, dvdt_term=1, **NODIFF)
    x = 0.004
    t = O.step_terms(bg, prm, _particle(x, 0.1, -0.2, mu), 0)
    th = math.tanh(x / w)
    V = V1 + (V2 - V1) * 0.5 * (1 + th)
    Vp = (V2 - V1) * 0.5 * (1 - th * th) / w
    v = t["v"]
    assert t["divv"] == pytest.approx(Vp, rel=1e-13)
    assert t["bbgv"] == pytest.approx(Vp, rel=1e-13)
    assert t["bdvdt"] == pytest.approx(V * Vp, rel=1e-13)
    assert t["pdot_p"] == pytest.approx(-mu * mu * Vp - mu / v * V * Vp, rel=1e-11, abs=1e-25)
    assert t["mudot"] == pytest.approx(0.5 * (1 - mu * mu) * (-2 * mu * Vp - 2 * V * Vp / v),
                                       rel=1e-11, abs=1e-25)


@pytest.mark.parametrize("mu", [-0.6, 0.0, 0.45])
def test_perpendicular_compression(mu):
    """B perpendicular to the flow: bb:grad V = 0 and b.dV/dt = 0, so dp/dt/p = -(1-mu^2)/2 V'."""
    V1, V2, w = 4e-6, 1e-6, 0.01
    bg = O.analytic_background("planar_shock", [V1, V2, w, 5.0, math.pi / 2])
    prm = Params(dt=1.0, dvdt_term=1, **NODIFF)
    x = -0.003
    t = O.step_terms(bg, prm, _particle(x, 0.0, 0.0, mu), 0)
    th = math.tanh(x / w)
    Vp = (V2 - V1) * 0.5 * (1 - th * th) / w
    assert abs(t["bbgv"]) < 1e-12 * abs(Vp)
    assert t["pdot_p"] == pytest.approx(-(1 - mu * mu) / 2 * Vp, rel=1e-10)
    assert t["mudot"] == pytest.approx((1 - mu * mu) / 2 * mu * Vp, rel=1e-10, abs=1e-15 * abs(Vp))


def test_radial_wind_adiabatic_rate():
    """V = V0 r_hat, radial B: div V = 2 V0 / r, bb:grad V = 0, so dp/dt/p = -(1-mu^2) V0 / r."""
    V0 = 2.67e-6
    bg = O.analytic_background("radial_wind", [V0, 5.0])
    prm = Params(dt=1.0, dvdt_term=1, **NODIFF)
    x, y, z, mu = 0.5, 0.5, 0.2, 0.3
    r = math.sqrt(x * x + y * y + z * z)
    t = O.step_terms(bg, prm, _particle(x, y, z, mu), 0)
    assert t["divv"] == pytest.approx(2 * V0 / r, rel=1e-13)
    assert abs(t["bbgv"]) < 1e-13 * V0 / r
    assert abs(t["bdvdt"]) < 1e-20
    assert t["pdot_p"] == pytest.approx(-(1 - mu * mu) * V0 / r, rel=1e-12)


def test_update_rules():
    """x' = x + (V + mu v b) dt (Eq. 2), mu' = mu + (mu_dot + dD/dmu) dt + sqrt(2 D dt) z,
    p' = p exp(p_dot/p dt) (or p (1 + p_dot/p dt))."""
    V0 = 2.67e-6
    bg = O.analytic_background("radial_wind", [V0, 5.0])
    prm = Params(dmumu="qlt", lambda_par=0.05, dt=7.0)
    P = _particle(0.4, -0.3, 0.1, 0.37, p=0.03, pid=17)
    t = O.step_terms(bg, prm, P, 123)
    z = O.normals(prm.seed, prm.set_id, 123, 17)
    assert (t["z0"], t["z1"], t["z2"]) == tuple(z)
    dt = prm.dt
    mu1 = 0.37 + (t["mudot"] + t["dD"]) * dt + math.sqrt(2 * t["D"] * dt) * z[0]
    assert t["mu1"] == pytest.approx(mu1, rel=1e-14)
    b = np.array([t["bx"], t["by"], t["bz"]])
    V = np.array([t["Vx"], t["Vy"], t["Vz"]])
    x1 = np.array([0.4, -0.3, 0.1]) + (V + 0.37 * t["v"] * b) * dt
    assert [t["x1"], t["y1"], t["z1_"]] == pytest.approx(list(x1), rel=1e-14)
    assert t["p1"] == pytest.approx(0.03 * math.exp(t["pdot_p"] * dt), rel=1e-14)
    prm.p_update = "euler"
    t2 = O.step_terms(bg, prm, P, 123)
    assert t2["p1"] == pytest.approx(0.03 * (1 + t["pdot_p"] * dt), rel=1e-14)
    assert t["t"] == 123 * dt


def test_kinematics():
    """v = c p / gamma; E = m c^2 (gamma - 1) (Sec. 2.1 definitions)."""
    bg = O.analytic_background("uniform_b", [5.0])
    for e in (0.01, 0.1, 1.0, 100.0):
        T = e / O.MC2
        p = math.sqrt(T * (T + 2))
        t = O.step_terms(bg, Params(**NODIFF), _particle(1, 0, 0, 0.1, p=p), 0)
        g = 1 + T
        assert t["E"] == pytest.approx(e, rel=1e-13)
        assert t["v"] == pytest.approx(O.C_AU * math.sqrt(1 - 1 / g ** 2), rel=1e-12)


def test_cross_field_drift_monopole():
    """Radial field lines: (b.grad) b = 0, div b = 2/r, so div(kappa_perp) = -kappa (2/r) r_hat."""
    bg = O.analytic_background("monopole", [5.0])
    lam_perp = 3e-4
    prm = Params(dt=1.0, lambda_perp=lam_perp, kappa_drift=1, **NODIFF)
    x, y, z = 0.3, 0.1, 0.2
    r = math.sqrt(x * x + y * y + z * z)
    t = O.step_terms(bg, prm, _particle(x, y, z, 0.2), 0)
    kap = t["v"] * lam_perp / 3
    assert t["kappa"] == pytest.approx(kap, rel=1e-14)
    u = np.array([t["ux"], t["uy"], t["uz"]])
    assert u == pytest.approx(-kap * 2 / r * np.array([x, y, z]) / r, rel=1e-10)


def test_cross_field_drift_curvature_on_grid():
    """Azimuthal field B = B0 phi_hat (circles about z): div b = 0 and (b.grad) b = -rho_hat / rho,
    so div(kappa_perp) = +kappa rho_hat / rho.  The curvature comes from the derivative of the
    trilinear interpolant of the gridded B; it converges to the analytic value."""
    g = GridSpec(nr=64, nth=64, nph=256, r_min=0.5, r_max=1.5)
    from fte_inputs.grid import cell_centres, REC
    r, th, ph = cell_centres(g)
    f = np.zeros((1, g.nph, g.nth, g.nr, REC), np.float32)
    f[0, ..., 0] = (-np.sin(ph))[:, None, None] * 5.0
    f[0, ..., 1] = (np.cos(ph))[:, None, None] * 5.0
    bg = O.grid_background(g, f)
    lam_perp = 3e-4
    prm = Params(dt=1.0, lambda_perp=lam_perp, kappa_drift=1, **NODIFF)
    x, y, z = 0.61, 0.52, 0.13
    rho = math.hypot(x, y)
    t = O.step_terms(bg, prm, _particle(x, y, z, 0.2), 0)
    kap = t["v"] * lam_perp / 3
    u = np.array([t["ux"], t["uy"], t["uz"]])
    expect = kap * np.array([x, y, 0.0]) / rho ** 2
    assert np.linalg.norm(u - expect) < 2e-3 * np.linalg.norm(expect)
