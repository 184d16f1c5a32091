"""Pins of the pitch-angle diffusion coefficient and its normalisation.

Sec. 2.1, Eq. 5: D_mumu = D0 (|mu|/(1+|mu|) + eps)(1 - mu^2), eps = 0.048, with D0
fixed by the particle's rigidity through a prescribed parallel mean free path.
The build reads the normalisation as the standard quasi-linear relation
lambda_par = (3v/8) int_{-1}^{1} (1-mu^2)^2 / D_mumu dmu; the quasi-linear slab
form (nu/2)(1-mu^2)(|mu|^(q-1) + H) and the isotropic form D(1-mu^2) are the
other modules.
"""
import math

import numpy as np

import pytest
import sympy as sp
from scipy import integrate

from fte_inputs.configs import Params
from oracle import oracle as O


def _closed_form_J(eps):
    m = sp.symbols("m", positive=True)
    e = sp.Rational(eps).limit_denominator(10 ** 9) if not isinstance(eps, sp.Rational) else eps
    expr = (1 - m ** 2) / (m / (1 + m) + e)
    return float(sp.integrate(sp.simplify(expr), (m, 0, 1)).evalf(30)), float(e)


def test_paper_eq5_normalisation_closed_form():
    """J = int_0^1 (1-mu^2)/(mu/(1+mu)+eps) dmu is elementary (rational integrand)."""
    for eps in (sp.Rational(48, 1000), sp.Rational(1, 10), sp.Rational(1, 100)):
        J, e = _closed_form_J(eps)
        assert O.norm_integral("paper", eps=e) == pytest.approx(J, rel=1e-12)


def test_qlt_normalisation_q2_closed_form():
    """For q = 2, I = int_0^1 (1-mu^2)/(mu+H) dmu = (1-H^2) ln((1+H)/H) + H - 1/2."""
    for H in (0.05, 0.2, 0.01):
        closed = (1 - H * H) * math.log((1 + H) / H) + H - 0.5
        assert O.norm_integral("qlt", q=2.0, H=H) == pytest.approx(closed, rel=1e-12)


def test_qlt_normalisation_library_quadrature():
    for q, H in ((5 / 3, 0.05), (1.5, 0.1), (5 / 3, 0.01)):
        ref, _ = integrate.quad(lambda m: (1 - m * m) / (m ** (q - 1) + H), 0, 1,
                                epsabs=1e-14, epsrel=1e-13, limit=400)
        assert O.norm_integral("qlt", q=q, H=H) == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("model", ["qlt", "paper", "iso"])
def test_mean_free_path_relation(model):
    """lambda_par = (3v/8) int (1-mu^2)^2 / D dmu, evaluated with a library quadrature on D."""
    prm = Params(dmumu=model, lambda_par=0.3)
    p = 0.0146
    v = O.speed_of_p(p)
    f = lambda m: (1 - m * m) ** 2 / O.dmumu(prm, m, v, p)[0]
    a, _ = integrate.quad(f, -1, 0, limit=400, epsrel=1e-12, points=[-1e-3])
    b, _ = integrate.quad(f, 0, 1, limit=400, epsrel=1e-12, points=[1e-3])
    assert 3 * v / 8 * (a + b) == pytest.approx(0.3, rel=1e-8)


@pytest.mark.parametrize("model", ["qlt", "paper", "iso"])
def test_derivative_matches_difference_quotient(model):
    prm = Params(dmumu=model, lambda_par=0.2, mu_floor=1e-12)
    p = 0.02
    v = O.speed_of_p(p)
    for mu in (-0.93, -0.5, -0.07, 0.03, 0.4, 0.88):
        h = 1e-6
        num = (O.dmumu(prm, mu + h, v, p)[0] - O.dmumu(prm, mu - h, v, p)[0]) / (2 * h)
        assert O.dmumu(prm, mu, v, p)[1] == pytest.approx(num, rel=1e-6, abs=1e-14)


def test_forms_and_floor():
    p = 0.02
    v = O.speed_of_p(p)
    prm = Params(dmumu="qlt", lambda_par=0.1, q=5 / 3, H=0.05, mu_floor=1e-4)
    D, dD, nu = O.dmumu(prm, 0.3, v, p)
    assert nu == pytest.approx(3 * v * O.norm_integral("qlt") / (2 * 0.1), rel=1e-14)
    assert D == pytest.approx(0.5 * nu * (1 - 0.09) * (0.3 ** (2 / 3) + 0.05), rel=1e-14)
    # at mu = 0: sgn(0) = 0, so the singular factor drops out
    assert O.dmumu(prm, 0.0, v, p)[1] == 0.0
    # below the floor the singular factor is held at mu_floor^(q-2)
    d_small = O.dmumu(prm, 1e-8, v, p)[1]
    expect = 0.5 * nu * (-2e-8 * (1e-8 ** (2 / 3) + 0.05) + (1 - 1e-16) * (2 / 3) * 1e-4 ** (-1 / 3))
    assert d_small == pytest.approx(expect, rel=1e-12)
    prm = Params(dmumu="paper", lambda_par=0.3, eps=0.048)
    D, dD, D0 = O.dmumu(prm, -0.6, v, p)
    assert D == pytest.approx(D0 * (0.6 / 1.6 + 0.048) * (1 - 0.36), rel=1e-14)
    prm = Params(dmumu="iso", lambda_par=0.3)
    D, dD, Dc = O.dmumu(prm, 0.5, v, p)
    assert Dc == pytest.approx(v / 0.6, rel=1e-14) and D == pytest.approx(Dc * 0.75, rel=1e-14)


def test_rigidity_scaling():
    p_ref = 0.0462  # ~1 MeV proton
    prm = Params(dmumu="iso", lambda_par=0.3, p_ref=p_ref, alpha=1 / 3)
    p = 2 * p_ref
    v = O.speed_of_p(p)
    lam = 0.3 * 2 ** (1 / 3)
    assert O.dmumu(prm, 0.0, v, p)[2] == pytest.approx(v / (2 * lam), rel=1e-13)


@pytest.mark.parametrize("model", ["qlt", "paper", "iso"])
def test_pitch_angle_amplification_record(model):
    """The oracle's record of how much the pitch-angle map amplifies differences in mu
    (amp_log after one step = max(0, ln|d mu'/d mu|)) equals a central finite difference
    of its own one-step update with the same noise, on a uniform-B background (no
    focusing or adiabatic terms, so d mu'/d mu comes from D_mumu alone)."""
    from oracle import oracle as O
    from fte_inputs.configs import Params
    bg = O.analytic_background("uniform_b", [5.0])
    prm = Params(dmumu=model, lambda_par=0.05, q=5 / 3, H=0.05, eps=0.048, dt=30.0)
    p0 = 0.0103
    n = 256
    mus = np.linspace(0.03, 0.6, n)
    ids = np.arange(n, dtype=np.uint32)
    P = O.make_particles(n, 1.0, 0.0, 0.0, mus, p0, ids=ids)
    O.advance(bg, prm, P, 0, 1)
    h = 1e-6
    Pp = O.make_particles(n, 1.0, 0.0, 0.0, mus + h, p0, ids=ids)
    Pm = O.make_particles(n, 1.0, 0.0, 0.0, mus - h, p0, ids=ids)
    O.advance(bg, prm, Pp, 0, 1)
    O.advance(bg, prm, Pm, 0, 1)
    clean = (Pp["n_div"] < 0) & (Pm["n_div"] < 0) & (P["n_div"] < 0)    # no reflection or sign change
    jac = (Pp["mu"] - Pm["mu"]) / (2 * h)
    expect = np.maximum(0.0, np.log(np.abs(jac)))
    assert clean.sum() > 100
    assert np.allclose(P["amp_log"][clean], expect[clean], rtol=0, atol=2e-4)
    assert (P["amp_log"][clean] > 0).sum() > 10          # some steps do expand
    # a 100-fold amplification is recorded as the first such step, none here after one step
    assert np.all(P["n_sens"][clean] == -1) or model == "qlt"
