"""Pins of the oracle's gradient of the smooth observable in the hybrid pathwise /
score (likelihood-ratio) form, or_observe_lr.

The Euler-Maruyama pitch-angle step of Sec. 2.1 draws mu' from a Gaussian of mean
m = mu + (mudot + dD/dmu) dt and width s = sqrt(2 D dt), reflected at +-1.  Eq. 5's
dD/dmu jumps at mu = 0 and the quasi-linear one is singular there (floored), so the
map mu -> mu' is discontinuous at mu = 0 and the derivative of a realised path
misses part of dE[J]/dtheta.  The oracle's estimator takes every step whose mean
lies within `window` widths of a value landing at mu = 0 in the score form (mu'
held, its transition density differentiated) and the others pathwise.

* or_mu_logpdf is the density of the reflected Gaussian: it integrates to 1 over
  [-1, 1] and equals the plain Gaussian away from the walls.
* On a four-step chain in a uniform field (V = 0, so m = mu + dD/dmu dt and the
  position moves by mu v dt) the observable J depends on the normals of the first
  two steps only; E[J](theta) is computed by Gauss-Legendre quadrature over them,
  split at every value where the first step lands at mu = 0 or at a wall, and its
  derivative by central differences.  The mean of the oracle's estimator over 1e5
  particles must match it within 4 standard errors, for Eq. 5, the quasi-linear
  form (one case where the mean passes mu = -1 and reflection lands near 0) and the
  isotropic form, while the pathwise derivative (window 0) misses it by more than
  10 standard errors for every parameter of Eq. 5 and the quasi-linear form.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

from fte_inputs.configs import Params, SmoothObserver
from oracle import oracle as O

E0 = 0.1
P0 = math.sqrt(E0 / O.MC2 * (E0 / O.MC2 + 2))
V0 = O.speed_of_p(P0)
DT = 100.0
Z0 = 0.5


@pytest.mark.parametrize("m,s", [(0.0, 0.05), (0.97, 0.05), (-1.0, 0.2), (0.4, 0.3), (1.6, 0.4)])
def test_mu_logpdf_is_the_reflected_gaussian(m, s):
    c = 1.0 / math.sqrt(2 * math.pi)
    tot = integrate.quad(lambda u: c * math.exp(O.mu_logpdf(u, m, s)), -1.0, 1.0, epsabs=1e-13, epsrel=1e-12,
                         points=[max(-1.0, min(1.0, m))], limit=200)[0]
    # the mass of y ~ N(m, s^2) inside [-3, 3], which one reflection maps into [-1, 1]
    inside = 0.5 * (math.erf((3 - m) / (s * math.sqrt(2))) - math.erf((-3 - m) / (s * math.sqrt(2))))
    assert tot == pytest.approx(inside, abs=1e-10)
    # where both images (2 - u, -2 - u) lie more than 30 widths from m the density is the Gaussian's
    for u in np.linspace(max(-1.0, m - 3 * s), min(1.0, m + 3 * s), 7):
        if abs(2 - u - m) > 30 * s and abs(-2 - u - m) > 30 * s:
            z = (u - m) / s
            assert O.mu_logpdf(u, m, s) == pytest.approx(-0.5 * z * z - math.log(s), abs=1e-12)


def _setup(prm, mu0):
    vdt = V0 * DT
    ob = SmoothObserver(r_o=Z0 + vdt, sigma_r=0.7 * vdt, e_c=E0, sigma_lnE=1.0, t_c=3 * DT, sigma_t=0.15 * DT)
    return ob, vdt


def _ms(prm, mu):
    D, dD, _ = O.dmumu(prm, mu, V0, P0)
    return mu + dD * DT, math.sqrt(2 * D * DT)


def _reflect(y):
    y = np.where(y > 1, 2 - y, y)
    y = np.where(y < -1, -2 - y, y)
    return np.clip(y, -1, 1)


def _expectation(prm, mu0):
    """E[J] over the four start-of-step states z_0..z_3 by quadrature over the first two normals."""
    ob, vdt = _setup(prm, mu0)

    def K(z, t):
        return (np.exp(-0.5 * ((z - ob.r_o) / ob.sigma_r) ** 2) * np.exp(-0.5 * ((t - ob.t_c) / ob.sigma_t) ** 2))

    m0, s0 = _ms(prm, mu0)
    # y0 = m0 + s0 z lands at mu = 0 for y0 in {0, 2, -2} and reaches a wall or the clamp at +-1, +-3
    cuts = sorted(c for c in ((v - m0) / s0 for v in (0.0, 2.0, -2.0, 1.0, -1.0, 3.0, -3.0)) if -14 < c < 14)
    edges = [-14.0] + cuts + [14.0]
    xo, wo = np.polynomial.legendre.leggauss(240)
    xi, wi = np.polynomial.legendre.leggauss(400)
    z1 = 14 * xi
    w1 = 14 * wi * np.exp(-0.5 * z1 * z1) / math.sqrt(2 * math.pi)
    total = 0.0
    for a, b in zip(edges[:-1], edges[1:]):
        z0 = 0.5 * (b - a) * xo + 0.5 * (b + a)
        w0 = 0.5 * (b - a) * wo * np.exp(-0.5 * z0 * z0) / math.sqrt(2 * math.pi)
        mu1 = _reflect(m0 + s0 * z0)
        for k in range(len(z0)):
            m1, s1 = _ms(prm, float(mu1[k]))
            mu2 = _reflect(m1 + s1 * z1)
            za = Z0 + mu0 * vdt
            zb = za + mu1[k] * vdt
            zc = zb + mu2 * vdt
            J = DT * (K(Z0, 0.0) + K(za, DT) + K(zb, 2 * DT) + K(zc, 3 * DT))
            total += w0[k] * np.sum(w1 * J)
    return total


def _estimate(prm, mu0, window, name, n=100_000):
    ob, _ = _setup(prm, mu0)
    bg = O.analytic_background("uniform_b", [5.0])
    P = O.make_particles(n, 0.0, 0.0, Z0, mu0, P0)
    P["id"] = np.arange(n)
    J, G, fl = O.observe_lr(bg, prm, P, 0, 4, ob, window, (name,))
    g = G[name][(fl & 6) == 0]
    assert len(g) > 0.99 * n
    return g.mean(), g.std() / math.sqrt(len(g)), J.mean()


CASES = [
    ("paper", Params(dmumu="paper", lambda_par=0.02, eps=0.048, dt=DT), 0.01, ("lambda_par", "eps"), True),
    ("qlt", Params(dmumu="qlt", lambda_par=0.05, q=5 / 3, H=0.05, dt=DT), 0.03, ("lambda_par", "q", "H"), True),
    ("qlt_reflected", Params(dmumu="qlt", lambda_par=0.01, q=5 / 3, H=0.05, dt=DT), -0.003, ("lambda_par",), False),
    ("iso", Params(dmumu="iso", lambda_par=0.02, dt=DT), 0.01, ("lambda_par",), False),
]


@pytest.mark.parametrize("case,prm,mu0,names,pathwise_biased", CASES, ids=[c[0] for c in CASES])
def test_score_gradient_matches_exact_derivative(case, prm, mu0, names, pathwise_biased):
    EJ = _expectation(prm, mu0)
    for name in names:
        th = getattr(prm, name)
        h = 1e-4 * th
        exact = (_expectation(dataclasses.replace(prm, **{name: th + h}), mu0)
                 - _expectation(dataclasses.replace(prm, **{name: th - h}), mu0)) / (2 * h)
        g, se, Jm = _estimate(prm, mu0, 4.0, name)
        assert Jm == pytest.approx(EJ, rel=5e-3)
        print(f"{case} d/d{name}: exact {exact:.6e}, window 4 {g:.6e} +- {se:.2e}")
        assert abs(g - exact) < 4 * se + 1e-6 * abs(exact), name
        g0, se0, _ = _estimate(prm, mu0, 0.0, name)
        print(f"{case} d/d{name}: pathwise {g0:.6e} +- {se0:.2e} ({(g0 - exact) / se0:+.1f} sigma)")
        if case == "iso":
            assert abs(g0 - exact) < 4 * se0, name
        elif pathwise_biased:
            assert abs(g0 - exact) > 10 * se0, name
