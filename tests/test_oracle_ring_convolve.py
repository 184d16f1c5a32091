"""Pins of the longitudinal-profile (ring) observer and of the Green's-function
convolution (Sec. 2.3: all particles are injected at t = 0; a time-independent
source follows by convolving that Green's-function solution with the source's
time profile; Figs. 5-7 show longitudinal intensity profiles at fixed r).

* a homogeneous isotropic population gives j = v n / (4 pi dE) in every
  longitude bin of a ring (the bin volume and the time normalisation);
* the longitude bin of a particle is floor(phi nt / 2 pi);
* the convolution reproduces the source for a one-bin Green's function,
  a cumulative sum (numpy) for a constant source, the closed-form geometric
  sum for an exponentially decaying Green's function, and is linear.
"""
import math

import numpy as np
import pytest

from fte_inputs.configs import Observer, Params
from oracle import oracle as O

DEG = math.pi / 180


def test_ring_intensity_per_longitude_bin():
    bg = O.analytic_background("uniform_b", [5.0])
    rng = np.random.default_rng(1)
    N = 400_000
    L = 1.3
    P = O.make_particles(N)
    P["x"], P["y"], P["z"] = (rng.uniform(-L, L, N) for _ in range(3))
    P["mu"] = rng.uniform(-1, 1, N)
    e = 0.1 * 2.0 ** rng.uniform(0, 1, N)
    T_ = e / O.MC2
    P["p"] = np.sqrt(T_ * (T_ + 2))
    nphi = 8
    ob = Observer(kind="ring", r=1.0, dr=0.2, th=90 * DEG, dth=20 * DEG, e_lo=0.1, e_hi=0.2, ne=1,
                  t_lo=0.0, t_hi=1.0, nt=nphi)
    prm = Params(dmumu="iso", lambda_par=1e300, dt=1.0)
    T = O.Tally([ob])
    O.advance(bg, prm, P, 0, 1, tally=T)
    n = N / (2 * L) ** 3
    ec = math.sqrt(0.1 * 0.2)
    vc = O.speed_of_p(math.sqrt(ec / O.MC2 * (ec / O.MC2 + 2)))
    expect = vc * n / (4 * math.pi * 0.1)
    J = T.intensity(0)[0]
    C = T.obs_view(0, T.C)[0].astype(float)
    assert np.all(C > 1000)
    for k in range(nphi):
        assert J[k] == pytest.approx(expect, rel=4 / math.sqrt(C[k]))


def test_ring_longitude_bins():
    """Particles at known longitudes land in bin floor(phi nt / 2 pi); outside the window, none."""
    bg = O.analytic_background("uniform_b", [5.0])
    phis = np.array([0.01, 0.5, 1.6, 3.0, 3.2, 4.8, 6.2])
    P = O.make_particles(len(phis))
    P["x"], P["y"], P["z"] = np.cos(phis), np.sin(phis), 0.0
    P["p"] = 0.0146
    ob = Observer(kind="ring", r=1.0, dr=0.01, th=90 * DEG, dth=1 * DEG, e_lo=0.01, e_hi=1.0, ne=4,
                  t_lo=0.0, t_hi=5.0, nt=12)
    prm = Params(dmumu="iso", lambda_par=1e300, dt=1.0)
    T = O.Tally([ob])
    O.advance(bg, prm, P.copy(), 0, 1, tally=T)
    C = T.obs_view(0, T.C).sum(axis=0)
    expect = np.bincount(np.floor(phis * 12 / (2 * math.pi)).astype(int), minlength=12)
    assert np.array_equal(C, expect)
    T2 = O.Tally([Observer(**{**ob.__dict__, "t_lo": 5.0, "t_hi": 10.0})])
    O.advance(bg, prm, P.copy(), 0, 1, tally=T2)
    assert T2.C.sum() == 0


def test_convolution_pins():
    rng = np.random.default_rng(2)
    ne, nt, dtb = 3, 12, 600.0
    src = rng.uniform(0.5, 2.0, nt)
    # one-bin Green's function: the output is the source (times the bin width)
    G = np.zeros((ne, nt))
    G[:, 0] = [1.0, 2.0, 3.0]
    out = O.convolve(G, dtb, src)
    assert np.allclose(out, dtb * np.outer([1.0, 2.0, 3.0], src), rtol=1e-14)
    # constant source: cumulative sum along time
    G = rng.uniform(0, 1, (ne, nt))
    assert np.allclose(O.convolve(G, dtb), dtb * np.cumsum(G, axis=1), rtol=1e-13)
    # exponentially decaying Green's function, constant source: geometric sum
    a = 0.7
    G = np.tile(a ** np.arange(nt), (ne, 1))
    k = np.arange(nt)
    assert np.allclose(O.convolve(G, dtb)[0], dtb * (1 - a ** (k + 1)) / (1 - a), rtol=1e-13)
    # linear in the Green's function and in the source
    G1, G2 = rng.uniform(0, 1, (2, ne, nt))
    s1, s2 = rng.uniform(0, 1, (2, nt))
    assert np.allclose(O.convolve(2 * G1 + G2, dtb, s1), 2 * O.convolve(G1, dtb, s1) + O.convolve(G2, dtb, s1))
    assert np.allclose(O.convolve(G1, dtb, s1 - 3 * s2), O.convolve(G1, dtb, s1) - 3 * O.convolve(G1, dtb, s2))
