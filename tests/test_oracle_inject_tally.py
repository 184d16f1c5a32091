"""Pins of the oracle's injection (Sec. 2.3, Eq. 7) and occupancy tallies (Figs. 5-8).

Eq. 7: j(r, E) = C delta(E - E0) r^-2 over the region where div V < 0, realised
by distributing particles uniformly in volume over that region with weight
1/r^2.  The tallies give the differential intensity j = v n / (4 pi) per unit
energy, which for a homogeneous isotropic population equals v n / (4 pi)
exactly; that pins the observer volume and the normalisation.
"""
import math

import numpy as np
import pytest
from scipy import stats

from fte_inputs import backgrounds, configs
from fte_inputs.configs import InjectSpec, Observer, Params
from fte_inputs.grid import GridSpec, cell_centres
from oracle import oracle as O

DEG = math.pi / 180


def _sph(P):
    r = np.sqrt(P["x"] ** 2 + P["y"] ** 2 + P["z"] ** 2)
    th = np.arctan2(np.hypot(P["x"], P["y"]), P["z"])
    ph = np.mod(np.arctan2(P["y"], P["x"]), 2 * math.pi)
    return r, th, ph


def _energy(P):
    g = np.sqrt(1 + P["p"] ** 2)
    return O.MC2 * P["p"] ** 2 / (g + 1)


def test_point_injection_isotropic_mono():
    bg = O.analytic_background("uniform_b", [5.0])
    spec = InjectSpec(region="point", r=0.1, th=90 * DEG, ph=0.0, e0=0.1, seed=0)
    P, led = O.inject(bg, spec, np.arange(20000))
    assert np.allclose(P["x"], 0.1) and np.allclose(P["y"], 0.0, atol=1e-17)
    assert np.allclose(P["z"], 0.0, atol=1e-15)
    assert stats.kstest(P["mu"], "uniform", args=(-1, 2)).pvalue > 0.01
    assert np.allclose(_energy(P), 0.1, rtol=1e-13)
    assert np.all(P["w"] == 1.0) and led.as_dict()["n"][0] == 20000


def test_box_volume_uniform_and_weights():
    bg = O.analytic_background("uniform_b", [5.0])
    spec = InjectSpec(region="box", r1=1.0, r2=2.0, th1=60 * DEG, th2=100 * DEG, ph1=1.0,
                      ph2=2.5, weight="r-2", seed=4)
    P, led = O.inject(bg, spec, np.arange(20000))
    r, th, ph = _sph(P)
    # r^3 uniform, cos(theta) uniform, phi uniform
    assert stats.kstest((r ** 3 - 1) / 7, "uniform").pvalue > 0.01
    c = (np.cos(th) - math.cos(60 * DEG)) / (math.cos(100 * DEG) - math.cos(60 * DEG))
    assert stats.kstest(c, "uniform").pvalue > 0.01
    assert stats.kstest((ph - 1.0) / 1.5, "uniform").pvalue > 0.01
    assert P["w"] == pytest.approx(1 / r ** 2, rel=1e-12)
    assert led.as_dict()["w"][0] == pytest.approx(P["w"].sum(), rel=1e-12)


def test_spiral_band_volume_uniform():
    """A box whose longitude range bounds the spiral phase phi_hat = phi + k (r - r_b)
    (the one-CIR region criterion of Sec. 2.3): r^3, cos(theta) and phi_hat are uniform, so
    the band is filled uniformly in volume, and at fixed r the longitudes lie on the
    sheared interval."""
    bg = O.analytic_background("uniform_b", [5.0])
    k, rb = 0.8, 0.1
    spec = InjectSpec(region="box", r1=0.12, r2=2.0, th1=88 * DEG, th2=92 * DEG, ph1=4.5, ph2=4.9,
                      spiral=k, spiral_rb=rb, weight="r-2", seed=6)
    P, led = O.inject(bg, spec, np.arange(20000))
    r, th, ph = _sph(P)
    assert stats.kstest((r ** 3 - 0.12 ** 3) / (8 - 0.12 ** 3), "uniform").pvalue > 0.01
    c = (np.cos(th) - math.cos(88 * DEG)) / (math.cos(92 * DEG) - math.cos(88 * DEG))
    assert stats.kstest(c, "uniform").pvalue > 0.01
    phat = np.mod(ph + k * (r - rb), 2 * math.pi)
    assert phat.min() >= 4.5 - 1e-12 and phat.max() <= 4.9 + 1e-12
    assert stats.kstest((phat - 4.5) / 0.4, "uniform").pvalue > 0.01
    # the longitudes themselves are not confined to [ph1, ph2]: the band winds with r
    assert np.mod(ph[r > 1.5], 2 * math.pi).max() < 4.5 - k * (1.5 - rb) + 0.4 + 1e-9
    assert P["w"] == pytest.approx(1 / r ** 2, rel=1e-12)


def test_power_law_energy():
    bg = O.analytic_background("uniform_b", [5.0])
    spec = InjectSpec(region="point", energy="powerlaw", e1=0.05, e2=5.0, gamma=3.0, seed=9)
    P, _ = O.inject(bg, spec, np.arange(20000))
    E = _energy(P)
    assert E.min() >= 0.05 * (1 - 1e-12) and E.max() <= 5.0 * (1 + 1e-12)
    cdf = lambda e: (0.05 ** -2 - e ** -2) / (0.05 ** -2 - 5.0 ** -2)
    assert stats.kstest(E, cdf).pvalue > 0.01


def test_divv_rejection_region():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=60, nph=90, n_snap=1)
    f = configs.build_background(w)
    g = w.grid
    bg = O.grid_background(g, f)
    P, led = O.inject(bg, w.inject, np.arange(4000))
    assert np.all(P["status"] == O.ALIVE)
    r, th, ph = _sph(P)
    assert np.all((r >= 1.0 - 1e-12) & (r <= 2.0 + 1e-12))
    assert np.all((th >= 88 * DEG - 1e-12) & (th <= 92 * DEG + 1e-12))
    assert np.all((ph >= math.pi - 1e-12) & (ph <= 2 * math.pi + 1e-12))
    # every particle sits in a cell whose stored div V is negative
    i = np.floor((r - g.r_min) / ((g.r_max - g.r_min) / g.nr)).astype(int)
    j = np.floor((th - g.th_min) / ((g.th_max - g.th_min) / g.nth)).astype(int)
    k = np.floor(ph / (2 * math.pi / g.nph)).astype(int) % g.nph
    rec = f[0, k, j, i]
    tr = (rec[:, 6] + rec[:, 10]).astype(np.float32) + rec[:, 14]
    ok = (tr < 0) | (P["flags"] & 1).astype(bool)
    assert ok.all()
    assert P["w"] == pytest.approx(1 / r ** 2, rel=1e-12)


def test_injection_failure_is_ledgered():
    g = GridSpec(nr=16, nth=8, nph=16, n_snap=1)
    f = backgrounds.parker(g)           # div V > 0 everywhere
    bg = O.grid_background(g, f)
    spec = InjectSpec(region="box", r1=0.5, r2=1.0, th1=80 * DEG, th2=100 * DEG, divv_max=0.0,
                      max_tries=16)
    P, led = O.inject(bg, spec, np.arange(50))
    assert np.all(P["status"] == O.INJ_FAIL) and np.all(P["w"] == 0)
    L = led.as_dict()
    assert L["n"][5] == 50 and L["n"][0] == 0


@pytest.mark.parametrize("kind", ["shell", "box", "ring"])
def test_intensity_of_homogeneous_isotropic_population(kind):
    """n particles per au^3 with energies uniform in one bin: j = v n / (4 pi dE)."""
    bg = O.analytic_background("uniform_b", [5.0])
    rng = np.random.default_rng(0)
    N = 200_000
    L = 2.0
    P = O.make_particles(N)
    P["x"], P["y"], P["z"] = (rng.uniform(-L, L, N) for _ in range(3))
    P["mu"] = rng.uniform(-1, 1, N)
    ob = Observer(kind=kind, r=1.0, dr=0.2, th=90 * DEG, dth=20 * DEG, ph=0.5, dph=30 * DEG,
                  e_lo=0.1, e_hi=0.2, ne=1, t_lo=0.0, t_hi=1.0, nt=1)
    e = 0.1 * 2.0 ** rng.uniform(0, 1, N)           # energies inside the single bin
    T_ = e / O.MC2
    P["p"] = np.sqrt(T_ * (T_ + 2))
    prm = Params(dmumu="iso", lambda_par=1e300, dt=1.0)
    T = O.Tally([ob])
    O.advance(bg, prm, P, 0, 1, tally=T)
    n = N / (2 * L) ** 3                              # per au^3
    J = T.intensity(0)[0, 0]
    # the tally evaluates v at the geometric bin centre: compare with the mean v in the bin
    ec = math.sqrt(0.1 * 0.2)
    vc = O.speed_of_p(math.sqrt(ec / O.MC2 * (ec / O.MC2 + 2)))
    expect = vc * n / (4 * math.pi * 0.1)
    inside = T.C.sum()
    assert J == pytest.approx(expect, rel=4 / math.sqrt(inside))


def test_time_bin_edges_exact():
    """Step times on a bin edge fall in the upper bin: floor((t - t_lo) nt / (t_hi - t_lo))."""
    bg = O.analytic_background("uniform_b", [5.0])
    prm = Params(dmumu="iso", lambda_par=1e300, dt=10.0)
    P = O.make_particles(1, 1.0, 0, 0, 0.0, 0.0146)
    ob = Observer(kind="shell", r=1.0, dr=0.01, e_lo=0.01, e_hi=1.0, ne=16, t_lo=0.0,
                  t_hi=86400.0, nt=144)
    T = O.Tally([ob])
    O.advance(bg, prm, P, 0, 121, tally=T)            # t = 0 .. 1200 s, bins of 600 s
    C = T.obs_view(0, T.C).sum(axis=0)
    assert C[0] == 60 and C[1] == 60 and C[2] == 1
