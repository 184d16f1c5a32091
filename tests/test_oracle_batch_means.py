"""Pins of the tally error estimate: batch means over particle-id classes.

The occupancy estimator adds w dt for every step a particle spends inside an
observer, so the consecutive steps of one particle are strongly correlated and
sqrt(sum (w dt)^2) / sum w dt understates the error of an observer total.  The
particles are independent, so the totals of the 32 classes id mod 32 are
independent estimates of 1/32 of the total, and sqrt(32 var(class totals)) is its
standard error (batch means).

* A particle resting inside an observer puts all its w dt into its own class,
  bin by bin.
* The class sums of every bin add up to the bin.
* Over 16 independent seeds of a diffusive workload the batch-means standard
  error predicts the seed-to-seed scatter of the total, while the per-step
  estimate falls short of it by more than a factor of 3.
"""
import math

import numpy as np
import pytest

from fte_inputs.configs import Observer, Params
from oracle import oracle as O

E0 = 0.1
P0 = math.sqrt(E0 / O.MC2 * (E0 / O.MC2 + 2))


def test_resting_particle_fills_its_own_class():
    bg = O.analytic_background("uniform_b", [5.0])
    obs = [Observer(kind="shell", r=1.0, dr=0.05, e_lo=0.05, e_hi=0.2, ne=2, t_lo=0.0, t_hi=1e4, nt=5)]
    P = O.make_particles(3, 1.0, 0.0, 0.0, 0.0, P0)
    P["id"] = [7, 39, 12]                       # classes 7, 7, 12
    P["w"] = [0.5, 2.0, 1.0]
    prm = Params(dmumu="iso", lambda_par=1e300, dt=10.0)
    T, _ = O.advance(bg, prm, P, 0, 100, tally=O.Tally(obs))
    expect = np.zeros(32)
    expect[7] = (0.5 + 2.0) * 10.0 * 100
    expect[12] = 1.0 * 10.0 * 100
    cls = T.classes(0)
    assert np.allclose(cls.reshape(-1, 32).sum(axis=0), expect, rtol=1e-12, atol=0)
    assert np.allclose(cls.sum(axis=-1), T.obs_view(0, T.S), rtol=1e-12, atol=0)


def test_batch_means_predicts_seed_to_seed_scatter():
    bg = O.analytic_background("uniform_b", [5.0])
    obs = [Observer(kind="shell", r=0.6, dr=0.02, e_lo=0.05, e_hi=0.2, ne=4, t_lo=0.0, t_hi=1.5e5, nt=30)]
    n, steps = 2000, 1500
    tot, bm, naive = [], [], []
    for seed in range(16):
        prm = Params(dmumu="qlt", lambda_par=0.05, q=5 / 3, H=0.05, dt=100.0, seed=seed)
        P = O.make_particles(n, 0.5, 0.0, 0.0, 0.0, P0)
        P["mu"] = (np.arange(n) + 0.5) / n * 2 - 1
        P["id"] = np.arange(n)
        T, _ = O.advance(bg, prm, P, 0, steps, tally=O.Tally(obs))
        c = T.classes(0).reshape(-1, 32).sum(axis=0)
        assert c.sum() == pytest.approx(T.S.sum(), rel=1e-10)
        tot.append(c.sum())
        bm.append(math.sqrt(32 * c.var(ddof=1)))
        naive.append(math.sqrt(T.S2.sum()))
    sd = np.std(tot, ddof=1)
    print(f"seed-to-seed sd {sd:.4e}, batch means {np.mean(bm):.4e}, per-step {np.mean(naive):.4e}")
    # 16 seeds fix the scatter to about 18 %: the band is about 2.5 of those either way
    assert 0.6 < np.mean(bm) / sd < 1.6
    assert np.mean(naive) / sd < 1.0 / 3.0
