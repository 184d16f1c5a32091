"""Longitudinal-profile (ring) observers and the Green's-function convolution on
the GPU against the FP64 oracle (Sec. 2.3; the output form of Figs. 5-8).

* deterministic trajectories (no scattering): ring counts equal the oracle's
  except events the oracle flags within 1e-4 of an edge (which may move one
  bin in energy or longitude);
* scattered trajectories: every ring bin within 3 sigma, intensities the same
  function of S on both sides;
* fte_tally_convolve equals the oracle's plain convolution of the same
  Green's-function tally, for a constant and for a time-varying source.
"""
import math

import numpy as np
import pytest

from fte_inputs import configs
from fte_inputs.configs import InjectSpec, Observer, Params
from oracle import oracle as O
from tests._parity import gpu_run, oracle_run

pytestmark = pytest.mark.gpu
DEG = math.pi / 180


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()


def _spread(a):
    """Ambiguity of each bin and of its neighbours along both axes (diagonals included;
    longitude wraps)."""
    s = a.copy()
    s[1:, :] += a[:-1, :]
    s[:-1, :] += a[1:, :]
    return s + np.roll(s, 1, axis=1) + np.roll(s, -1, axis=1)


def test_ring_counts_exact_for_deterministic_trajectories():
    w = configs.scaled(configs.parker_1e4(), n_particles=6000)
    w.inject = InjectSpec(region="box", r1=0.8, r2=1.2, th1=80 * DEG, th2=100 * DEG, ph1=0.0,
                          ph2=2 * math.pi, energy="powerlaw", e1=0.02, e2=0.8, gamma=1.5, seed=9)
    w.params = Params(dmumu="iso", lambda_par=1e30, dt=10.0)
    obs = [Observer(kind="ring", r=1.0, dr=0.05, th=90 * DEG, dth=5 * DEG, e_lo=0.01, e_hi=1.0, ne=8,
                    t_lo=0.0, t_hi=20000.0, nt=36),
           Observer(kind="ring", r=1.1, dr=0.05, th=92 * DEG, dth=4 * DEG, e_lo=0.01, e_hi=1.0, ne=4,
                    t_lo=5000.0, t_hi=15000.0, nt=72)]
    f = configs.build_background(w)
    g = gpu_run(w, f, 2000, observers=obs)
    o = oracle_run(w, f, 2000, observers=obs)
    for k in range(len(obs)):
        Cg = g["tallies"][k]["C"].astype(np.int64)
        Co = o["tallies"][k]["C"].astype(np.int64)
        A = o["tallies"][k]["A"].astype(np.int64)
        assert Co.sum() > 1000
        amb = _spread(A)
        assert np.array_equal(Cg[amb == 0], Co[amb == 0])
        assert np.all(np.abs(Cg - Co) <= amb)
        assert np.abs(Cg - Co).sum() <= 2 * A.sum()


def test_ring_tallies_within_three_sigma():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_particles=6000, n_snap=3)
    w.grid.periodic = False
    obs = [Observer(kind="ring", r=1.3, dr=0.1, th=90 * DEG, dth=4 * DEG, e_lo=0.01, e_hi=1.0, ne=6,
                    t_lo=0.0, t_hi=6000.0, nt=24)]
    f = configs.build_background(w)
    g = gpu_run(w, f, 600, observers=obs)
    o = oracle_run(w, f, 600, observers=obs)
    tg, to = g["tallies"][0], o["tallies"][0]
    assert to["C"].sum() > 5000
    sig = np.sqrt(tg["S2"] + to["S2"])
    assert np.all(np.abs(tg["S"] - to["S"]) <= 3 * sig + 1e-9 * to["S"].max())
    nz = to["S"] > 0
    assert np.allclose(tg["J"][nz] / tg["S"][nz], to["J"][nz] / to["S"][nz], rtol=1e-12)


def test_convolution_equals_oracle():
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    w = configs.scaled(configs.parker_1e4(), n_particles=4000)
    ob = Observer(kind="shell", r=0.5, dr=0.05, e_lo=0.01, e_hi=1.0, ne=10, t_lo=0.0, t_hi=30000.0, nt=40)
    f = configs.build_background(w)
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(w.n_particles)
    tally = api.Tally([ob])
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally)
    api.fte_advance(pool, bg, w.params, tally, 0, 3000)
    S = api.fte_tally(tally, 0, A.FTE_TALLY_S)
    J = api.fte_tally(tally, 0, A.FTE_TALLY_INTENSITY)
    assert S.sum() > 0
    dtb = (ob.t_hi - ob.t_lo) / ob.nt
    rng = np.random.default_rng(3)
    src = rng.uniform(0.0, 2.0, ob.nt)
    src_dev = torch.tensor(src, dtype=torch.float64, device="cuda")
    for kind, G in ((A.FTE_TALLY_S, S), (A.FTE_TALLY_INTENSITY, J)):
        for s_host, s_dev in ((None, None), (src, src_dev)):
            got = api.fte_tally_convolve(tally, 0, kind, s_dev)
            ref = O.convolve(G, dtb, s_host)
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-300), (kind, s_host is None)
    # a constant source accumulates the Green's function: the last bin is the steady state so far
    ss = api.fte_tally_convolve(tally, 0, A.FTE_TALLY_S)
    assert np.allclose(ss[:, -1], dtb * S.sum(axis=1), rtol=1e-12)
    # ring observers bin longitude, not time: refused
    ring = api.Tally([Observer(kind="ring", r=1.0, dr=0.1, ne=2, nt=8)])
    api.fte_tally_reset(ring)
    with pytest.raises(A.FteError) as e:
        api.fte_tally_convolve(ring, 0)
    assert e.value.status == A.FTE_EINVAL
