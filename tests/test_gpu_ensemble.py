"""Ensembles of parameter sets on the GPU (batched form of the transport of
Sec. 2.1: independent runs with their own lambda_par, q, H, Philox key and
injection energy, advanced in the same launches).

* every set's trajectories agree with the single-set kernel run on that set
  alone to FP32 rounding (the two kernels are compiled separately, so the last
  bit of a step may differ; trajectories then separate only where a rounding
  difference is amplified), for both tally layouts and both block sizes, and
  the tallies agree within 3 sigma;
* every set agrees with the FP64 oracle run on that set alone (per trajectory
  to 1e-4, tallies within 3 sigma, ledger conserved);
* the autotuner advances the run exactly as a fixed configuration does;
* a CUDA graph of inject + advance replays to the eager result;
* bad ensembles are refused.
"""
import dataclasses
import math

import numpy as np
import pytest

from fte_inputs import configs
from fte_inputs.configs import Observer
from oracle import oracle as O
from tests._parity import trajectory_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import build
    build.build()
    from oracle import build as ob
    ob.build()


@pytest.fixture(scope="module")
def cir_small():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_snap=3)
    w.grid.periodic = False
    w.params.sort_every = 32
    return w, configs.build_background(w)


def _sets(w, counts, rng_seed=7):
    sets = configs.ensemble_sets(len(counts), total=sum(counts), base_inject=w.inject, rng_seed=rng_seed)
    return [dataclasses.replace(s, count=int(c)) for s, c in zip(sets, counts)]


def _obs(t_hi):
    return [Observer(kind="shell", r=1.5, dr=0.05, e_lo=0.005, e_hi=1.0, ne=12, t_lo=0.0, t_hi=t_hi, nt=10),
            Observer(kind="box", r=1.2, dr=0.05, th=math.pi / 2, dth=0.1, ph=4.0, dph=0.5,
                     e_lo=0.005, e_hi=1.0, ne=8, t_lo=0.0, t_hi=t_hi, nt=5)]


def _batched(w, f, sets, obs, chunks, config=None):
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    n = sum(s.count for s in sets)
    pool = api.Particles(n)
    tally = api.Tally(obs, n_sets=len(sets))
    api.fte_tally_reset(tally)
    api.fte_inject_batched(pool, bg, sets, tally)
    ws = api.Workspace()
    prev = 0
    for c in chunks:
        api.fte_advance_batched(pool, bg, w.params, sets, tally, prev, c, ws, config=config)
        prev = c
    state = pool.state()
    tallies = [[{k: api.fte_tally_set(tally, s, o, kind) for k, kind in
                 (("S", A.FTE_TALLY_S), ("S2", A.FTE_TALLY_S2), ("C", A.FTE_TALLY_C))}
                for o in range(len(obs))] for s in range(len(sets))]
    lw, ln = api.fte_ledger(tally)
    torch.cuda.synchronize()
    return dict(state=state, tallies=tallies, ledger_w=lw, ledger_n=ln)


def _single(w, f, s, obs, chunks):
    """One set alone through the single-set entry points."""
    from paper_2404_12164_gb300 import api, _abi as A
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(s.count)
    tally = api.Tally(obs)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, s.inject, s.count, tally, id_base=0)
    prm = dataclasses.replace(w.params, lambda_par=s.lambda_par, q=s.q, H=s.H, eps=s.eps, seed=s.seed,
                              set_id=s.set_id)
    ws = api.Workspace()
    prev = 0
    for c in chunks:
        api.fte_advance(pool, bg, prm, tally, prev, c, ws)
        prev = c
    tallies = [{k: api.fte_tally(tally, o, kind) for k, kind in
                (("S", A.FTE_TALLY_S), ("S2", A.FTE_TALLY_S2), ("C", A.FTE_TALLY_C))} for o in range(len(obs))]
    return dict(state=pool.state(), tallies=tallies)


def _slice(state, a, b):
    return {k: v[a:b] for k, v in state.items()}


COUNTS = [37, 1500, 513, 2048, 5, 700]


@pytest.mark.parametrize("config", [None,
                                    {"threads": 128, "steps_per_launch": 64, "tally_layout": "shared"},
                                    {"threads": 256, "steps_per_launch": 32, "tally_layout": "global"},
                                    {"threads": 128, "steps_per_launch": 128, "tally_layout": "global"}])
def test_batched_matches_single_set_runs(cir_small, config):
    w, f = cir_small
    sets = _sets(w, COUNTS)
    obs = _obs(3000.0)
    chunks = [40, 300]
    b = _batched(w, f, sets, obs, chunks, config)
    off = 0
    for k, s in enumerate(sets):
        one = _single(w, f, s, obs, chunks)
        got, ref = _slice(b["state"], off, off + s.count), one["state"]
        assert np.array_equal(got["id"], ref["id"]) and np.array_equal(got["w"], ref["w"])
        same = got["status"] == ref["status"]
        assert same.mean() >= 0.98, (k, same.mean())
        r = np.sqrt(ref["x"] ** 2 + ref["y"] ** 2 + ref["z"] ** 2)
        dpos = np.sqrt((got["x"] - ref["x"]) ** 2 + (got["y"] - ref["y"]) ** 2 + (got["z"] - ref["z"]) ** 2) / r
        dmu = np.abs(got["mu"] - ref["mu"])
        dp = np.abs(got["p"] - ref["p"]) / ref["p"]
        for name, d in (("pos", dpos), ("mu", dmu), ("p", dp)):
            d = d[same]
            assert np.median(d) <= 1e-6, (k, name, float(np.median(d)))
            assert np.mean(d <= 1e-4) >= 0.95, (k, name)
        for o in range(len(obs)):
            tb, ts = b["tallies"][k][o], one["tallies"][o]
            sig = np.sqrt(tb["S2"] + ts["S2"])
            assert np.all(np.abs(tb["S"] - ts["S"]) <= 3 * sig + 1e-9 * max(ts["S"].max(), 1e-30)), (k, o)
        off += s.count
    assert int(b["ledger_n"][0]) == sum(COUNTS)


def test_ensemble_configs_agree_bitwise(cir_small):
    """Every launch configuration of the ensemble kernel gives the same trajectories and counts."""
    w, f = cir_small
    sets = _sets(w, COUNTS)
    obs = _obs(3000.0)
    runs = [_batched(w, f, sets, obs, [300], cfg) for cfg in
            (None, {"threads": 128, "steps_per_launch": 64, "tally_layout": "shared"},
             {"threads": 256, "steps_per_launch": 100, "tally_layout": "global"})]
    for other in runs[1:]:
        for key in ("x", "y", "z", "mu", "p", "status"):
            assert np.array_equal(other["state"][key], runs[0]["state"][key]), key
        for k in range(len(sets)):
            for o in range(len(obs)):
                assert np.array_equal(other["tallies"][k][o]["C"], runs[0]["tallies"][k][o]["C"]), (k, o)


def test_batched_vs_oracle(cir_small):
    w, f = cir_small
    sets = _sets(w, [900, 2500, 1200], rng_seed=11)
    obs = _obs(3000.0)
    chunks = [300]
    b = _batched(w, f, sets, obs, chunks)
    obg = O.grid_background(w.grid, f)
    off = 0
    for k, s in enumerate(sets):
        prm = dataclasses.replace(w.params, lambda_par=s.lambda_par, q=s.q, H=s.H, eps=s.eps, seed=s.seed,
                                  set_id=s.set_id)
        P, led = O.inject(obg, s.inject, np.arange(s.count, dtype=np.uint32))
        T = O.Tally(obs)
        O.advance(obg, prm, P, 0, 300, tally=T, ledger=led)
        g = _slice(b["state"], off, off + s.count)
        ok, e = trajectory_errors(g, P, 300)
        assert ok.sum() >= 0.3 * s.count, (k, ok.sum())
        for key in ("pos", "mu", "p", "w"):
            assert e[key].max() <= 1e-4, (k, key, float(e[key].max()))
        assert e["status"].sum() == 0
        for o in range(len(obs)):
            tg = b["tallies"][k][o]
            So, S2o = T.obs_view(o, T.S), T.obs_view(o, T.S2)
            sig = np.sqrt(tg["S2"] + S2o)
            assert np.all(np.abs(tg["S"] - So) <= 3 * sig + 1e-9 * max(So.max(), 1e-30)), (k, o)
        off += s.count
    alive = b["state"]["status"] == 0
    total = b["state"]["w"][alive].astype(np.float64).sum() + b["ledger_w"][1:5].sum()
    assert total == pytest.approx(b["ledger_w"][0], rel=1e-12)


def test_autotune_advances_like_fixed_config(cir_small):
    from paper_2404_12164_gb300 import api
    w, f = cir_small
    sets = _sets(w, COUNTS)
    obs = _obs(20000.0)
    n_steps = 256 * 16 * 2 + 100      # every candidate twice, then a ragged remainder
    ref = _batched(w, f, sets, obs, [n_steps])
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(sum(COUNTS))
    tally = api.Tally(obs, n_sets=len(sets))
    api.fte_tally_reset(tally)
    api.fte_inject_batched(pool, bg, sets, tally)
    best, tried = api.fte_autotune_batched(pool, bg, w.params, sets, tally, 0, n_steps)
    got = pool.state()
    for key in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(got[key], ref["state"][key]), key
    assert len(tried) == 16 and all(r > 0 for _, r in tried)
    assert best in [c for c, _ in tried]
    for s in range(len(sets)):
        assert np.array_equal(api.fte_tally_set(tally, s, 0, 2), ref["tallies"][s][0]["C"])


def test_graph_replay_equals_eager(cir_small):
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    w, f = cir_small
    sets = _sets(w, COUNTS)
    obs = _obs(3000.0)
    ref = _batched(w, f, sets, obs, [200])
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    n = sum(COUNTS)
    pool = api.Particles(n)
    tally = api.Tally(obs, n_sets=len(sets))
    ws = api.Workspace()
    ws.ensure(api.fte_workspace_bytes_batched(bg, tally, n, 200))
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = api.Graph()
    with torch.cuda.stream(side):
        with g.capture(side):
            api.fte_tally_reset(tally, stream=side)
            api.fte_inject_batched(pool, bg, sets, tally, stream=side)
            api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, 200, ws, stream=side)
        for rep in range(2):
            g.launch(side)
            side.synchronize()
            st = pool.state()
            for key in ("x", "y", "z", "mu", "p", "status"):
                assert np.array_equal(st[key], ref["state"][key]), (rep, key)
            for s in range(len(sets)):
                assert np.array_equal(api.fte_tally_set(tally, s, 0, A.FTE_TALLY_C, stream=side),
                                      ref["tallies"][s][0]["C"]), (rep, s)


def test_bad_ensembles_refused(cir_small):
    from paper_2404_12164_gb300 import api, _abi as A
    w, f = cir_small
    sets = _sets(w, [100, 200])
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(300)
    big = [Observer(kind="shell", r=1.5, dr=0.05, e_lo=0.01, e_hi=1.0, ne=16, t_lo=0.0, t_hi=1e4, nt=600)]
    tally = api.Tally(big, n_sets=2)
    api.fte_tally_reset(tally)
    api.fte_inject_batched(pool, bg, sets, tally)
    # counts that do not add up to the pool
    bad = [dataclasses.replace(sets[0], count=99), sets[1]]
    with pytest.raises(A.FteError) as e:
        api.fte_advance_batched(pool, bg, w.params, bad, tally, 0, 10)
    assert e.value.status == A.FTE_EINVAL
    # 2 x 9600 bins do not fit the shared layout
    with pytest.raises(A.FteError) as e:
        api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, 10,
                                config={"threads": 256, "steps_per_launch": 32, "tally_layout": "shared"})
    assert e.value.status == A.FTE_ENOTSUP
    # the global layout takes them; a tally with fewer sets than the ensemble is refused
    api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, 10)
    small = api.Tally(big, n_sets=1)
    with pytest.raises(A.FteError) as e:
        api.fte_advance_batched(pool, bg, w.params, sets, small, 10, 20)
    assert e.value.status == A.FTE_EINVAL
    with pytest.raises(A.FteError) as e:
        api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, 10,
                                config={"threads": 64, "steps_per_launch": 32, "tally_layout": "global"})
    assert e.value.status == A.FTE_EINVAL
