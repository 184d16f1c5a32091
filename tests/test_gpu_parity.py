"""GPU (C ABI) vs FP64 oracle parity on identical seeded inputs.

Tolerances (FP32 device arithmetic against the FP64 oracle):
* per trajectory, up to the first divergence event the oracle records
  (reflection, mu sign change, a boundary or acceptance decision within
  rounding): position within 1e-4 of r, mu within 1e-4, p within 1e-4 relative;
* injection: mu bit-exact (one Philox draw, exact FP32 uniform), positions 1e-5;
* tally counts: exact for deterministic trajectories except events the oracle
  flags within 1e-4 of a bin or observer edge;
* tally sums: every bin within 3 sigma (sigma^2 = S2_gpu + S2_oracle).
"""
import math

import numpy as np
import pytest

from fte_inputs import configs
from fte_inputs.configs import InjectSpec, Observer, Params
from tests._parity import gpu_run, oracle_run, trajectory_errors

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


@pytest.fixture(scope="module")
def parker():
    w = configs.scaled(configs.parker_1e4(), n_particles=6000)
    return w, configs.build_background(w)


@pytest.fixture(scope="module")
def cir_small():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_particles=4000)
    return w, configs.build_background(w)


def _assert_traj(g, o, step, tol=1e-4, min_matched=200):
    ok, e = trajectory_errors(g, o, step)
    assert ok.sum() >= min_matched, f"only {ok.sum()} matched trajectories at step {step}"
    for k in ("pos", "mu", "p", "w"):
        assert e[k].max() <= tol, (step, k, float(e[k].max()), float(np.percentile(e[k], 99)))
    assert e["status"].sum() == 0, (step, "status")


def test_injection_point_mu_bitexact(parker):
    w, f = parker
    g = gpu_run(w, f, 0, chunks=[])["states"][0]
    o = oracle_run(w, f, 0, chunks=[])["states"][0]
    assert np.array_equal(g["mu"], o["mu"].astype(np.float32))
    assert np.array_equal(g["id"], o["id"])
    assert np.allclose(g["p"], o["p"], rtol=1e-6)
    assert np.allclose(g["x"], o["x"], rtol=1e-6, atol=1e-7)
    assert np.abs(g["y"]).max() < 1e-7 and np.abs(g["z"]).max() < 1e-7
    assert np.all(g["status"] == 0) and np.all(g["w"] == 1.0)


def test_injection_box_divv(cir_small):
    w, f = cir_small
    gr = gpu_run(w, f, 0, chunks=[])
    orr = oracle_run(w, f, 0, chunks=[])
    g, o = gr["states"][0], orr["states"][0]
    assert gr["failed"] == 0
    clean = (o["flags"] & 1) == 0
    assert clean.mean() > 0.9
    r_o = np.sqrt(o["x"] ** 2 + o["y"] ** 2 + o["z"] ** 2)
    dx = np.sqrt((g["x"] - o["x"]) ** 2 + (g["y"] - o["y"]) ** 2 + (g["z"] - o["z"]) ** 2) / r_o
    assert dx[clean].max() < 1e-5
    assert np.abs(g["w"] - o["w"])[clean].max() / o["w"].max() < 1e-5
    assert np.array_equal(g["mu"], o["mu"].astype(np.float32))
    assert np.array_equal(g["status"], o["status"].astype(np.uint8))
    # injected weight in the ledger
    assert gr["ledger_w"][0] == pytest.approx(g["w"].astype(np.float64).sum(), rel=1e-12)
    assert gr["ledger_w"][0] == pytest.approx(orr["ledger_w"][0], rel=1e-5)


def test_injection_spiral_band():
    """The block-AMR workload's injection (a band of spiral phase from 0.12 to 2 au) on a
    uniform grid of the same wind: positions to 1e-5, mu bit-exact, weights and ledger."""
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_snap=2, n_particles=20000)
    w.inject = configs.cir_amr_1e7().inject
    f = configs.build_background(w)
    gr = gpu_run(w, f, 0, chunks=[])
    orr = oracle_run(w, f, 0, chunks=[])
    g, o = gr["states"][0], orr["states"][0]
    assert gr["failed"] == 0
    r_o = np.sqrt(o["x"] ** 2 + o["y"] ** 2 + o["z"] ** 2)
    dx = np.sqrt((g["x"] - o["x"]) ** 2 + (g["y"] - o["y"]) ** 2 + (g["z"] - o["z"]) ** 2) / r_o
    assert dx.max() < 1e-5
    assert np.abs(g["w"] - o["w"]).max() / o["w"].max() < 1e-5
    assert np.array_equal(g["mu"], o["mu"].astype(np.float32))
    assert gr["ledger_w"][0] == pytest.approx(orr["ledger_w"][0], rel=1e-5)
    assert r_o.min() < 0.2 and r_o.max() > 1.9


def test_trajectories_parker_qlt(parker):
    w, f = parker
    chunks = [1, 10, 60, 250, 700]
    g = gpu_run(w, f, 0, chunks=chunks)["states"]
    o = oracle_run(w, f, 0, chunks=chunks)["states"]
    for c in chunks:
        _assert_traj(g[c], o[c], c)


def test_trajectories_cir_time_interpolated(cir_small):
    w, f = cir_small
    chunks = [1, 37, 400, 800]          # crosses the first snapshot boundary (360 steps)
    g = gpu_run(w, f, 0, chunks=chunks)["states"]
    o = oracle_run(w, f, 0, chunks=chunks)["states"]
    for c in chunks:
        _assert_traj(g[c], o[c], c)


@pytest.mark.parametrize("model", ["paper", "iso"])
def test_trajectories_other_dmumu_log_grid(model):
    w = configs.scaled(configs.parker_1e4(), n_particles=3000)
    w.grid.radial = "log"
    w.params = Params(dmumu=model, lambda_par=0.3, dt=10.0, seed=7)
    f = configs.build_background(w)
    chunks = [5, 120, 400]
    g = gpu_run(w, f, 0, chunks=chunks)["states"]
    o = oracle_run(w, f, 0, chunks=chunks)["states"]
    for c in chunks:
        _assert_traj(g[c], o[c], c)


def test_trajectories_cross_field_diffusion(parker):
    w, f = parker
    prm = Params(dmumu="qlt", lambda_par=0.3, lambda_perp=3e-4, kappa_drift=1, dt=10.0, seed=3)
    chunks = [3, 100, 400]
    g = gpu_run(w, f, 0, chunks=chunks, params=prm)["states"]
    o = oracle_run(w, f, 0, chunks=chunks, params=prm)["states"]
    for c in chunks:
        _assert_traj(g[c], o[c], c)


def test_counts_exact_for_deterministic_trajectories():
    """No scattering (D = 0): trajectories never diverge, so every tally count must match
    except events the oracle flags within 1e-4 of an energy-bin or observer edge."""
    w = configs.scaled(configs.parker_1e4(), n_particles=4000)
    w.inject = InjectSpec(region="box", r1=0.8, r2=1.2, th1=80 * DEG, th2=100 * DEG, ph1=0.0,
                          ph2=2 * math.pi, energy="powerlaw", e1=0.02, e2=0.8, gamma=1.5, seed=5)
    w.params = Params(dmumu="iso", lambda_par=1e30, dt=10.0)
    obs = [Observer(kind="shell", r=1.0, dr=0.05, e_lo=0.01, e_hi=1.0, ne=16, t_lo=0.0,
                    t_hi=20000.0, nt=40),
           Observer(kind="box", r=1.1, dr=0.05, th=90 * DEG, dth=8 * DEG, ph=1.0, dph=20 * DEG,
                    e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=20000.0, nt=20)]
    f = configs.build_background(w)
    g = gpu_run(w, f, 2000, observers=obs)
    o = oracle_run(w, f, 2000, observers=obs)
    for k in range(len(obs)):
        Cg = g["tallies"][k]["C"].astype(np.int64)
        Co = o["tallies"][k]["C"].astype(np.int64)
        A = o["tallies"][k]["A"].astype(np.int64)
        assert Co.sum() > 1000
        amb = A.copy()
        amb[1:] += A[:-1]
        amb[:-1] += A[1:]
        assert np.all(np.abs(Cg - Co) <= amb), np.abs(Cg - Co).max()
        assert np.array_equal(Cg[amb == 0], Co[amb == 0])
        assert np.abs(Cg - Co).sum() <= 2 * A.sum()
        # observer totals by particle-id class: the same steps in the same classes (weights are
        # 1 here, so a class total is dt times its tallied steps), up to the ambiguous events
        cg, co = g["S_class"][k], o["S_class"][k]
        assert cg.sum() == pytest.approx(g["tallies"][k]["S"].sum(), rel=1e-6)
        assert np.abs(cg - co).sum() <= 2 * A.sum() * w.params.dt + 1e-6 * co.sum()


def test_tallies_within_three_sigma(parker):
    w, f = parker
    obs = [Observer(kind="shell", r=0.5, dr=0.05, e_lo=0.01, e_hi=1.0, ne=16, t_lo=0.0,
                    t_hi=30000.0, nt=30)]
    g = gpu_run(w, f, 3000, observers=obs)
    o = oracle_run(w, f, 3000, observers=obs)
    tg, to = g["tallies"][0], o["tallies"][0]
    assert to["C"].sum() > 10000
    sig = np.sqrt(tg["S2"] + to["S2"])
    assert np.all(np.abs(tg["S"] - to["S"]) <= 3 * sig + 1e-9 * to["S"].max())
    # intensity normalisation is the same function of S on both sides
    nz = to["S"] > 0
    assert np.allclose(tg["J"][nz] / tg["S"][nz], to["J"][nz] / to["S"][nz], rtol=1e-12)
    # total occupancy agrees to a few per cent of its own statistical error
    tot_sig = math.sqrt(tg["S2"].sum() + to["S2"].sum())
    assert abs(tg["S"].sum() - to["S"].sum()) < 3 * tot_sig
    # class totals (batch means): they add up to the total, and the two batch-means errors
    # of the total, from the same Philox streams, agree
    cg, co = g["S_class"][0], o["S_class"][0]
    assert cg.sum() == pytest.approx(tg["S"].sum(), rel=1e-6)
    bm_g = math.sqrt(32 * cg.var(ddof=1))
    bm_o = math.sqrt(32 * co.var(ddof=1))
    assert abs(cg.sum() - co.sum()) < 3 * math.hypot(bm_g, bm_o)
    assert 0.7 < bm_g / bm_o < 1.4


def test_ledger_conservation(cir_small):
    w, f = cir_small
    g = gpu_run(w, f, 1500)
    st = g["states"][1500]
    lw, ln = g["ledger_w"], g["ledger_n"]
    alive = st["status"] == 0
    assert int(ln[0]) == w.n_particles
    assert int(ln[0]) == alive.sum() + int(ln[1:5].sum())
    for k in (1, 2, 3):
        assert int(ln[k]) == (st["status"] == k).sum()
    total = st["w"][alive].astype(np.float64).sum() + lw[1:5].sum()
    assert total == pytest.approx(lw[0], rel=1e-12)
    assert 0 < int(ln[6]) <= w.n_particles * 1500


def test_chunking_is_bitwise_invariant(parker):
    w, f = parker
    a = gpu_run(w, f, 300, chunks=[300])["states"][300]
    b = gpu_run(w, f, 300, chunks=[17, 100, 300])["states"][300]
    for k in ("x", "y", "z", "mu", "p", "w", "status"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("n", [1, 31, 257, 1000])
def test_ragged_particle_counts(parker, n):
    w, f = parker
    g = gpu_run(w, f, 50, n_particles=n)["states"][50]
    o = oracle_run(w, f, 50, n_particles=n)["states"][50]
    ok, e = trajectory_errors(g, o, 50)
    assert ok.sum() >= 1 or n == 1
    for k in ("pos", "mu", "p"):
        assert (e[k].max() if e[k].size else 0) <= 1e-4


def test_empty_and_zero_step_calls(parker):
    import torch
    from paper_2404_12164_gb300 import api
    w, f = parker
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(16)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_advance(pool, bg, w.params, tally, 0, 100)       # empty pool
    assert api.fte_inject(pool, bg, w.inject, 0, tally) == 0
    api.fte_inject(pool, bg, w.inject, 16, tally)
    before = pool.state()
    api.fte_advance(pool, bg, w.params, tally, 5, 5)         # zero steps
    after = pool.state()
    for k in ("x", "mu", "p"):
        assert np.array_equal(before[k], after[k])
    lw, ln = api.fte_ledger(tally)
    assert int(ln[6]) == 0 and int(ln[0]) == 16
    torch.cuda.synchronize()


def test_failed_injection_reported():
    from paper_2404_12164_gb300 import api
    w = configs.scaled(configs.parker_1e4(), n_particles=64)
    w.inject = InjectSpec(region="box", r1=0.5, r2=1.0, th1=80 * DEG, th2=100 * DEG,
                          divv_max=0.0, max_tries=8)        # Parker: div V > 0 everywhere
    f = configs.build_background(w)
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(64)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    assert api.fte_inject(pool, bg, w.inject, 64, tally) == 64
    st = pool.state()
    assert np.all(st["status"] == 5) and np.all(st["w"] == 0)
    api.fte_advance(pool, bg, w.params, tally, 0, 10)        # nothing alive to advance
    lw, ln = api.fte_ledger(tally)
    assert int(ln[5]) == 64 and int(ln[0]) == 0 and int(ln[6]) == 0


def test_spatial_reordering_changes_nothing(cir_small):
    """Reordering the alive particles by cell (sort_every > 0) only changes which thread
    advances which particle: states, counts and the ledger are identical."""
    import dataclasses
    w, f = cir_small
    prm_sorted = dataclasses.replace(w.params, sort_every=64)
    a = gpu_run(w, f, 700, chunks=[300, 700])
    b = gpu_run(w, f, 700, chunks=[300, 700], params=prm_sorted)
    for c in (300, 700):
        for k in ("x", "y", "z", "mu", "p", "w", "status"):
            assert np.array_equal(a["states"][c][k], b["states"][c][k]), (c, k)
    assert np.array_equal(a["tallies"][0]["C"], b["tallies"][0]["C"])
    assert np.allclose(a["tallies"][0]["S"], b["tallies"][0]["S"], rtol=1e-5, atol=1e-12)
    assert np.array_equal(a["ledger_n"], b["ledger_n"])


def test_half_pools_and_block_compaction_change_nothing():
    """A reordered pool of more particles than the step kernel has resident threads runs as two
    halves on two streams, and each half (fewer particles than resident threads) launches on
    only the blocks that give each thread one particle: states, counts and the ledger equal those
    of the unordered run on one stream."""
    import dataclasses
    import torch
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_particles=120_000)
    f = configs.build_background(w)
    threads = torch.cuda.get_device_properties(0).multi_processor_count * 512
    assert threads <= w.n_particles < 2 * threads
    a = gpu_run(w, f, 300, params=dataclasses.replace(w.params, sort_every=0))
    b = gpu_run(w, f, 300, params=dataclasses.replace(w.params, sort_every=64))
    for k in ("x", "y", "z", "mu", "p", "w", "status"):
        assert np.array_equal(a["states"][300][k], b["states"][300][k]), k
    assert np.array_equal(a["tallies"][0]["C"], b["tallies"][0]["C"])
    assert np.allclose(a["tallies"][0]["S"], b["tallies"][0]["S"], rtol=1e-9, atol=1e-12)
    assert np.array_equal(a["ledger_n"], b["ledger_n"])
    assert int(a["ledger_n"][6]) > 0


def test_checkpoint_resume_is_bit_exact(tmp_path, parker):
    """A run saved to disk after 150 steps and resumed in a fresh pool ends where the
    uninterrupted run ends (every random number depends on (seed, set, step, id) only)."""
    from paper_2404_12164_gb300 import api
    w, f = parker
    full = gpu_run(w, f, 300, chunks=[300])["states"][300]
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally)
    api.fte_advance(pool, bg, w.params, tally, 0, 150)
    np.savez(tmp_path / "ckpt.npz", **pool.state())
    del pool
    saved = dict(np.load(tmp_path / "ckpt.npz"))
    resumed = api.Particles(w.n_particles)
    resumed.load_state(saved)
    api.fte_advance(resumed, bg, w.params, tally, 150, 300)
    st = resumed.state()
    for k in ("x", "y", "z", "mu", "p", "w", "id", "status"):
        assert np.array_equal(st[k], full[k]), k


def test_undersized_workspace_is_refused(parker):
    import ctypes as C
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    w, f = parker
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(100)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, 100, tally)
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")     # far below the partial histograms
    st = A.lib().fte_advance(C.byref(pool.c), C.byref(bg.c), C.byref(api.params_c(w.params)), C.byref(tally.c),
                             0, 50, C.c_void_p(buf.data_ptr()), buf.numel(), None)
    assert st == A.FTE_ENOMEM
    assert b"workspace" in A.lib().fte_last_error()


def test_tally_layouts_agree(cir_small):
    """Warp-merged FP64 atomics (the default) and per-block shared-memory histograms tally the
    same events: counts equal, sums to FP32 partial-sum rounding, trajectories identical."""
    import dataclasses
    w, f = cir_small
    obs = w.observers + [Observer(kind="shell", r=1.5, dr=0.05, e_lo=0.01, e_hi=10.0, ne=16, t_lo=0.0,
                                  t_hi=20000.0, nt=40)]
    g = gpu_run(w, f, 1200, observers=obs)
    s = gpu_run(w, f, 1200, observers=obs, params=dataclasses.replace(w.params, tally_layout="shared"))
    for k in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(g["states"][1200][k], s["states"][1200][k]), k
    for o in range(len(obs)):
        assert np.array_equal(g["tallies"][o]["C"], s["tallies"][o]["C"])
        Sg, Ss = g["tallies"][o]["S"], s["tallies"][o]["S"]
        assert np.allclose(Sg, Ss, rtol=1e-5, atol=1e-12 * max(Sg.max(), 1e-30))
    assert np.array_equal(g["ledger_n"], s["ledger_n"])


def test_maximum_observer_count(parker):
    """A tally with the maximum number of observers (8) of all four kinds: every
    observer's occupancy agrees with the oracle's within 3 sigma, and a ninth observer
    is refused."""
    from paper_2404_12164_gb300 import api
    w, f = parker
    from paper_2404_12164_gb300 import _abi as A
    assert A.FTE_MAX_OBS == 8
    obs = [Observer(kind="shell", r=r, dr=0.03, e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=20000.0, nt=10)
           for r in (0.2, 0.35, 0.5, 0.8)]
    obs += [Observer(kind="box", r=0.3, dr=0.05, th=math.pi / 2, dth=0.3, ph=0.3, dph=0.6,
                     e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=20000.0, nt=10),
            Observer(kind="box", r=0.6, dr=0.1, th=math.pi / 2, dth=0.3, ph=6.0, dph=0.6,
                     e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=20000.0, nt=10),
            Observer(kind="slab", r=0.3, dr=0.05, e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=20000.0, nt=10),
            Observer(kind="ring", r=0.4, dr=0.05, th=math.pi / 2, dth=0.2, e_lo=0.01, e_hi=1.0, ne=8,
                     t_lo=0.0, t_hi=20000.0, nt=12)]
    assert len(obs) == A.FTE_MAX_OBS
    g = gpu_run(w, f, 2000, observers=obs)
    o = oracle_run(w, f, 2000, observers=obs)
    busy = 0
    for k in range(len(obs)):
        tg, to = g["tallies"][k], o["tallies"][k]
        sig = np.sqrt(tg["S2"] + to["S2"])
        assert np.all(np.abs(tg["S"] - to["S"]) <= 3 * sig + 1e-9 * max(to["S"].max(), 1e-30)), k
        busy += int(to["C"].sum() > 100)
    assert busy >= 6
    with pytest.raises(ValueError):
        api.Tally(obs + [obs[0]])
