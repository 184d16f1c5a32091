"""Parity at the full size of the benchmark workload, in the launch configuration
bench.py times: the synthetic CIR on the 512 x 60 x 180 grid with 24 hourly
snapshots (12.7 GB of cell records), 1e6 protons injected in the div V < 0 cells,
4 days of 10-s steps advanced in calls of up to 1024 steps with the particles
reordered every 64 steps and the warp-merged global tally.

The FP64 oracle advances a seeded sample of the particles one by one over the same
steps.  At every call boundary each sampled particle's state agrees within 1e-4
(position relative to r, mu, p relative) up to its first divergence event, the
parity protocol, or the first step at which the pitch-angle map has amplified an
earlier difference in mu more than 100-fold (under the quasi-linear D_mumu near
mu = 0, where the derivative of sqrt(D) grows as |mu|^(q-2): there FP32 and FP64
rounding grow apart by orders of magnitude within tens of steps); absorbed counts
and the weight ledger are checked over the whole population.  Call boundaries at 64, 256 and 512 steps add early comparisons: a
call of 1024 steps launches the same 64-step kernels as these shorter calls, and
the results do not depend on how the steps are split into calls (tested bitwise
elsewhere)."""
import dataclasses

import numpy as np
import pytest

from fte_inputs import configs
from fte_inputs.configs import SmoothObserver
from oracle import oracle as O

from _parity import trajectory_errors

pytestmark = pytest.mark.gpu

N_SAMPLE = 2048
BOUNDS = [64, 256, 512, 1024] + list(range(2048, 34560, 1024)) + [34560]


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
def cir_full():
    w = configs.cir_uniform_1e6()
    assert (w.grid.nr, w.grid.nth, w.grid.nph, w.grid.n_snap) == (512, 60, 180, 24)
    assert w.n_particles == 1_000_000 and w.n_steps == 34560
    w.params.sort_every = 64
    return w, configs.build_background(w)


@pytest.fixture(scope="module")
def full_run(cir_full):
    import torch
    from paper_2404_12164_gb300 import api
    w, f = cir_full
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    failed = api.fte_inject(pool, bg, w.inject, w.n_particles, tally, check_failed=False)
    rng = np.random.default_rng(20240418)
    sample = np.sort(rng.choice(w.n_particles, N_SAMPLE, replace=False))
    ws = api.Workspace()
    states = {}
    prev = 0
    for b in BOUNDS:
        api.fte_advance(pool, bg, w.params, tally, prev, b, ws)
        prev = b
        st = pool.state()
        states[b] = {k: v[sample] for k, v in st.items()}
    final = pool.state()
    lw, ln = api.fte_ledger(tally)
    torch.cuda.synchronize()
    del bg
    torch.cuda.empty_cache()

    obg = O.grid_background(w.grid, f)
    P, _ = O.inject(obg, w.inject, sample.astype(np.uint32))
    ostates = {}
    prev = 0
    for b in BOUNDS:
        O.advance(obg, w.params, P, prev, b)
        prev = b
        ostates[b] = P.copy()
    return dict(w=w, sample=sample, g=states, o=ostates, final=final, lw=lw, ln=ln, failed=failed)


def test_sampled_trajectories_match_oracle(full_run):
    g, o = full_run["g"], full_run["o"]
    assert np.array_equal(g[BOUNDS[0]]["id"], full_run["sample"].astype(np.uint32))
    total = 0
    # what the amplification reading (n_sens, 100-fold growth of a mu difference) removes beyond
    # the protocol's divergence events: (particle, boundary) pairs and whole trajectories
    pairs_proto = pairs_sens = 0
    traj_sens = np.zeros(len(full_run["sample"]), dtype=bool)
    for b in BOUNDS:
        injected = o[b]["status"] != 5
        proto, _ = trajectory_errors(g[b], o[b], b, sel=injected)
        ok, e = trajectory_errors(g[b], o[b], b, sel=injected, expanding=True)   # 5: not injected
        pairs_proto += int(proto.sum())
        pairs_sens += int((proto & ~ok).sum())
        traj_sens |= proto & ~ok
        total += int(ok.sum())
        if b <= 256:
            assert ok.sum() >= 500, f"only {ok.sum()} matched trajectories at step {b}"
        if ok.any():
            for k in ("pos", "mu", "p", "w"):
                assert e[k].max() <= 1e-4, (b, k, float(e[k].max()))
            assert e["status"].sum() == 0, (b, "status")
    print(f"{total} (particle, boundary) pairs compared over {len(BOUNDS)} boundaries")
    share_pairs = pairs_sens / max(pairs_proto, 1)
    share_traj = traj_sens.sum() / len(full_run["sample"])
    print(f"the amplification reading removes {pairs_sens} of {pairs_proto} pairs the protocol keeps "
          f"({share_pairs:.3f}) and touches {traj_sens.sum()} of {len(traj_sens)} sampled trajectories "
          f"({share_traj:.3f})")
    assert total >= 2000
    assert share_pairs < 0.25 and share_traj < 0.25


def test_full_population_ledger(full_run):
    """Exact counts and the FP64 weight ledger over all 1e6 particles after 4 days."""
    st, lw, ln = full_run["final"], full_run["lw"], full_run["ln"]
    n_inj = int(ln[0])
    assert n_inj + int(ln[5]) == full_run["w"].n_particles
    status = st["status"]
    alive = status == 0
    for code in (1, 2, 3, 4):            # absorbed at r_min, r_max, a theta face; non-finite
        assert int(ln[code]) == int((status == code).sum()), code
    assert int(alive.sum()) + sum(int(ln[c]) for c in (1, 2, 3, 4)) == n_inj
    w = st["w"].astype(np.float64)
    assert lw[0] == pytest.approx(w[status != 5].sum(), rel=1e-9)
    absorbed = sum(float(lw[c]) for c in (1, 2, 3, 4))
    assert absorbed + w[alive].sum() == pytest.approx(float(lw[0]), rel=1e-9)
    # alive particle-steps: more than a day's worth for every particle injected
    assert int(ln[6]) > 8640 * n_inj


def test_parker_full_config_all_particles():
    """The Parker-spiral workload at its full size (128 x 16 x 32 grid, 1e4 protons at
    100 keV from 0.1 au, quasi-linear D_mumu, 1 day of 10-s steps): every particle is
    recomputed by the oracle, states agree at the call boundaries up to the first
    divergence or 100-fold amplification, absorbed counts match, and the 1 au shell
    tally agrees within 3 sigma in every bin with enough events."""
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    w = configs.parker_1e4()
    assert (w.grid.nr, w.grid.nth, w.grid.nph, w.n_particles, w.n_steps) == (128, 16, 32, 10_000, 8640)
    f = configs.build_background(w)
    bounds = [64, 512, 1024, 2048, 4096, 8640]
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally)
    ws = api.Workspace()
    g, prev = {}, 0
    for b in bounds:
        api.fte_advance(pool, bg, w.params, tally, prev, b, ws)
        prev = b
        g[b] = pool.state()
    gS = api.fte_tally(tally, 0, A.FTE_TALLY_S)
    gS2 = api.fte_tally(tally, 0, A.FTE_TALLY_S2)
    lw, ln = api.fte_ledger(tally)
    torch.cuda.synchronize()

    obg = O.grid_background(w.grid, f)
    P, led = O.inject(obg, w.inject, np.arange(w.n_particles, dtype=np.uint32))
    T = O.Tally(w.observers)
    prev = 0
    total = 0
    for b in bounds:
        O.advance(obg, w.params, P, prev, b, tally=T, ledger=led)
        prev = b
        ok, e = trajectory_errors(g[b], P, b, expanding=True)
        total += int(ok.sum())
        if ok.any():
            for k in ("pos", "mu", "p"):
                assert e[k].max() <= 1e-4, (b, k, float(e[k].max()))
            assert e["status"].sum() == 0, (b, "status")
    assert total >= 10_000
    L = led.as_dict()
    for code in (0, 1, 2, 3, 4):
        # counts of whole trajectories: equal up to the few that diverged near a boundary
        assert abs(int(ln[code]) - int(L["n"][code])) <= max(3, 1e-3 * int(L["n"][code])), code
    oS, oS2 = T.obs_view(0, T.S), T.obs_view(0, T.S2)
    sigma = np.sqrt(gS2 + oS2)
    busy = oS2 > 0
    assert busy.sum() > 50
    assert np.all(np.abs(gS - oS)[busy] <= 3 * sigma[busy] + 1e-12 * np.abs(oS).max())


def test_amr_full_config():
    """The block-AMR workload at its full size (39,520 leaves of 16^3 cells, 2 snapshots,
    44 GB of padded FP32 leaf lattices, 1e7 protons, 1800 steps of 2 s) in the benchmark's
    launch configuration: exact counts and the FP64 weight ledger over all particles, and a
    seeded sample of 1024 particles recomputed by the oracle (which interpolates across leaf
    faces from the neighbours on each query, without the ghost layers) on a host copy of
    the lattices, compared as above at the call boundaries."""
    import torch
    from fte_inputs import amr
    from fte_inputs.grid import REC
    from paper_2404_12164_gb300 import api
    w = configs.cir_amr_1e7()
    assert w.n_particles == 10_000_000 and w.n_steps == 1800
    w.params.sort_every = 64
    spec = w.grid
    leaves = amr.build_leaves(spec, amr.divv_refiner_batched(spec, w.amr_divv, device="cuda"))
    assert len(leaves) == 39_520
    bg = api.AmrBackground(spec, leaves)
    P = spec.bsize + 2
    view = bg.dev.view(spec.n_snap, len(leaves), P, P, P, REC)
    view.zero_()
    amr.fields_batched(spec, leaves, device="cuda", out=view)
    api.fte_amr_prepare(bg)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally, check_failed=False)
    rng = np.random.default_rng(20240419)
    sample = np.sort(rng.choice(w.n_particles, 1024, replace=False))
    bounds = [64, 256, 512, 1024, 1800]
    ws = api.Workspace()
    g, prev = {}, 0
    for b in bounds:
        api.fte_advance(pool, bg, w.params, tally, prev, b, ws)
        prev = b
        st = pool.state()
        g[b] = {k: v[sample] for k, v in st.items()}
    lw, ln = api.fte_ledger(tally)
    torch.cuda.synchronize()
    status = st["status"]
    n_inj = int(ln[0])
    assert n_inj + int(ln[5]) == w.n_particles
    for code in (1, 2, 3, 4):
        assert int(ln[code]) == int((status == code).sum()), code
    alive = status == 0
    assert int(alive.sum()) + sum(int(ln[c]) for c in (1, 2, 3, 4)) == n_inj
    wts = st["w"].astype(np.float64)
    absorbed = sum(float(lw[c]) for c in (1, 2, 3, 4))
    assert absorbed + wts[alive].sum() == pytest.approx(float(lw[0]), rel=1e-9)
    assert 0.5 * n_inj * w.n_steps < int(ln[6]) <= n_inj * w.n_steps
    del st, pool, tally, ws
    fields = view.cpu().numpy()              # the lattices on the host (ghost values ignored)
    del view, bg
    torch.cuda.empty_cache()

    obg = O.amr_background(spec, leaves, fields)
    Po, _ = O.inject(obg, w.inject, sample.astype(np.uint32))
    total, prev = 0, 0
    for b in bounds:
        O.advance(obg, w.params, Po, prev, b)
        prev = b
        ok, e = trajectory_errors(g[b], Po, b, sel=Po["status"] != 5, expanding=True)
        total += int(ok.sum())
        if b <= 256:
            assert ok.sum() >= 300, f"only {ok.sum()} matched trajectories at step {b}"
        if ok.any():
            for k in ("pos", "mu", "p", "w"):
                assert e[k].max() <= 1e-4, (b, k, float(e[k].max()))
            assert e["status"].sum() == 0, (b, "status")
    print(f"AMR: {total} (particle, boundary) pairs compared")


def test_ensemble_full_config_sampled(cir_full):
    """The 64-set ensemble at its full size (2e7 protons on the full CIR grid, 2160 steps)
    through the ensemble kernel in its default launch configuration: 8 seeded sets, 128
    particles each, recomputed by the oracle with their set's parameters and Philox key."""
    import torch
    from paper_2404_12164_gb300 import api
    _, f = cir_full
    w = configs.cir_ensemble_64()
    assert w.n_particles == 20_000_000 and len(w.sets) == 64
    w.params.sort_every = 64
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(w.observers, n_sets=64)
    api.fte_tally_reset(tally)
    api.fte_inject_batched(pool, bg, w.sets, tally)
    rng = np.random.default_rng(20240420)
    chosen = np.sort(rng.choice(64, 8, replace=False))
    starts = np.concatenate([[0], np.cumsum([s.count for s in w.sets])])
    picks = {int(k): np.sort(rng.choice(w.sets[k].count, 128, replace=False)) for k in chosen}
    index = np.concatenate([starts[k] + picks[k] for k in picks])
    bounds = [64, 256, 1024, 2160]
    ws = api.Workspace()
    g, prev = {}, 0
    for b in bounds:
        api.fte_advance_batched(pool, bg, w.params, w.sets, tally, prev, b, ws)
        prev = b
        st = pool.state()
        g[b] = {key: v[index] for key, v in st.items()}
    torch.cuda.synchronize()
    del pool, tally, ws, bg
    torch.cuda.empty_cache()
    obg = O.grid_background(w.grid, f)
    total, pos = 0, 0
    for k, ids in picks.items():
        s = w.sets[k]
        prm = dataclasses.replace(w.params, lambda_par=s.lambda_par, q=s.q, H=s.H, eps=s.eps, seed=s.seed,
                                  set_id=s.set_id)
        P, _ = O.inject(obg, s.inject, ids.astype(np.uint32))
        prev = 0
        for b in bounds:
            O.advance(obg, prm, P, prev, b)
            prev = b
            gb = {key: v[pos:pos + len(ids)] for key, v in g[b].items()}
            ok, e = trajectory_errors(gb, P, b, sel=P["status"] != 5, expanding=True)
            total += int(ok.sum())
            if ok.any():
                for key in ("pos", "mu", "p", "w"):
                    assert e[key].max() <= 1e-4, (k, b, key, float(e[key].max()))
                assert e["status"].sum() == 0, (k, b, "status")
        pos += len(ids)
    print(f"ensemble: {total} (particle, boundary) pairs compared")
    assert total >= 1000


def test_adjoint_full_grid_and_population(cir_full):
    """The adjoint on the full CIR grid with 1e6 E^-3 protons and the benchmark's launch
    configuration (checkpoints every 256 steps, reordering every 64), over one 256-step
    segment with the observable centred in it: on a seeded sample of 512 particles, J_i
    equals the oracle's and the per-particle gradients equal the FP64 oracle's estimate of
    the same form (pathwise, with the steps whose pitch-angle Gaussian reaches mu = 0 in
    score form; same noise and held values) on paths whose GPU and oracle end states agree,
    without a 100-fold amplification of the pitch-angle map or a decision within rounding of
    the score window's edge."""
    import torch
    from paper_2404_12164_gb300 import api
    w, f = cir_full
    inj = dataclasses.replace(w.inject, energy="powerlaw", e1=0.05, e2=5.0, gamma=3.0)
    prm = dataclasses.replace(w.params, sort_every=64)
    obs = SmoothObserver(r_o=1.5, sigma_r=0.2, e_c=0.1, sigma_lnE=0.7, t_c=1280.0, sigma_t=1000.0)
    n, steps = w.n_particles, 256
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(n)
    tally = api.Tally([])
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, inj, n, tally, id_base=0, check_failed=False)
    adj = api.Adjoint(bg, prm, obs, 0, steps, 256)
    J = adj.forward(pool)
    _, pp = adj.reverse(pool, inj, per_particle=True)
    torch.cuda.synchronize()
    pp = pp.cpu().numpy()
    st = pool.state()
    assert float(J) == pytest.approx(pp[:, 0].astype(np.float64).sum(), rel=1e-5)
    del pool, tally, adj, bg
    torch.cuda.empty_cache()

    rng = np.random.default_rng(20240421)
    sample = np.sort(rng.choice(n, 512, replace=False))
    obg = O.grid_background(w.grid, f)
    P, _ = O.inject(obg, inj, sample.astype(np.uint32))
    names = ("lambda_par", "q", "H")
    Jo, Go, fl = O.observe_lr(obg, prm, P, 0, steps, obs, 4.0, names)
    same = (fl == 0) & (P["n_sens"] < 0) & (P["status"] != 5) & (st["status"][sample] == P["status"])
    for key in ("x", "y", "z", "mu"):
        same &= np.abs(st[key][sample].astype(np.float64) - P[key]) <= 1e-4
    same &= np.abs(st["p"][sample].astype(np.float64) - P["p"]) <= 1e-4 * P["p"]
    print(f"{same.sum()} of 512 sampled trajectories agree end to end")
    assert same.sum() >= 100
    g = pp[sample]
    scale = np.abs(Jo).max()
    assert np.all(np.abs(g[same, 0] - Jo[same]) <= 1e-4 * np.abs(Jo[same]) + 1e-6 * scale)
    for col, name in ((1, "lambda_par"), (2, "q"), (3, "H")):
        ref = Go[name]
        gs = np.abs(ref[same]).max()
        err = np.abs(g[same, col] - ref[same]) / (np.abs(ref[same]) + 1e-3 * gs)
        print(f"d/d{name}: median rel err {np.median(err):.2e}, 95% {np.percentile(err, 95):.2e}")
        assert np.median(err) < 1e-3, name
        assert np.percentile(err, 95) < 1e-2, name