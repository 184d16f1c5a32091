"""Helpers shared by the GPU parity tests: run one workload through the C ABI and
through the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

from oracle import oracle as O


def gpu_run(w, fields, n_steps, chunks=None, params=None, observers=None, n_particles=None):
    """Inject + advance through the library; returns (pool state dicts at each
    checkpoint, tally arrays per observer, ledger)."""
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    n = n_particles or w.n_particles
    obs = w.observers if observers is None else observers
    bg = api.Background(w.grid)
    api.fte_load_background(bg, fields)
    pool = api.Particles(n)
    tally = api.Tally(obs)
    api.fte_tally_reset(tally)
    failed = api.fte_inject(pool, bg, w.inject, n, tally)
    states = {0: pool.state()}
    ws = api.Workspace()
    prev = 0
    for c in (chunks or [n_steps]):
        api.fte_advance(pool, bg, params or w.params, tally, prev, c, ws)
        prev = c
        states[c] = pool.state()
    tallies = []
    for o in range(len(obs)):
        tallies.append({k: api.fte_tally(tally, o, kind) for k, kind in
                        (("S", A.FTE_TALLY_S), ("S2", A.FTE_TALLY_S2), ("C", A.FTE_TALLY_C),
                         ("J", A.FTE_TALLY_INTENSITY))})
    lw, ln = api.fte_ledger(tally)
    # per observer: the bins by particle-id class [ne, nt, 32] and the class totals [32]
    bins = [tally.classes(o) for o in range(len(obs))]
    cls = [b.reshape(-1, b.shape[-1]).sum(axis=0) for b in bins]
    torch.cuda.synchronize()
    return dict(states=states, tallies=tallies, ledger_w=lw, ledger_n=ln, failed=failed, S_class=cls, classes=bins)


def oracle_run(w, fields, n_steps, chunks=None, params=None, observers=None, n_particles=None,
               ids=None, shock_divv=0.0):
    n = n_particles or w.n_particles
    obs = w.observers if observers is None else observers
    bg = O.grid_background(w.grid, fields)
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, dtype=np.uint32)
    P, led = O.inject(bg, w.inject, ids)
    states = {0: P.copy()}
    T = O.Tally(obs)
    prev = 0
    for c in (chunks or [n_steps]):
        O.advance(bg, params or w.params, P, prev, c, tally=T, ledger=led, shock_divv=shock_divv)
        prev = c
        states[c] = P.copy()
    tallies = []
    for o in range(len(obs)):
        tallies.append(dict(S=T.obs_view(o, T.S), S2=T.obs_view(o, T.S2), C=T.obs_view(o, T.C),
                            A=T.obs_view(o, T.A), J=T.intensity(o)))
    L = led.as_dict()
    bins = [T.classes(o) for o in range(len(obs))]
    cls = [b.reshape(-1, 32).sum(axis=0) for b in bins]
    return dict(states=states, tallies=tallies, ledger_w=L["w"], ledger_n=L["n"], S_class=cls, classes=bins)


def trajectory_errors(g, o, step, sel=None, expanding=False):
    """Per-particle errors at checkpoint `step` for particles the oracle saw no
    divergence event for before `step` and that both sides have alive or absorbed
    identically.  expanding=True also leaves out particles whose pitch-angle map
    had amplified an earlier difference in mu more than 100-fold before `step`
    (the oracle's n_sens).  Returns (mask, dict of error arrays)."""
    ok = ((o["n_div"] < 0) | (o["n_div"] >= step)) & ((o["flags"] & 1) == 0)
    if expanding:
        ok &= (o["n_sens"] < 0) | (o["n_sens"] >= step)
    if sel is not None:
        ok &= sel
    r_o = np.sqrt(o["x"] ** 2 + o["y"] ** 2 + o["z"] ** 2)
    dx = np.sqrt((g["x"] - o["x"]) ** 2 + (g["y"] - o["y"]) ** 2 + (g["z"] - o["z"]) ** 2)
    errs = dict(
        pos=dx / r_o,
        mu=np.abs(g["mu"] - o["mu"]),
        p=np.abs(g["p"] - o["p"]) / np.abs(o["p"]),
        w=np.abs(g["w"] - o["w"]) / np.maximum(np.abs(o["w"]), 1e-30),
        status=(g["status"] != o["status"]).astype(float),
    )
    return ok, {k: v[ok] for k, v in errs.items()}
