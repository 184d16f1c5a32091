"""The pair record layout (each record holds a cell and its upper r-neighbour) on
the GPU: it stores the same values as the cell layout, so every kernel that reads
the background gives bit-identical results on it.

* the FP32 pair image equals the cell records rearranged (exact, byte work), and
  a 16-bit pair image holds the same 16-bit values as the 16-bit cell image;
* trajectories, tallies and injection (which reads the stored div V) are bit for
  bit those of the cell layout, for FP32, BF16 and FP16, uniform and block AMR;
* the ensemble and adjoint kernels give the same results on both layouts.
"""
import math

import numpy as np
import pytest

from fte_inputs import amr, configs
from fte_inputs.configs import InjectSpec, Params, SmoothObserver

pytestmark = pytest.mark.gpu
DEG = math.pi / 180


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def cir_small():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=96, nth=24, nph=72, n_snap=3, n_particles=5000)
    w.grid.periodic = False
    w.params.sort_every = 32
    return w, configs.build_background(w)


def _backgrounds(w, f, dtype):
    from paper_2404_12164_gb300 import api
    b32 = api.Background(w.grid)
    api.fte_load_background(b32, f)
    cell = b32
    if dtype != "f32":
        cell = api.Background(w.grid, dtype=dtype)
        api.fte_quantize_background(cell, b32)
    pair = api.Background(w.grid, dtype=dtype, layout="pair")
    api.fte_quantize_background(pair, b32)
    return b32, cell, pair


def _run(bg, w, n, steps):
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    pool = api.Particles(n)
    tally = api.Tally(w.observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, n, tally)
    inj = pool.state()
    api.fte_advance(pool, bg, w.params, tally, 0, steps)
    torch.cuda.synchronize()
    return inj, pool.state(), api.fte_tally(tally, 0, A.FTE_TALLY_C), api.fte_tally(tally, 0, A.FTE_TALLY_S)


def _same(a, b, s_rtol=1e-6):
    for sa, sb in ((a[0], b[0]), (a[1], b[1])):
        for k in ("x", "y", "z", "mu", "p", "w", "status"):
            assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a[2], b[2])
    assert np.allclose(a[3], b[3], rtol=s_rtol, atol=0)      # FP32 partial sums in another order


def test_pair_images(cir_small):
    from paper_2404_12164_gb300 import api
    w, f = cir_small
    nr = w.grid.nr
    b32, _, p32 = _backgrounds(w, f, "f32")
    img = api.device_bytes(p32).view(np.float32).reshape(-1, 40)
    cells = f.reshape(-1, f.shape[-1])[:, :18]
    assert np.array_equal(img[:, :18], cells)
    last = (np.arange(len(cells)) % nr) == nr - 1
    assert np.array_equal(img[~last, 18:36], cells[1:][~last[:-1]])
    assert np.all(img[last, 18:] == 0) and np.all(img[:, 36:] == 0)
    for dt in ("bf16", "f16"):
        _, hc, hp = _backgrounds(w, f, dt)
        ci = api.device_bytes(hc)
        pi = api.device_bytes(hp)
        assert np.array_equal(ci[:128], pi[:128])                      # the same scale header
        cv = ci[128:].view(np.uint16).reshape(-1, 32)[:, :18]
        pv = pi[128:].view(np.uint16).reshape(-1, 48)
        assert np.array_equal(pv[:, :18], cv)
        assert np.array_equal(pv[~last, 18:36], cv[1:][~last[:-1]])
        assert np.all(pv[last, 18:] == 0) and np.all(pv[:, 36:] == 0)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_pair_layout_equals_cell_layout(cir_small, dtype):
    w, f = cir_small
    _, cell, pair = _backgrounds(w, f, dtype)
    _same(_run(pair, w, w.n_particles, 400), _run(cell, w, w.n_particles, 400))


def test_pair_layout_on_amr():
    from paper_2404_12164_gb300 import api
    spec = amr.AmrSpec(nbr=4, nbt=2, nbp=4, bsize=8, levels=3, n_snap=2, periodic=False, dt_snap=3600.0)
    leaves = amr.build_leaves(spec, amr.divv_refiner(spec, threshold=8e-6, r_from=0.9))
    f = amr.fields(spec, leaves)
    w = configs.cir_uniform_1e6()
    w.inject = InjectSpec(region="box", r1=1.0, r2=1.8, th1=88 * DEG, th2=92 * DEG, ph1=math.pi, ph2=2 * math.pi,
                          divv_max=0.0, energy="mono", e0=0.05, weight="r-2", seed=4)
    w.params = Params(dmumu="qlt", lambda_par=0.1, dt=10.0, sort_every=32)
    cell = api.AmrBackground(spec, leaves)
    api.fte_load_background(cell, f)
    api.fte_amr_prepare(cell)
    for dt in ("f32", "bf16"):
        pair = api.AmrBackground(spec, leaves, dtype=dt, share=cell, layout="pair")
        api.fte_quantize_background(pair, cell)
        ref = cell
        if dt != "f32":
            ref = api.AmrBackground(spec, leaves, dtype=dt, share=cell)
            api.fte_quantize_background(ref, cell)
        _same(_run(pair, w, 3000, 300), _run(ref, w, 3000, 300))


def test_ensemble_and_adjoint_on_pair_layout(cir_small):
    import torch
    from paper_2404_12164_gb300 import api
    w, f = cir_small
    _, cell, pair = _backgrounds(w, f, "f32")
    sets = configs.ensemble_sets(3, total=3000, base_inject=w.inject, rng_seed=5)
    out = []
    for bg in (cell, pair):
        pool = api.Particles(3000)
        tally = api.Tally(w.observers, n_sets=3)
        api.fte_tally_reset(tally)
        api.fte_inject_batched(pool, bg, sets, tally)
        api.fte_advance_batched(pool, bg, w.params, sets, tally, 0, 200)
        out.append(pool.state())
    for k in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(out[0][k], out[1][k]), k
    obs = SmoothObserver(r_o=1.3, sigma_r=0.1, e_c=0.05, sigma_lnE=0.5, t_c=1000.0, sigma_t=800.0)
    prm = Params(dmumu="iso", lambda_par=0.1, dt=10.0)
    inj = InjectSpec(region="box", r1=1.0, r2=1.5, th1=86 * DEG, th2=94 * DEG, ph1=math.pi, ph2=2 * math.pi,
                     energy="powerlaw", e1=0.05, e2=0.5, gamma=3.0, seed=6)
    res = []
    for bg in (cell, pair):
        pool = api.Particles(2000)
        tally = api.Tally([])
        api.fte_tally_reset(tally)
        api.fte_inject(pool, bg, inj, 2000, tally)
        adj = api.Adjoint(bg, prm, obs, 0, 200, 50)
        adj.forward(pool)
        g, pp = adj.reverse(pool, inj, per_particle=True)
        torch.cuda.synchronize()
        res.append(pp.cpu().numpy())
    assert np.array_equal(res[0], res[1])
