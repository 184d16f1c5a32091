"""Adjoint on the GPU against the FP64 oracle.

The observable J = sum_i w_i sum_n dt K(r_n, E_n, t_n) (Gaussians in r, ln E, t)
is a smooth function of each particle's path.  The gradient is pathwise (Philox
noise held) except at steps whose pitch-angle Gaussian reaches mu = 0, which
enter in the score form (mu' held, its transition density differentiated); with
the default window that is every such step of Eq. 5 and the quasi-linear form and
none of the isotropic form.  Checks:

* J per particle equals the oracle's (the forward pass is the transport);
* per-particle gradients equal the FP64 oracle's estimate of the same form
  (or_observe_lr: central differences of the density-reweighted observable with
  the same held values and noise) on particles whose GPU and oracle end states
  agree and whose gate decisions are not within rounding of the window's edge,
  for all three D_mumu forms;
* dJ/dgamma equals the finite difference of the likelihood-ratio weights of
  the injected energies (normalisation by numerical quadrature);
* for all three forms the total gradient agrees with central differences of the
  GPU forward pass with common random numbers within their statistical errors
  (batch means over 32 particle-id classes); the checkpoint interval changes
  nothing;
* torch.autograd through SmoothIntensity returns the adjoint gradient.
"""
import dataclasses
import math

import numpy as np
import pytest

import bench
from fte_inputs import configs
from fte_inputs.configs import InjectSpec, Params, SmoothObserver
from oracle import oracle as O

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
def cir_small():
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_snap=3)
    w.grid.periodic = False
    w.inject = InjectSpec(region="box", r1=1.0, r2=1.3, th1=86 * DEG, th2=94 * DEG, ph1=math.pi,
                          ph2=2 * math.pi, divv_max=None, energy="powerlaw", e1=0.05, e2=0.5, gamma=3.0,
                          weight="r-2", seed=3)
    return w, configs.build_background(w)


OBS = SmoothObserver(r_o=1.15, sigma_r=0.05, e_c=0.08, sigma_lnE=0.5, t_c=1500.0, sigma_t=1000.0)


def _gpu(w, f, prm, n, steps, K=64, per_particle=True, obs=OBS, dtype="f32"):
    import torch
    from paper_2404_12164_gb300 import api
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    if dtype != "f32":
        b32, bg = bg, api.Background(w.grid, dtype=dtype)
        api.fte_quantize_background(bg, b32)
    pool = api.Particles(n)
    tally = api.Tally([])
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, n, tally, id_base=0)
    adj = api.Adjoint(bg, prm, obs, 0, steps, K)
    J = adj.forward(pool)
    g, pp = adj.reverse(pool, w.inject, per_particle=True)
    torch.cuda.synchronize()
    return float(J), g.cpu().numpy(), pp.cpu().numpy(), pool.state()


def _oracle_J(w, f, prm, n, steps):
    bg = O.grid_background(w.grid, f)
    P, _ = O.inject(bg, w.inject, np.arange(n, dtype=np.uint32))
    J = O.observe(bg, prm, P, 0, steps, OBS)
    return J, P


MODELS = [
    ("qlt", Params(dmumu="qlt", lambda_par=0.1, q=5 / 3, H=0.05, dt=10.0), ("lambda_par", "q", "H")),
    ("paper", Params(dmumu="paper", lambda_par=0.1, eps=0.048, dt=10.0), ("lambda_par", "eps")),
    ("iso", Params(dmumu="iso", lambda_par=0.1, dt=10.0), ("lambda_par",)),
]
GI = {"lambda_par": 1, "q": 2, "H": 3, "eps": 4}
WINDOW = {"qlt": 4.0, "paper": 4.0, "iso": 0.0}      # the library's default window per form


def _batch_sigma(x, ids, nb=32):
    """Standard error of sum(x) from the sums over nb classes of particle id."""
    s = np.bincount(ids % nb, weights=x, minlength=nb)
    return math.sqrt(nb * s.var(ddof=1))


@pytest.mark.parametrize("name,prm,names", MODELS, ids=[m[0] for m in MODELS])
def test_gradients_match_oracle(cir_small, name, prm, names):
    w, f = cir_small
    n, steps = 4000, 200
    J, g, pp, st = _gpu(w, f, prm, n, steps)
    bg = O.grid_background(w.grid, f)
    P, _ = O.inject(bg, w.inject, np.arange(n, dtype=np.uint32))
    Jo, Go, fl = O.observe_lr(bg, prm, P, 0, steps, OBS, WINDOW[name], names)
    # trajectories that FP32 and FP64 computed alike: same status, end states within 1e-4, no
    # 100-fold amplification of mu differences by the pitch-angle map on the way, and no gate
    # decision, mu = 0 passage or end step within rounding of a decision
    same = (st["status"] == P["status"]) & (fl == 0) & (P["n_sens"] < 0)
    for key, tol in (("x", 1e-4), ("y", 1e-4), ("z", 1e-4), ("mu", 1e-4)):
        same &= np.abs(st[key].astype(np.float64) - P[key]) <= tol
    same &= np.abs(st["p"].astype(np.float64) - P["p"]) <= 1e-4 * P["p"]
    print(f"{name}: {same.sum()} of {n} trajectories agree end to end")
    assert same.sum() >= 0.5 * n
    # the forward observable, particle by particle
    scale = np.abs(Jo).max()
    assert np.all(np.abs(pp[same, 0] - Jo[same]) <= 1e-4 * np.abs(Jo[same]) + 1e-6 * scale)
    assert J == pytest.approx(pp[:, 0].astype(np.float64).sum(), rel=1e-5)
    for nm in names:
        ref = Go[nm]
        ga = pp[:, GI[nm]].astype(np.float64)
        gscale = np.abs(ref[same]).max()
        err = np.abs(ga[same] - ref[same]) / (np.abs(ref[same]) + 1e-3 * gscale)
        print(f"{name} d/d{nm}: median rel err {np.median(err):.2e}, 99% {np.percentile(err, 99):.2e}, "
              f"max {err.max():.2e}; total adjoint {g[GI[nm] - 1]:.6e}, oracle {ref.sum():.6e}")
        assert np.median(err) < 1e-3, nm
        assert np.percentile(err, 95) < 1e-2, nm


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_gradient_storage_error(cir_small, dtype):
    """Stated error of the gradients on a 16-bit background: the adjoint's totals on BF16 or
    FP16 storage against the oracle's estimate of the same form on the FP32 fields (same
    noise, so nearly the same paths), in units of the batch-means error of the per-particle
    differences, and relative."""
    w, f = cir_small
    name, prm, names = MODELS[0]
    n, steps = 4000, 200
    _, g, pp, _ = _gpu(w, f, prm, n, steps, dtype=dtype)
    bg = O.grid_background(w.grid, f)
    P, _ = O.inject(bg, w.inject, np.arange(n, dtype=np.uint32))
    Jo, Go, fl = O.observe_lr(bg, prm, P, 0, steps, OBS, WINDOW[name], names)
    ids = np.arange(n)
    dJ = pp[:, 0].astype(np.float64) - Jo
    print(f"{dtype} J: total {pp[:, 0].sum():.6e} vs oracle {Jo.sum():.6e} "
          f"(rel {dJ.sum() / Jo.sum():+.2e}, {dJ.sum() / _batch_sigma(dJ, ids):+.1f} sigma)")
    bound = bench.STORAGE_ERROR_COMMON["adjoint"]
    assert abs(dJ.sum()) <= bound["J_rel"] * abs(Jo.sum())
    for nm in names:
        d = pp[:, GI[nm]].astype(np.float64) - Go[nm]
        sd = _batch_sigma(d, ids)
        rel = d.sum() / abs(Go[nm].sum())
        print(f"{dtype} d/d{nm}: total {pp[:, GI[nm]].sum():.6e} vs oracle {Go[nm].sum():.6e} "
              f"(rel {rel:+.2e}, {d.sum() / sd:+.1f} sigma of the difference)")
        assert abs(d.sum()) <= bound["gradient_total_sigma"] * sd + bound["gradient_total_rel"] * abs(Go[nm].sum()), nm


def test_gamma_gradient_is_likelihood_ratio(cir_small):
    from scipy import integrate
    w, f = cir_small
    prm = MODELS[0][1]
    n, steps = 3000, 200
    _, g, pp, _ = _gpu(w, f, prm, n, steps)
    bg = O.grid_background(w.grid, f)
    P, _ = O.inject(bg, w.inject, np.arange(n, dtype=np.uint32))
    E0 = O.MC2 * P["p"] ** 2 / (np.sqrt(1 + P["p"] ** 2) + 1)
    e1, e2, gam = w.inject.e1, w.inject.e2, w.inject.gamma

    def pdf(gm):
        Z = integrate.quad(lambda e: e ** -gm, e1, e2, epsabs=0, epsrel=1e-13)[0]
        return E0 ** -gm / Z
    h = 1e-5
    lr = (pdf(gam + h) - pdf(gam - h)) / (2 * h) / pdf(gam)
    Ji = pp[:, 0].astype(np.float64)
    assert np.allclose(pp[:, 5], lr * Ji, rtol=2e-4, atol=1e-7 * np.abs(lr * Ji).max())
    assert g[4] == pytest.approx((lr * Ji).sum(), rel=1e-4)


@pytest.mark.parametrize("model", [0, 1, 2], ids=["qlt", "paper", "iso"])
def test_checkpoint_interval_changes_nothing(cir_small, model):
    w, f = cir_small
    name, prm, names = MODELS[model]
    J, g, _, _ = _gpu(w, f, prm, 5000, 300, K=64)
    J2, g2, _, _ = _gpu(w, f, prm, 5000, 300, K=7)
    J3, g3, _, _ = _gpu(w, f, prm, 5000, 300, K=1000)
    for Jx, gx in ((J2, g2), (J3, g3)):
        assert Jx == pytest.approx(J, rel=1e-12)
        assert np.allclose(gx, g, rtol=1e-5, atol=1e-9 * np.abs(g).max())


def test_spatial_ordering_changes_nothing(cir_small):
    """Each launch may take the particles in spatial order; every particle's J_i and
    gradients are the same."""
    w, f = cir_small
    prm = MODELS[0][1]
    _, g0, pp0, s0 = _gpu(w, f, prm, 5000, 300, K=32)
    _, g1, pp1, s1 = _gpu(w, f, dataclasses.replace(prm, sort_every=32), 5000, 300, K=32)
    assert np.array_equal(pp0, pp1)
    for key in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(s0[key], s1[key]), key
    assert np.allclose(g0, g1, rtol=1e-9, atol=0)


def test_half_pools_change_nothing(cir_small):
    """With reordering on, a pool of at least one wave of the forward kernel's threads runs
    both passes as two halves on two streams, each half with its own workspace region; every
    particle's end state, J_i and gradients equal those of the single pool in the original
    order (reordering off), bit for bit, and the totals agree to the order of their FP64 sums."""
    w, f = cir_small
    prm = MODELS[0][1]
    n = 1 << 18                       # more particles than resident forward-kernel threads
    J0, g0, pp0, s0 = _gpu(w, f, prm, n, 200, K=64)
    J1, g1, pp1, s1 = _gpu(w, f, dataclasses.replace(prm, sort_every=32), n, 200, K=64)
    assert np.array_equal(pp0, pp1)
    for key in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(s0[key], s1[key]), key
    assert J1 == pytest.approx(J0, rel=1e-12)
    assert np.allclose(g0, g1, rtol=1e-9, atol=0)
    assert (s1["status"] == 0).sum() > n // 2 and np.count_nonzero(pp1[:, 0]) > 1000


def test_graph_capture_of_both_passes(cir_small):
    """The injection, the forward and the reverse pass captured in one CUDA graph and replayed
    twice give the eager run's J and gradients.  The pool is large enough for two halves,
    which then go in turn on the capturing stream (no second stream inside a capture)."""
    import torch
    from paper_2404_12164_gb300 import api
    w, f = cir_small
    prm = dataclasses.replace(MODELS[0][1], sort_every=32)
    n, steps, K = 1 << 18, 200, 64
    J0, g0, _, _ = _gpu(w, f, prm, n, steps, K=K)
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(n)
    tally = api.Tally([])
    adj = api.Adjoint(bg, prm, OBS, 0, steps, K)
    adj.ws.ensure(api.fte_adjoint_workspace_bytes(bg, n, steps, K))    # no allocation while capturing
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = api.Graph()
    with torch.cuda.stream(side):
        with g.capture(side):
            api.fte_tally_reset(tally, stream=side)
            api.fte_inject(pool, bg, w.inject, n, tally, id_base=0, check_failed=False, stream=side)
            adj.forward(pool, stream=side)
            adj.reverse(pool, w.inject, stream=side)
        for rep in range(2):
            adj.out.zero_()
            g.launch(side)
            side.synchronize()
            assert float(adj.out[0]) == pytest.approx(J0, rel=1e-12), rep
            assert np.allclose(adj.out[1:].cpu().numpy(), g0, rtol=1e-9, atol=0), rep
    assert J0 > 0 and np.abs(g0[:3]).max() > 0


@pytest.mark.parametrize("name,prm,names", MODELS, ids=[m[0] for m in MODELS])
def test_total_matches_gpu_finite_differences(cir_small, name, prm, names):
    """Sum over many particles against central differences (2 % of each parameter) of
    the GPU forward pass with common random numbers, within 4 combined standard errors
    (batch means over 32 particle-id classes).  The pathwise-only total (window 0) is
    printed beside it; the oracle's exact-derivative pins show its bias."""
    w, f = cir_small
    n, steps = 40000, 400
    J, g, pp, st = _gpu(w, f, prm, n, steps)
    ids = np.arange(n)
    for nm in names:
        v0 = getattr(prm, nm)
        h = 2e-2 * v0
        Jp = _gpu(w, f, dataclasses.replace(prm, **{nm: v0 + h}), n, steps)[2][:, 0].astype(np.float64)
        Jm = _gpu(w, f, dataclasses.replace(prm, **{nm: v0 - h}), n, steps)[2][:, 0].astype(np.float64)
        fd = (Jp - Jm) / (2 * h)
        ga = pp[:, GI[nm]].astype(np.float64)
        sa, sf = _batch_sigma(ga, ids), _batch_sigma(fd, ids)
        band = 4 * math.sqrt(sa * sa + sf * sf)
        print(f"{name} total d/d{nm}: adjoint {ga.sum():.6e} +- {sa:.2e}, GPU central difference "
              f"{fd.sum():.6e} +- {sf:.2e}")
        assert g[GI[nm] - 1] == pytest.approx(ga.sum(), rel=1e-4, abs=1e-6 * abs(ga).sum())
        assert abs(ga.sum() - fd.sum()) < band, nm
        if name != "iso":
            g0 = _gpu(w, f, prm, n, steps, obs=dataclasses.replace(OBS, lr_window=0.0))[2][:, GI[nm]]
            g0 = g0.astype(np.float64)
            print(f"{name} total d/d{nm}: pathwise only {g0.sum():.6e} +- {_batch_sigma(g0, ids):.2e}")


def test_autograd_function(cir_small):
    import torch
    from paper_2404_12164_gb300 import api
    w, f = cir_small
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    prm = MODELS[0][1]

    class Run:
        pass
    run = Run()
    run.bg, run.params, run.inject, run.obs = bg, prm, w.inject, OBS
    run.n_steps, run.n_particles, run.checkpoint_every = 200, 2000, 50
    theta = torch.tensor([prm.lambda_par, prm.q, prm.H, prm.eps, w.inject.gamma], dtype=torch.float64,
                         requires_grad=True)
    J = api.SmoothIntensity.apply(theta, run)
    (gt,) = torch.autograd.grad(2.0 * J, theta)
    _, g, _, _ = _gpu(w, f, prm, 2000, 200, K=50)
    assert np.allclose(gt.numpy(), 2.0 * g, rtol=1e-6, atol=0)


def test_refused_configurations(cir_small):
    from paper_2404_12164_gb300 import api, _abi as A
    w, f = cir_small
    bg = api.Background(w.grid)
    api.fte_load_background(bg, f)
    pool = api.Particles(10)
    tally = api.Tally([])
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, 10, tally)
    for bad, status in ((Params(lambda_perp=0.001), A.FTE_ENOTSUP),
                        (Params(p_ref=0.05, alpha=0.3), A.FTE_ENOTSUP)):
        with pytest.raises(A.FteError) as e:
            api.Adjoint(bg, bad, OBS, 0, 10).forward(pool)
        assert e.value.status == status
    with pytest.raises(A.FteError) as e:
        api.Adjoint(bg, Params(), dataclasses.replace(OBS, sigma_t=0.0), 0, 10).forward(pool)
    assert e.value.status == A.FTE_EINVAL
