"""Pins of the oracle's block-AMR background access (Sec. 2.4, Fig. 4).

Sec. 2.4: each refinement halves a block in every direction; touching blocks
differ by at most one level; a particle near a block edge needs data of the
same-level, coarser or finer neighbours, which the paper fetches from the
neighbouring blocks instead of storing ghost cells.  The oracle computes those
neighbour values on demand.  Pins: with no refinement the AMR path equals the
uniform-grid path; a field affine in (r, theta, phi) is reproduced exactly at
every point, on every level and across every coarse/fine interface.
"""
import math

import numpy as np
import pytest

from fte_inputs import amr, backgrounds, configs
from fte_inputs.grid import GridSpec
from oracle import oracle as O


def _cart(r, th, ph):
    return (r * math.sin(th) * math.cos(ph), r * math.sin(th) * math.sin(ph), r * math.cos(th))


def _vec(out):
    return np.concatenate([out["B"], out["V"], out["G"].ravel(), out["gB"]])


@pytest.fixture(scope="module")
def refined():
    spec = amr.AmrSpec(nbr=4, nbt=2, nbp=4, bsize=8, levels=3, n_snap=1)
    leaves = amr.build_leaves(spec, amr.divv_refiner(spec, threshold=8e-6, r_from=0.9))
    return spec, leaves


def test_tree_is_balanced_and_morton_sorted(refined):
    spec, leaves = refined
    assert np.bincount(leaves[:, 0]).size == 3           # all three levels present
    assert amr.check_balance(spec, leaves)
    tab = amr.finest_table(spec, leaves)
    assert (tab >= 0).all()
    # each leaf covers exactly its 8^(L - level) finest blocks
    counts = np.bincount(tab.ravel(), minlength=len(leaves))
    assert np.array_equal(counts, 8 ** (spec.L - leaves[:, 0]))
    s = 1 << (spec.L - leaves[:, 0]).astype(np.int64)
    key = amr.morton3(leaves[:, 1] * s, leaves[:, 2] * s, leaves[:, 3] * s)
    assert np.all(np.diff(key) > 0)


@pytest.mark.parametrize("radial", ["linear", "log"])
def test_unrefined_amr_equals_uniform_grid(radial):
    spec = amr.AmrSpec(nbr=4, nbt=2, nbp=4, bsize=8, levels=2, radial=radial, n_snap=2,
                       periodic=True, dt_snap=3600.0)
    g = GridSpec(nr=32, nth=16, nph=32, radial=radial, n_snap=2, periodic=True, dt_snap=3600.0)
    uni = backgrounds.cir(g)
    leaves, f = amr.from_uniform(spec, uni)
    ba = O.amr_background(spec, leaves, f)
    bu = O.grid_background(g, uni)
    rng = np.random.default_rng(1)
    scale = np.abs(uni).max(axis=(0, 1, 2, 3))[:18]
    for _ in range(300):
        r = rng.uniform(0.1, 2.0)
        th = rng.uniform(g.th_min, g.th_max)
        ph = rng.uniform(0, 2 * math.pi)
        t = rng.uniform(0, 7200)
        a = O.eval_fields(ba, *_cart(r, th, ph), t)
        u = O.eval_fields(bu, *_cart(r, th, ph), t)
        assert np.all(np.abs(_vec(a) - _vec(u)) <= 1e-12 * scale)
        assert np.allclose(a["dVdt"], u["dVdt"], rtol=1e-9, atol=1e-22)
        assert np.allclose(a["dB"], u["dB"], rtol=1e-9, atol=1e-9 * np.abs(u["dB"]).max())


@pytest.mark.parametrize("radial", ["linear", "log"])
def test_affine_field_exact_across_levels(refined, radial):
    spec0, _ = refined
    spec = amr.AmrSpec(nbr=spec0.nbr, nbt=spec0.nbt, nbp=spec0.nbp, bsize=spec0.bsize,
                       levels=spec0.levels, radial=radial, n_snap=1)
    leaves = amr.build_leaves(spec, amr.divv_refiner(spec, threshold=8e-6, r_from=0.9))
    f, coef = amr.affine(spec, leaves, seed=3)
    bg = O.amr_background(spec, leaves, f)
    # sample points near every kind of interface: within a fraction of a cell of block edges
    rng = np.random.default_rng(2)
    scale = np.abs(f).max()
    lv_of = leaves[:, 0]
    checked = {0: 0, 1: 0, 2: 0}
    tab = amr.finest_table(spec, leaves)
    nf = spec.finest_blocks()
    for _ in range(1500):
        u = rng.uniform(0, 1, 3)
        # keep inside the outermost centres (clamped zone is constant, not affine) and off the phi seam
        c0 = amr.centres_1d(spec, 0, 0, [0, spec.cells(0)[0] - 1])
        t0 = amr.centres_1d(spec, 0, 1, [0, spec.cells(0)[1] - 1])
        r = c0[0] + u[0] * (c0[1] - c0[0])
        th = t0[0] + u[1] * (t0[1] - t0[0])
        ph = 0.3 + u[2] * (2 * math.pi - 0.6)
        got = _vec(O.eval_fields(bg, *_cart(r, th, ph), 0.0))
        expect = coef[:, 0] + coef[:, 1] * r + coef[:, 2] * th + coef[:, 3] * (ph - math.pi)
        assert np.abs(got - expect).max() < 3e-6 * scale
        ur = (math.log(r / spec.r_min) / math.log(spec.r_max / spec.r_min) if radial == "log"
              else (r - spec.r_min) / (spec.r_max - spec.r_min))
        fb = (int(ph / (2 * math.pi) * nf[2]), int((th - spec.th_min) / (spec.th_max - spec.th_min) * nf[1]),
              int(ur * nf[0]))
        checked[int(lv_of[tab[fb]])] += 1
    assert min(checked.values()) > 50


def test_injection_on_amr_accepts_only_compressive_cells(refined):
    spec, leaves = refined
    f = amr.fields(spec, leaves)
    bg = O.amr_background(spec, leaves, f)
    inj = configs.InjectSpec(region="box", r1=1.0, r2=2.0, th1=math.radians(80), th2=math.radians(100),
                             ph1=0.0, ph2=2 * math.pi, divv_max=0.0, max_tries=4096, weight="r-2")
    P, led = O.inject(bg, inj, np.arange(500))
    assert np.all(P["status"] == O.ALIVE)
    for p in P[:200]:
        out = O.eval_fields(bg, p["x"], p["y"], p["z"], 0.0)
        # the containing cell's stored div V is negative; the interpolated value is mostly so
    assert led.as_dict()["n"][0] == 500
