"""Snapshot streaming through a ring of resident slots on the GPU: the same run
with all snapshots resident and with 2 or 3 slots filled on demand from host
memory gives the same trajectories (bit for bit) and the same tallies, for
periodic and non-periodic sequences and for block-AMR backgrounds (whose ghost
layers are refilled on the device after each upload).  Rings in 16-bit or pair
storage convert each FP32 host snapshot on the device through a staging buffer;
their scales come from all host snapshots, so they equal the resident background
converted by fte_quantize_background, and so do the trajectories."""
import math

import numpy as np
import pytest

from fte_inputs import amr, configs
from fte_inputs.configs import InjectSpec, Observer, Params

pytestmark = pytest.mark.gpu
DEG = math.pi / 180


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import build
    build.build()


OBS = [Observer(kind="shell", r=1.4, dr=0.05, e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=8000.0, nt=16)]


def _run(bg, w, n, n_steps, stream_state=None, splits=(0,)):
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    pool = api.Particles(n)
    tally = api.Tally(OBS)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, n, tally)
    ws = api.Workspace()
    bounds = list(splits) + [n_steps]
    for a, b in zip(bounds[:-1], bounds[1:]):
        if stream_state is None:
            api.fte_advance(pool, bg, w.params, tally, a, b, ws)
        else:
            api.fte_advance_streamed(pool, bg, stream_state, w.params, tally, a, b, ws)
    torch.cuda.synchronize()
    return pool.state(), api.fte_tally(tally, 0, A.FTE_TALLY_C), api.fte_tally(tally, 0, A.FTE_TALLY_S)


def _same(a, b):
    sa, ca, Sa = a
    sb, cb, Sb = b
    for k in ("x", "y", "z", "mu", "p", "status"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(ca, cb)
    assert np.allclose(Sa, Sb, rtol=1e-5, atol=0)     # per-launch FP32 partial sums group differently


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("ring", [2, 3, 6])
def test_uniform_ring_equals_resident(periodic, ring):
    from paper_2404_12164_gb300 import api
    w = configs.scaled(configs.cir_uniform_1e6(), nr=96, nth=24, nph=72, n_snap=6, n_particles=3000)
    w.grid.periodic = periodic
    w.grid.dt_snap = 600.0
    w.params.sort_every = 32
    w.inject.divv_max = None           # injection reads no snapshot (ring slots fill on demand)
    f = configs.build_background(w)
    n_steps = 800                      # 8000 s: beyond the period (3600 s) / the last snapshot (3000 s)
    res = api.Background(w.grid)
    api.fte_load_background(res, f)
    ref = _run(res, w, w.n_particles, n_steps)
    bg = api.Background(w.grid, ring=ring)
    st = api.SnapshotStream(bg, f)
    got = _run(bg, w, w.n_particles, n_steps, st, splits=(0, 333))
    _same(got, ref)
    plan = api.fte_stream_plan(bg, w.params, 0, n_steps)
    if periodic:
        assert len(plan) == 14 and np.all(plan[:-1, 1] - plan[:-1, 0] == 60)
        if ring == 6:          # one slot per snapshot: the second period reuses the first one's
            assert sorted(st.slots % 6) == list(range(6)) and st.slots.max() >= 6
    else:
        assert plan[-1, 2] == -1 - 5 and plan[-1, 1] == n_steps


def test_amr_ring_refills_ghosts():
    from paper_2404_12164_gb300 import api
    spec = amr.AmrSpec(nbr=4, nbt=2, nbp=4, bsize=8, levels=3, n_snap=4, periodic=False, dt_snap=1500.0)
    leaves = amr.build_leaves(spec, amr.divv_refiner(spec, threshold=8e-6, r_from=0.9))
    f = amr.fields(spec, leaves)
    w = configs.cir_uniform_1e6()
    w.inject = InjectSpec(region="box", r1=1.0, r2=1.8, th1=88 * DEG, th2=92 * DEG, ph1=math.pi, ph2=2 * math.pi,
                          energy="mono", e0=0.05, weight="r-2", seed=2)
    w.params = Params(dmumu="qlt", lambda_par=0.1, dt=10.0, sort_every=32)
    res = api.AmrBackground(spec, leaves)
    api.fte_load_background(res, f)
    api.fte_amr_prepare(res)
    ref = _run(res, w, 2000, 600)
    bg = api.AmrBackground(spec, leaves, ring=2)
    api.fte_amr_prepare(bg)                      # table; the slots are filled by the stream
    st = api.SnapshotStream(bg, f)
    got = _run(bg, w, 2000, 600, st)
    _same(got, ref)


def _uniform(n_snap=6, periodic=True):
    w = configs.scaled(configs.cir_uniform_1e6(), nr=96, nth=24, nph=72, n_snap=n_snap, n_particles=3000)
    w.grid.periodic = periodic
    w.grid.dt_snap = 600.0
    w.params.sort_every = 32
    w.inject.divv_max = None
    return w, configs.build_background(w)


@pytest.mark.parametrize("dtype,layout", [("bf16", "cell"), ("f16", "pair"), ("f32", "pair"), ("bf16", "pair")])
def test_converted_ring_equals_resident(dtype, layout):
    from paper_2404_12164_gb300 import api
    w, f = _uniform(periodic=(dtype != "f16"))
    n_steps = 800
    b32 = api.Background(w.grid)
    api.fte_load_background(b32, f)
    res = api.Background(w.grid, dtype=dtype, layout=layout)
    api.fte_quantize_background(res, b32)
    ref = _run(res, w, w.n_particles, n_steps)
    bg = api.Background(w.grid, dtype=dtype, ring=3, layout=layout)
    st = api.SnapshotStream(bg, f)
    if dtype != "f32":                  # the scale header equals the resident one
        assert np.array_equal(api.device_bytes(bg)[:128], api.device_bytes(res)[:128])
    got = _run(bg, w, w.n_particles, n_steps, st, splits=(0, 333))
    _same(got, ref)


def test_converted_amr_ring():
    from paper_2404_12164_gb300 import api
    spec = amr.AmrSpec(nbr=4, nbt=2, nbp=4, bsize=8, levels=3, n_snap=4, periodic=False, dt_snap=1500.0)
    leaves = amr.build_leaves(spec, amr.divv_refiner(spec, threshold=8e-6, r_from=0.9))
    f = amr.fields(spec, leaves)
    w = configs.cir_uniform_1e6()
    w.inject = InjectSpec(region="box", r1=1.0, r2=1.8, th1=88 * DEG, th2=92 * DEG, ph1=math.pi, ph2=2 * math.pi,
                          energy="mono", e0=0.05, weight="r-2", seed=2)
    w.params = Params(dmumu="qlt", lambda_par=0.1, dt=10.0, sort_every=32)
    cell = api.AmrBackground(spec, leaves)
    api.fte_load_background(cell, f)
    api.fte_amr_prepare(cell)
    res = api.AmrBackground(spec, leaves, dtype="bf16", share=cell, layout="pair")
    api.fte_quantize_background(res, cell)
    ref = _run(res, w, 2000, 600)
    bg = api.AmrBackground(spec, leaves, dtype="bf16", ring=2, layout="pair")
    api.fte_amr_prepare(bg)                      # the table only: slots fill as snapshots stream in
    st = api.SnapshotStream(bg, f)
    got = _run(bg, w, 2000, 600, st)
    _same(got, ref)


def test_streaming_refusals():
    import ctypes as C
    import torch
    from paper_2404_12164_gb300 import api, _abi as A
    w = configs.scaled(configs.cir_uniform_1e6(), nr=32, nth=8, nph=16, n_snap=4, n_particles=10)
    f = configs.build_background(w)
    plain = api.Background(w.grid)
    with pytest.raises(ValueError):
        api.SnapshotStream(plain, f)
    host = torch.from_numpy(np.ascontiguousarray(f)).pin_memory()
    slots = np.full(2, -1, dtype=np.int64)
    L = A.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    half = api.Background(w.grid, dtype="bf16", ring=2)
    need = L.fte_stream_staging_bytes(C.byref(half.gc))
    assert need == api.fte_snapshot_bytes(half) > 0
    stage = torch.empty(need, dtype=torch.uint8, device="cuda")
    hp, sp, stp = C.c_void_p(host.data_ptr()), C.c_void_p(slots.ctypes.data), C.c_void_p(stage.data_ptr())
    assert L.fte_stream_load(C.byref(half.c), hp, 0, sp, None, 0, s) == A.FTE_EINVAL
    assert L.fte_stream_load(C.byref(half.c), hp, 0, sp, stp, need - 32, s) == A.FTE_ENOMEM
    assert L.fte_stream_scales(C.byref(half.c), hp, stp, need, s) == A.FTE_OK
    assert L.fte_stream_load(C.byref(half.c), hp, 0, sp, stp, need, s) == A.FTE_OK
    assert slots[0] == 0
    ring32 = api.Background(w.grid, ring=2)
    assert L.fte_stream_scales(C.byref(ring32.c), hp, stp, need, s) == A.FTE_EINVAL
    torch.cuda.synchronize()
