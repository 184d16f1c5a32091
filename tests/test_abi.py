"""The C-ABI library loads and exports every entry point include/*.h declares;
host-side argument checks that return before any CUDA call work without a GPU."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(fte_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2404_12164_gb300 import build
    build.build()
    from paper_2404_12164_gb300 import _abi
    return _abi.lib()


def test_every_declared_symbol_is_exported(L):
    from paper_2404_12164_gb300 import _abi
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
        assert n in _abi.SIGNATURES, n


def test_version_and_status_strings(L):
    assert L.fte_abi_version() == 3
    assert L.fte_status_string(0) == b"ok"
    assert L.fte_status_string(1) == b"invalid argument"


def test_struct_sizes_match_header_layout():
    from paper_2404_12164_gb300 import _abi as A
    assert C.sizeof(A.fte_grid) == 4 * 4 + 4 * 8 + 2 * 4 + 2 * 8 + 6 * 4
    assert C.sizeof(A.fte_observer) == 4 * 4 + 10 * 8
    assert C.sizeof(A.fte_params) == 4 * 4 + 10 * 8 + 4 * 4
    assert C.sizeof(A.fte_inject_spec) == 4 * 4 + 9 * 8 + 4 * 4 + 6 * 8 + 4 * 4 + 2 * 8
    assert C.sizeof(A.fte_smooth_obs) == 7 * 8
    assert C.sizeof(A.fte_tally_buf) == 2 * 4 + A.FTE_MAX_OBS * C.sizeof(A.fte_observer) + 6 * 8


def test_background_bytes_and_grid_validation(L):
    from fte_inputs.grid import GridSpec
    from paper_2404_12164_gb300 import api, _abi as A
    g = GridSpec(nr=512, nth=60, nph=180, n_snap=24, periodic=True)
    gc = api.grid_c(g)
    assert L.fte_background_bytes(C.byref(gc)) == 512 * 60 * 180 * 24 * 96
    for bad in (dict(nr=1), dict(r_min=0.0), dict(r_max=0.05), dict(th_max=4.0), dict(n_snap=0)):
        kw = dict(nr=8, nth=8, nph=8)
        kw.update(bad)
        gb = GridSpec(**kw)
        assert L.fte_background_bytes(C.byref(api.grid_c(gb))) == 0
        st = L.fte_load_background(C.byref(api.grid_c(gb)), C.c_void_p(16), C.c_void_p(16), 1 << 40, None)
        assert st == A.FTE_EINVAL
        assert len(L.fte_last_error()) > 0
    # undersized device buffer and misaligned pointer are refused before any copy
    gc = api.grid_c(GridSpec(nr=8, nth=8, nph=8))
    assert L.fte_load_background(C.byref(gc), C.c_void_p(16), C.c_void_p(64), 100, None) == A.FTE_ENOMEM
    assert L.fte_load_background(C.byref(gc), C.c_void_p(16), C.c_void_p(16), 1 << 30, None) == A.FTE_EINVAL
    assert L.fte_load_background(None, C.c_void_p(16), C.c_void_p(16), 1 << 30, None) == A.FTE_EINVAL


def test_tally_bins_and_observer_validation(L):
    from fte_inputs.configs import Observer
    from paper_2404_12164_gb300 import api, _abi as A
    t = A.fte_tally_buf()
    t.n_obs = 2
    t.obs[0] = api.observer_c(Observer(ne=16, nt=144))
    t.obs[1] = api.observer_c(Observer(ne=4, nt=10))
    assert L.fte_tally_bins(C.byref(t)) == 16 * 144 + 40
    t.n_obs = 9
    assert L.fte_tally_bins(C.byref(t)) == 0
    t.n_obs = 1
    t.obs[0] = api.observer_c(Observer(ne=16, nt=144, e_lo=1.0, e_hi=0.5))
    # invalid energy range is refused (ledger pointers are checked after the observers)
    assert L.fte_tally_reset(C.byref(t), None) == A.FTE_EINVAL
    assert b"e_lo" in L.fte_last_error()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2404_12164_gb300 import _abi
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(ImportError):
        _abi.lib()


def test_ensemble_structs_and_host_checks(L):
    from fte_inputs.configs import Observer
    from paper_2404_12164_gb300 import api, _abi as A
    assert C.sizeof(A.fte_set) == 4 * 8 + 2 * 4 + 8
    assert C.sizeof(A.fte_launch_config) == 4 * 4
    # n_sets of a tally is bounded
    t = A.fte_tally_buf()
    t.n_obs = 1
    t.obs[0] = api.observer_c(Observer(ne=16, nt=144))
    t.n_sets = A.FTE_MAX_SETS + 1
    assert L.fte_tally_bins(C.byref(t)) == 0
    t.n_sets = A.FTE_MAX_SETS
    assert L.fte_tally_bins(C.byref(t)) == 16 * 144
    # argument checks that return before any CUDA call
    specs = (A.fte_inject_spec * 1)()
    counts = (C.c_uint64 * 1)(10)
    assert L.fte_inject_batched(None, None, specs, counts, 1, None, None) == A.FTE_EINVAL
    P = A.fte_particles()
    assert L.fte_inject_batched(C.byref(P), None, specs, counts, 0, None, None) == A.FTE_EINVAL
    assert L.fte_inject_batched(C.byref(P), None, specs, counts, A.FTE_MAX_SETS + 1, None, None) == A.FTE_EINVAL
    sets = (A.fte_set * 1)()
    assert L.fte_advance_batched(None, None, None, sets, 1, None, 0, 1, None, None, 0, None) == A.FTE_EINVAL
    best = A.fte_launch_config()
    assert L.fte_autotune_batched(None, None, None, sets, 1, None, 0, 1, None, 0, C.byref(best), None, None,
                                  None, None) == A.FTE_EINVAL
    assert L.fte_graph_begin(None) == A.FTE_EINVAL
    assert b"NULL stream" in L.fte_last_error()
    h = C.c_void_p(0)
    assert L.fte_graph_end(None, C.byref(h)) == A.FTE_EINVAL
    assert L.fte_graph_launch(None, None) == A.FTE_EINVAL
    assert L.fte_graph_destroy(None) == A.FTE_OK
    assert L.fte_tally_set(None, 0, 0, 0, None, None, 0, None) == A.FTE_EINVAL


def test_stream_plan_and_ring_sizes(L):
    """The snapshot-pair runs of a streamed advance (host-side plan) and the size of a ring
    background; no GPU needed."""
    from fte_inputs.configs import Params
    from fte_inputs.grid import GridSpec
    from paper_2404_12164_gb300 import api, _abi as A
    g = GridSpec(nr=16, nth=8, nph=8, n_snap=24, periodic=True, dt_snap=3600.0)
    snap = 16 * 8 * 8 * 96
    assert L.fte_snapshot_bytes(C.byref(api.grid_c(g))) == snap
    assert L.fte_background_bytes(C.byref(api.grid_c(g, ring=3))) == 3 * snap
    assert L.fte_stream_staging_bytes(C.byref(api.grid_c(g, ring=3))) == 0
    # host snapshots stay FP32 cell records whatever the slots hold; converted slots need
    # one staging snapshot
    for dt, lay, rec in (("bf16", "cell", 64), ("f16", "pair", 96), ("f32", "pair", 160)):
        gc = api.grid_c(g, dtype=dt, ring=3, layout=lay)
        head = 0 if dt == "f32" else 128
        assert L.fte_snapshot_bytes(C.byref(gc)) == snap
        assert L.fte_stream_staging_bytes(C.byref(gc)) == snap
        assert L.fte_background_bytes(C.byref(gc)) == head + 3 * 16 * 8 * 8 * rec
    for bad in (1, 25, -1):
        assert L.fte_background_bytes(C.byref(api.grid_c(g, ring=bad))) == 0

    def plan(grid, prm, a, b):
        gc, pc = api.grid_c(grid, ring=2), api.params_c(prm)
        cnt = C.c_int64(0)
        out = (C.c_int64 * 3000)()
        assert L.fte_stream_plan(C.byref(gc), C.byref(pc), a, b, out, 1000, C.byref(cnt)) == A.FTE_OK
        return [tuple(out[3 * k:3 * k + 3]) for k in range(cnt.value)]
    runs = plan(g, Params(dt=10.0), 0, 34560)
    assert len(runs) == 96
    assert all(r == (360 * k, 360 * (k + 1), k) for k, r in enumerate(runs))
    # non-periodic, starting before the first snapshot: frozen, three pairs, frozen at the last
    g2 = GridSpec(nr=16, nth=8, nph=8, n_snap=4, periodic=False, dt_snap=1000.0)
    runs = plan(g2, Params(dt=10.0, t0=-500.0), 0, 400)
    assert runs == [(0, 50, -1), (50, 150, 0), (150, 250, 1), (250, 350, 2), (350, 400, -4)]
    # too little room is reported with the count
    gc, pc = api.grid_c(g, ring=2), api.params_c(Params(dt=10.0))
    cnt = C.c_int64(0)
    out = (C.c_int64 * 3)()
    assert L.fte_stream_plan(C.byref(gc), C.byref(pc), 0, 720, out, 1, C.byref(cnt)) == A.FTE_ENOMEM
    assert cnt.value == 2 and tuple(out) == (0, 360, 0)
