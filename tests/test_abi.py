"""The C-ABI library loads and exports every entry point include/fte.h declares;
host-side argument checks that return before any CUDA call work without a GPU."""
import ctypes as C
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fte.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fte_[a-z_]+)\s*\(", src)
    return sorted(set(names))


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
    assert L.fte_abi_version() == 1
    assert L.fte_status_string(0) == b"ok"
    assert L.fte_status_string(1) == b"invalid argument"


def test_struct_sizes_match_header_layout():
    from paper_2404_12164_gb300 import _abi as A
    assert C.sizeof(A.fte_grid) == 4 * 4 + 4 * 8 + 2 * 4 + 2 * 8 + 4 * 4
    assert C.sizeof(A.fte_observer) == 4 * 4 + 10 * 8
    assert C.sizeof(A.fte_params) == 4 * 4 + 10 * 8 + 4 * 4
    assert C.sizeof(A.fte_inject_spec) == 4 * 4 + 9 * 8 + 4 * 4 + 6 * 8 + 4 * 4


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
