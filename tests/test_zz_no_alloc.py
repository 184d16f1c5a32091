"""The allocation-free entry point gives the same results as fte_advance.

fte_advance_noalloc serves callers that cannot allocate device memory while
they run (their own allocator owns the GPU's memory, or a cudaMalloc in the
middle of a run is not allowed); it keeps its scratch in a device array the
library places statically.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import dataclasses

import numpy as np
import pytest

from fte_inputs import configs
from fte_inputs.configs import Observer

pytestmark = pytest.mark.gpu


def _setup(api, w, fields, observers):
    bg = api.Background(w.grid)
    api.fte_load_background(bg, fields)
    pool = api.Particles(w.n_particles)
    tally = api.Tally(observers)
    api.fte_tally_reset(tally)
    api.fte_inject(pool, bg, w.inject, w.n_particles, tally)
    return bg, pool, tally


def test_noalloc_matches_fte_advance_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import api, build, _abi as A
    build.build()
    w = configs.scaled(configs.cir_uniform_1e6(), nr=128, nth=30, nph=90, n_particles=5000)
    fields = configs.build_background(w)
    obs = w.observers + [Observer(kind="shell", r=1.5, dr=0.05, e_lo=0.01, e_hi=10.0, ne=16,
                                  t_lo=0.0, t_hi=4 * 86400.0, nt=144)]
    bg_a, pool_a, tally_a = _setup(api, w, fields, obs)
    bg_b, pool_b, tally_b = _setup(api, w, fields, obs)
    ws = api.Workspace()
    # the allocation-free call keeps per-block histograms in shared memory and never reorders:
    # compare with fte_advance in the shared-memory layout (which reorders, changing no result)
    prm = dataclasses.replace(w.params, tally_layout="shared")
    for n0, n1 in ((0, 700), (700, 2300)):          # two calls in a row; the second spans 2 launches
        api.fte_advance(pool_a, bg_a, prm, tally_a, n0, n1, ws)
        api.fte_advance_noalloc(pool_b, bg_b, w.params, tally_b, n0, n1)
        a, b = pool_a.state(), pool_b.state()
        for k in ("x", "y", "z", "mu", "p", "w", "status", "id"):
            assert np.array_equal(a[k], b[k]), (n1, k)
        for o in range(len(obs)):
            Ca = api.fte_tally(tally_a, o, A.FTE_TALLY_C)
            Cb = api.fte_tally(tally_b, o, A.FTE_TALLY_C)
            assert np.array_equal(Ca, Cb), (n1, o)
            Sa = api.fte_tally(tally_a, o, A.FTE_TALLY_S)
            Sb = api.fte_tally(tally_b, o, A.FTE_TALLY_S)
            assert np.allclose(Sa, Sb, rtol=1e-5, atol=1e-12 * max(Sa.max(), 1.0)), (n1, o)
        la, lb = api.fte_ledger(tally_a), api.fte_ledger(tally_b)
        assert np.array_equal(la[1], lb[1])
        assert np.allclose(la[0], lb[0], rtol=1e-12)
    assert int(lb[1][6]) > 0 and int(Cb.sum()) > 0
    torch.cuda.synchronize()


def test_noalloc_rejects_oversized_tally():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12164_gb300 import api, build, _abi as A
    build.build()
    w = configs.scaled(configs.parker_1e4(), n_particles=64)
    fields = configs.build_background(w)
    # a tally whose per-block histograms (12 bytes per bin) fit one block's shared memory
    # (at most 16,384 bins) but not one block per SM in the 24 MiB array
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nt = (24 * 2 ** 20 // (12 * sms)) // 32 + 1              # two observers of 16 x nt bins
    if 32 * nt > 16384:
        pytest.skip(f"{sms} SMs: every tally that fits a block also fits the array")
    big = [Observer(ne=16, nt=nt), Observer(ne=16, nt=nt)]
    bg, pool, tally = _setup(api, w, fields, big)
    with pytest.raises(A.FteError) as e:
        api.fte_advance_noalloc(pool, bg, w.params, tally, 0, 10)
    assert e.value.status == A.FTE_ENOMEM
    api.fte_advance(pool, bg, w.params, tally, 0, 10)            # the workspace path takes it
