"""The multi-process path on CPU (gloo, world size 2): each rank advances its own
batch with disjoint particle ids, the tallies and ledgers are summed over the
ranks, and the step time is the slowest rank's.  The per-rank work here is the
FP64 oracle, so the reduced tallies (and the observer totals by particle-id
class) must equal one oracle run over both batches (counts exactly, sums to
rounding)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from fte_inputs import configs
from fte_inputs.configs import Observer

N_PER_RANK = 600
STEPS = 400


def _workload():
    w = configs.scaled(configs.parker_1e4(), n_particles=N_PER_RANK)
    obs = [Observer(kind="shell", r=0.16, dr=0.04, e_lo=0.01, e_hi=1.0, ne=8, t_lo=0.0, t_hi=4000.0, nt=10)]
    return w, obs


class _T:
    pass


def _oracle_batch(w, f, obs, ids):
    from oracle import oracle as O
    bg = O.grid_background(w.grid, f)
    P, led = O.inject(bg, w.inject, np.asarray(ids, dtype=np.uint32))
    T = O.Tally(obs)
    O.advance(bg, w.params, P, 0, STEPS, tally=T, ledger=led, threads=2)
    L = led.as_dict()
    return T, L


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    from paper_2404_12164_gb300 import dist as pdist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w, obs = _workload()
    f = configs.build_background(w)
    base = pdist.id_base(rank, N_PER_RANK)
    T, L = _oracle_batch(w, f, obs, np.arange(base, base + N_PER_RANK))
    t = _T()
    t.S, t.S2 = torch.tensor(T.S), torch.tensor(T.S2)
    t.C = torch.tensor(T.C.astype(np.int64))
    t.ledger_w = torch.tensor(np.asarray(L["w"], dtype=np.float64))
    t.ledger_n = torch.tensor(np.asarray(L["n"], dtype=np.int64))
    t.S_class = torch.tensor(T.SC)
    pdist.reduce_tally(t)
    (slowest,) = pdist.max_over_ranks([10.0 + rank])
    if rank == 0:
        np.savez(os.path.join(out_dir, "reduced.npz"), S=t.S.numpy(), S2=t.S2.numpy(), C=t.C.numpy(),
                 SC=t.S_class.numpy(),
                 lw=t.ledger_w.numpy(), ln=t.ledger_n.numpy(), slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_equal_one_run(tmp_path):
    from oracle import build as ob
    ob.build()
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(tmp_path / "reduced.npz")
    w, obs = _workload()
    f = configs.build_background(w)
    T, L = _oracle_batch(w, f, obs, np.arange(2 * N_PER_RANK))
    assert T.C.sum() > 100
    assert np.array_equal(got["C"], T.C.astype(np.int64))
    assert np.allclose(got["S"], T.S, rtol=1e-12, atol=0)
    assert np.allclose(got["S2"], T.S2, rtol=1e-12, atol=0)
    # observer totals by particle-id class (batch means of the total) sum over ranks too
    assert np.allclose(got["SC"], T.SC, rtol=1e-12, atol=0) and T.SC.sum() > 0
    assert np.array_equal(got["ln"], np.asarray(L["n"], dtype=np.int64))
    assert np.allclose(got["lw"], L["w"], rtol=1e-12)
    assert int(got["ln"][0]) == 2 * N_PER_RANK
    assert float(got["slowest"]) == 11.0


def test_single_process_helpers():
    from paper_2404_12164_gb300 import dist as pdist
    assert pdist.id_base(3, 1000) == 3000
    t = _T()
    t.S = torch.ones(4, dtype=torch.float64)
    t.S2, t.C = t.S.clone(), torch.ones(4, dtype=torch.int64)
    t.ledger_w, t.ledger_n = torch.zeros(8, dtype=torch.float64), torch.zeros(8, dtype=torch.int64)
    assert pdist.reduce_tally(t) is t and float(t.S.sum()) == 4.0
    assert pdist.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
