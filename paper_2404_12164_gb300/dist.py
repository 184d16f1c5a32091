"""Data-parallel runs over several processes (one GPU each): particles are
independent given the background, so every rank advances its own batch with
distinct particle ids (weak scaling) and the only exchange is the sum of the
tallies and ledgers; the step time of a run is the slowest rank's."""
import torch
import torch.distributed as dist


def id_base(rank, n_per_rank):
    """First particle id of `rank`'s batch: ranks draw disjoint Philox streams."""
    return int(rank) * int(n_per_rank)


def reduce_tally(tally):
    """Sum S, S2, C, both ledgers and the class totals S_class (when present) over the ranks,
    in place (every rank gets the totals).  `tally` has tensors S, S2, C, ledger_w, ledger_n
    (api.Tally or any object with them)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tally
    ts = [tally.S, tally.S2, tally.C, tally.ledger_w, tally.ledger_n]
    if getattr(tally, "S_class", None) is not None:
        ts.append(tally.S_class)
    for t in ts:
        dist.all_reduce(t)
    return tally


def max_over_ranks(values, device=None):
    """Element-wise maximum over the ranks of a list of floats (e.g. timed milliseconds)."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()
