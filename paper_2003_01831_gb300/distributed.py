"""Walker-parallel runs over several processes (one GPU each).

Walkers are independent once their fields are fixed, so a population of ``W_total`` walkers
is split into consecutive ranges, one per rank, with no exchange on the data path.  Each
rank's walker set is created with ``walker_offset`` = the global index of its first walker,
so the Philox fields -- and with them every walker's trajectory -- are exactly those of a
single run over the whole population.  The only cross-rank quantity is the mixed estimator
``E_mix = sum_w w E_L / sum_w w``, combined from per-rank partial sums by one all-reduce of
four doubles per measurement.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def shard(W_total: int, rank: int, world: int) -> Tuple[int, int]:
    """(offset, count) of rank's consecutive walker range; the first W_total % world ranks
    take one extra walker."""
    if world < 1 or not 0 <= rank < world or W_total < world:
        raise ValueError("need 0 <= rank < world <= W_total")
    base, extra = divmod(W_total, world)
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def partial_sums(w: np.ndarray, E_L: np.ndarray) -> np.ndarray:
    """[Re, Im] of sum_w w E_L and of sum_w w over this rank's walkers (float64[4])."""
    w = np.asarray(w)
    num = np.sum(w * np.asarray(E_L))
    den = np.sum(w)
    return np.array([num.real, num.imag, np.real(den), np.imag(den)], dtype=np.float64)


def combine_emix(partial: np.ndarray, group=None) -> complex:
    """All-reduce the partial sums of every rank (torch.distributed, any backend) and
    return the population's E_mix."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.asarray(partial, dtype=np.float64))
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    s = t.cpu().numpy()
    return complex(s[0], s[1]) / complex(s[2], s[3])
