"""Walker-parallel runs over several processes (one GPU each).

Walkers are independent once their fields are fixed, so a population of ``W_total`` walkers
is split into consecutive ranges, one per rank, with no exchange on the data path.  Each
rank's walker set is created with ``walker_offset`` = the global index of its first walker,
so the Philox fields -- and with them every walker's trajectory -- are exactly those of a
single run over the whole population.  The cross-rank quantities are:

* the mixed estimator ``E_mix = sum_w w E_L / sum_w w``, combined from per-rank partial sums
  by one all-reduce of four doubles per measurement.  On GPUs the library forms the partial
  sums on the device (``afqmc_mixed_sums``) and the all-reduce runs on the device tensor, so
  nothing of the estimator is computed in Python;
* back-propagated density matrices, from every rank's estimate and weight sum by one
  all-reduce (``combine_rdm1``);
* population control over the whole population (the comb of ``afqmc_population_control``,
  which acts within one walker set): the ranks gather every weight, each runs the same comb
  on the full vector, and the selected walkers move between ranks point to point (each
  source walker once per destination).  Every rank keeps its walker count, so the slot
  ranges, and with them the Philox streams, stay those of one process running the whole
  population and its comb.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence, Tuple

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
    """[Re, Im] of sum_w w E_L and of sum_w w over this rank's walkers (float64[4]), from host
    arrays: the form used where a CPU model of a rank stands in for its GPU (the tests); a
    GPU walker set gives the same sums on the device through ``device_partial_sums``."""
    w = np.asarray(w)
    num = np.sum(w * np.asarray(E_L))
    den = np.sum(w)
    return np.array([num.real, num.imag, np.real(den), np.imag(den)], dtype=np.float64)


def device_partial_sums(g, nmeas: int = 1):
    """The partial sums of the last measurement call of a ``walkers.AFQMC`` walker set, as a
    float64 [nmeas, 4] CUDA tensor written by the library on the walker set's stream."""
    import torch
    from . import api
    t = torch.empty((nmeas, 4), dtype=torch.float64, device="cuda")
    api.afqmc_mixed_sums(g.wk, nmeas, t, g.stream)
    return t


def allreduce_sums(t, group=None):
    """Sum partial sums ([..., 4] float64 tensor) over the ranks in place.  Under NCCL a CUDA
    tensor stays on the device (no host round trip); under gloo the tensor must be on the
    host."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def emix_from_sums(t) -> np.ndarray:
    """E_mix = S / D for every row (S, D complex from (Re S, Im S, Re D, Im D))."""
    s = np.asarray(t.cpu().numpy() if hasattr(t, "cpu") else t, dtype=np.float64).reshape(-1, 4)
    return (s[:, 0] + 1j * s[:, 1]) / (s[:, 2] + 1j * s[:, 3])


def combine_emix(partial, group=None) -> complex:
    """All-reduce the partial sums of every rank (torch.distributed, any backend) and
    return the population's E_mix.  partial: float64[4] (numpy, or a tensor on the group's
    device)."""
    import torch
    import torch.distributed as dist
    t = partial if isinstance(partial, torch.Tensor) else torch.as_tensor(np.asarray(partial, dtype=np.float64))
    if dist.is_available() and dist.is_initialized():
        t = t.to(_device_for(group))
        allreduce_sums(t, group)
    return complex(emix_from_sums(t)[0])


def combine_rdm1(G_up: np.ndarray, G_dn: np.ndarray, w_sum: complex, group=None):
    """Population back-propagated density matrices from every rank's afqmc_bp_rdm1 result
    (each normalised by its own weights): sum_r W_r G_r / sum_r W_r, with W_r = sum of the
    rank's end-of-window weights.  One all-reduce of 4 M^2 + 2 doubles."""
    import torch
    import torch.distributed as dist
    M = G_up.shape[0]
    w_sum = complex(w_sum)
    buf = np.concatenate([(w_sum * np.asarray(G_up)).ravel(), (w_sum * np.asarray(G_dn)).ravel(), [w_sum]])
    t = torch.from_numpy(buf.astype(np.complex128).view(np.float64).copy())
    if dist.is_available() and dist.is_initialized():
        t = t.to(_device_for(group))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    s = t.cpu().numpy().view(np.complex128)
    return s[:M * M].reshape(M, M) / s[-1], s[M * M:2 * M * M].reshape(M, M) / s[-1]


def _device_for(group):
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def _library_comb(w: np.ndarray, xi: float):
    from . import api
    return api.afqmc_comb_indices(w, xi)


def comb_across_ranks(w_local: np.ndarray, xi: float, group=None,
                      comb: Optional[Callable[[np.ndarray, float], Tuple[np.ndarray, float]]] = None):
    """The comb over the whole population.  Returns (idx [W_total]: the global source walker of
    every global slot, counts [world]: walkers per rank in rank order, total weight); every
    rank computes the same.  comb(w, xi) -> (idx, total) selects; by default the library's
    kernel (afqmc_comb_indices)."""
    import torch
    import torch.distributed as dist
    comb = comb or _library_comb
    w_local = np.asarray(w_local, dtype=np.float64).real
    world = dist.get_world_size(group)
    dev = _device_for(group)
    n = torch.tensor([w_local.size], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    counts = np.array([int(t.item()) for t in ns])
    pad = torch.zeros(int(counts.max()), dtype=torch.float64, device=dev)
    pad[:w_local.size] = torch.from_numpy(w_local).to(dev)
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    w_all = np.concatenate([p.cpu().numpy()[:c] for p, c in zip(parts, counts)])
    idx, total = comb(w_all, xi)
    return np.asarray(idx, dtype=np.int64), counts, float(total)


def exchange_walkers(P_local: np.ndarray, idx: np.ndarray, counts: Sequence[int], group=None) -> np.ndarray:
    """This rank's walkers after the comb: row k is global walker idx[off + k] (off = this
    rank's first global slot).  P_local [W_r, ...] holds this rank's walkers (any dtype, one
    row each); rows owned by other ranks arrive by point-to-point messages, each source row
    once per destination."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    dev = _device_for(group)
    counts = np.asarray(counts, dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)])
    P_local = np.ascontiguousarray(P_local)
    row_shape = P_local.shape[1:]

    def owner(j):
        return int(np.searchsorted(offs, j, side="right") - 1)

    def needs(r):   # sorted global indices rank r's slots take from each owner
        src = idx[offs[r]:offs[r + 1]]
        out = {}
        for j in np.unique(src):
            out.setdefault(owner(int(j)), []).append(int(j))
        return out

    def pack(rows):
        a = np.ascontiguousarray(rows)
        return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).to(dev)

    # every send and receive of this rank goes into one batch_isend_irecv, so a backend whose
    # point-to-point calls between two ranks share one stream (NCCL) sees them as one group
    # instead of two blocking sends facing each other
    ops, incoming = [], {}
    for r in range(world):           # what this rank sends
        if r == rank:
            continue
        mine = needs(r).get(rank, [])
        if mine:
            ops.append(dist.P2POp(dist.isend, pack(P_local[np.array(mine) - offs[rank]]), r, group))
    for q, js in needs(rank).items():   # what this rank receives
        if q == rank:
            continue
        buf = torch.zeros(len(js) * P_local[0].nbytes // 8, dtype=torch.float64, device=dev)
        ops.append(dist.P2POp(dist.irecv, buf, q, group))
        incoming[q] = (js, buf)
    if ops:
        for rq in dist.batch_isend_irecv(ops):
            rq.wait()
    rows = {}
    for q, (js, buf) in incoming.items():
        got = buf.cpu().numpy().view(P_local.dtype).reshape((len(js),) + row_shape)
        for j, row in zip(js, got):
            rows[j] = row
    out = np.empty((int(counts[rank]),) + row_shape, dtype=P_local.dtype)
    for k, j in enumerate(idx[offs[rank]:offs[rank + 1]]):
        j = int(j)
        out[k] = P_local[j - offs[rank]] if owner(j) == rank else rows[j]
    return out


def population_control(g, xi: float, group=None) -> np.ndarray:
    """Comb population control of a walker population spread over the ranks, one
    ``walkers.AFQMC`` walker set per rank (phaseless or local-energy weights).  Every new
    walker gets the weight total / W_total.  Returns the global source of every global slot.
    A back-propagation window open on a walker set is closed (``set_walkers``)."""
    Pu, Pd, w, step = g.walkers()
    W = w.size
    idx, counts, total = comb_across_ranks(w, xi, group)
    P = np.concatenate([Pu.reshape(W, -1), Pd.reshape(W, -1)], axis=1)
    P = exchange_walkers(P, idx, counts, group)
    n_up = Pu[0].size
    w_new = np.full(W, total / float(np.sum(counts)))
    g.set_walkers(P[:, :n_up].reshape(Pu.shape), P[:, n_up:].reshape(Pd.shape), w_new, step)
    return idx
