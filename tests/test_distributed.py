"""Walker-parallel host logic on CPU with gloo, world size 2: each rank steps its shard of the
population (the oracle stands in for its GPU), the partial sums are all-reduced, and the
combined E_mix trace equals that of one process stepping every walker -- also with a comb over
the whole population between steps, whose selected walkers move between the ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import afqmc as O
from oracle import backprop as BP
from oracle.philox import philox_fields
from paper_2003_01831_gb300 import distributed as D
from paper_2003_01831_gb300 import synthetic as syn

W_TOTAL, NSTEPS, SEED, TAU = 7, 4, 21, 0.01


def system():
    d = syn.UnevenSystem(M=8, N=2, Nchol=12, W=W_TOTAL)
    h, L, E0, Psi = syn.make_uneven_system(d, 0, seed=5)
    return h, L, E0, Psi


COMB_AT, XI = 2, 0.83


def oracle_comb(w, xi):
    return O.comb(w, xi), float(np.sum(w))


def run_oracle(offset, count, comb=None):
    """E_mix partial sums per step for walkers [offset, offset + count).  comb: None, "single"
    (one process combs its walkers, which must be the whole population) or "ranks" (the comb
    over every rank's walkers, exchanging walkers) after step COMB_AT."""
    h, L, E0, Psi = system()
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=TAU, k_taylor=6, k_qr=2)
    B = O.half_one_body_propagator(ham, TAU)
    wk = O.init_walkers(ham, Psi, count)
    out, moved = [], None
    for t in range(NSTEPS):
        x = philox_fields(SEED, t, W_TOTAL, L.shape[0])[offset:offset + count]
        E_L = O.local_energy(ham, Psi, wk.Phi)[0]
        out.append(D.partial_sums(wk.w, E_L))
        O.step(ham, Psi, B, wk, x, p)
        if t + 1 == COMB_AT and comb is not None and offset <= 4 < offset + count:
            wk.w[4 - offset] *= 3.0      # a heavy walker of rank 1 also fills a slot of rank 0
        if t + 1 == COMB_AT and comb == "single":
            O.population_control(wk, XI)
        elif t + 1 == COMB_AT and comb == "ranks":
            idx, counts, total = D.comb_across_ranks(wk.w, XI, comb=oracle_comb)
            P = np.concatenate([wk.Phi[0].reshape(count, -1), wk.Phi[1].reshape(count, -1), wk.logS[:, None]], axis=1)
            P = D.exchange_walkers(P, idx, counts)
            nu = wk.Phi[0][0].size
            wk.Phi = [P[:, :nu].reshape(wk.Phi[0].shape).copy(), P[:, nu:-1].reshape(wk.Phi[1].shape).copy()]
            wk.logS = P[:, -1].copy()
            wk.w = np.full(count, total / W_TOTAL)
            offs = np.concatenate([[0], np.cumsum(counts)])
            owner = np.searchsorted(offs, idx, side="right") - 1
            moved = int(np.sum(owner != np.searchsorted(offs, np.arange(W_TOTAL), side="right") - 1))
    return out, moved


def worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = D.shard(W_TOTAL, rank, world)
        trace = [D.combine_emix(ps) for ps in run_oracle(off, cnt)[0]]
        parts, moved = run_oracle(off, cnt, comb="ranks")
        trace_comb = [D.combine_emix(ps) for ps in parts]
        if rank == 0:
            q.put((trace, trace_comb, moved))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_population():
    for W, world in [(7, 2), (1024, 8), (5, 5), (100, 3)]:
        ranges = [D.shard(W, r, world) for r in range(world)]
        assert ranges[0][0] == 0
        assert all(a[0] + a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        assert ranges[-1][0] + ranges[-1][1] == W
        assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    with pytest.raises(ValueError):
        D.shard(3, 0, 4)


def test_two_rank_emix_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    trace, trace_comb, moved = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    single = [complex(*ps[:2]) / complex(*ps[2:]) for ps in run_oracle(0, W_TOTAL)[0]]
    assert np.max(np.abs(np.array(trace) - np.array(single))) < 1e-12 * max(abs(s) for s in single)
    # the comb over the whole population: walkers crossed ranks, and the trace is the one of a
    # single process combing all of its walkers
    assert moved > 0
    single_comb = [complex(*ps[:2]) / complex(*ps[2:]) for ps in run_oracle(0, W_TOTAL, comb="single")[0]]
    assert np.max(np.abs(np.array(trace_comb) - np.array(single_comb))) < 1e-12 * max(abs(s) for s in single_comb)
    assert np.max(np.abs(np.array(single_comb) - np.array(single))) > 1e-9     # the comb changed the run


def exchange_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        counts = np.array([3, 2, 4])
        offs = np.concatenate([[0], np.cumsum(counts)])
        idx = np.random.default_rng(4).integers(0, 9, size=9)    # with repeats and dropped walkers
        g = np.arange(offs[rank], offs[rank + 1])
        P = np.stack([g + 0.5j, -g + 0.25j, g * g + 0j], axis=1)   # one row per walker
        out = D.exchange_walkers(P, idx, counts)
        want = idx[offs[rank]:offs[rank + 1]]
        q.put((rank, bool(np.array_equal(out, np.stack([want + 0.5j, -want + 0.25j, want * want + 0j], axis=1)))))
    finally:
        dist.destroy_process_group()


def test_three_rank_walker_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=exchange_worker, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(3))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: True, 1: True, 2: True}


def run_bp_oracle(offset, count):
    """A back-propagation window of 3 steps after 1, for walkers [offset, offset + count):
    (G_up, G_dn, sum of the end-of-window weights)."""
    h, L, E0, Psi = system()
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=TAU, k_taylor=6, k_qr=2)
    B = O.half_one_body_propagator(ham, TAU)
    wk = O.init_walkers(ham, Psi, count)
    O.step(ham, Psi, B, wk, philox_fields(SEED, 0, W_TOTAL, L.shape[0])[offset:offset + count], p)
    win = BP.Window(wk.Phi)
    for t in range(1, 4):
        O.step(ham, Psi, B, wk, philox_fields(SEED, t, W_TOTAL, L.shape[0])[offset:offset + count], p,
               record=win.coefs)
    G = win.estimate(L, Psi, B, wk.w, TAU, 6)
    return G[0], G[1], np.sum(wk.w)


def bp_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = D.shard(W_TOTAL, rank, world)
        Gu, Gd, ws = run_bp_oracle(off, cnt)
        out = D.combine_rdm1(Gu, Gd, ws)
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


def test_two_rank_back_propagated_rdm1_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=bp_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    Gu, Gd = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Su, Sd, _ = run_bp_oracle(0, W_TOTAL)
    assert np.max(np.abs(Gu - Su)) < 1e-12 * np.max(np.abs(Su))
    assert np.max(np.abs(Gd - Sd)) < 1e-12 * np.max(np.abs(Sd))
