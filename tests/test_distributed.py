"""Walker-parallel host logic on CPU with gloo, world size 2: each rank steps its shard of the
population (the oracle stands in for its GPU), the partial sums are all-reduced, and the
combined E_mix trace equals that of one process stepping every walker."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import afqmc as O
from oracle.philox import philox_fields
from paper_2003_01831_gb300 import distributed as D
from paper_2003_01831_gb300 import synthetic as syn

W_TOTAL, NSTEPS, SEED, TAU = 7, 4, 21, 0.01


def system():
    d = syn.UnevenSystem(M=8, N=2, Nchol=12, W=W_TOTAL)
    h, L, E0, Psi = syn.make_uneven_system(d, 0, seed=5)
    return h, L, E0, Psi


def run_oracle(offset, count):
    """E_mix partial sums per step for walkers [offset, offset + count)."""
    h, L, E0, Psi = system()
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=TAU, k_taylor=6, k_qr=2)
    B = O.half_one_body_propagator(ham, TAU)
    wk = O.init_walkers(ham, Psi, count)
    out = []
    for t in range(NSTEPS):
        x = philox_fields(SEED, t, W_TOTAL, L.shape[0])[offset:offset + count]
        E_L = O.local_energy(ham, Psi, wk.Phi)[0]
        out.append(D.partial_sums(wk.w, E_L))
        O.step(ham, Psi, B, wk, x, p)
    return out


def worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        off, cnt = D.shard(W_TOTAL, rank, world)
        trace = [D.combine_emix(ps) for ps in run_oracle(off, cnt)]
        if rank == 0:
            q.put(trace)
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
    trace = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    single = [complex(*ps[:2]) / complex(*ps[2:]) for ps in run_oracle(0, W_TOTAL)]
    assert np.max(np.abs(np.array(trace) - np.array(single))) < 1e-12 * max(abs(s) for s in single)
