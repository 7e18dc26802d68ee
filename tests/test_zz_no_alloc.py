"""The allocation-free log-overlap entry point against afqmc_energy's log-overlaps.

afqmc_log_overlap_noalloc serves callers that must not allocate device memory when they
call it (a service whose memory pool owns the whole device, or a latency-critical loop
that must stay off the allocator).  It keeps its scratch in a fixed device array inside
the library; this test calls it twice in a row through the C ABI (device buffers) and
compares both results with the log-overlaps the regular walker-set path reports."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu


def test_noalloc_log_overlap_matches_energy_entry_point():
    import torch
    from paper_2003_01831_gb300 import build
    build.build()
    rng = np.random.default_rng(12)
    M, Nup, Ndn, nch, W = 40, 6, 5, 30, 7
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = list(syn.make_trial(h, Nup, Ndn))
    Psi = [p + 0.1 * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)) for p in Psi]
    Phi0 = [syn.make_random_walkers(M, Nup, W, 1), syn.make_random_walkers(M, Ndn, W, 2)]
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi0) as g:
        _, _, ref, _ = g.energy()
    dev = torch.device("cuda", 0)
    Pu = torch.from_numpy(np.ascontiguousarray(Psi[0])).to(dev)
    Pd = torch.from_numpy(np.ascontiguousarray(Psi[1])).to(dev)
    Phi = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([Phi0[0].reshape(W, -1), Phi0[1].reshape(W, -1)], axis=1))).to(dev)
    for call in range(2):
        out = torch.zeros(W, dtype=torch.complex128, device=dev)
        api.afqmc_log_overlap_noalloc(Pu, Pd, Nup, Ndn, M, W, Phi, out,
                                      stream=torch.cuda.current_stream().cuda_stream)
        got = out.cpu().numpy()
        assert np.max(np.abs(got.real - ref.real)) < 1e-10 * np.max(np.abs(ref.real)) + 1e-12, call
        assert np.max(np.abs(np.exp(1j * (got.imag - ref.imag)) - 1)) < 1e-9, call


def test_noalloc_rejects_oversize_and_host_pointers():
    import torch
    dev = torch.device("cuda", 0)
    M, N = 128, 128
    W = 40                                   # 40 * (2 * 128^2 + 2) * 16 bytes > 16 MiB
    Pu = torch.zeros((M, N), dtype=torch.complex128, device=dev)
    Phi = torch.zeros((W, 2 * M * N), dtype=torch.complex128, device=dev)
    out = torch.zeros(W, dtype=torch.complex128, device=dev)
    with pytest.raises(api.AfqmcError) as e:
        api.afqmc_log_overlap_noalloc(Pu, Pu, N, N, M, W, Phi, out)
    assert e.value.code == -2
    with pytest.raises(api.AfqmcError) as e:
        api.afqmc_log_overlap_noalloc(Pu.cpu(), Pu, N, N, M, 1, Phi, out)
    assert e.value.code == -1
