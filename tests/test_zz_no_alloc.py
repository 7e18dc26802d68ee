"""The allocation-free log-overlap entry point against afqmc_energy's log-overlaps.

afqmc_log_overlap_noalloc serves callers that must not allocate device memory when they
call it (a service whose memory pool owns the whole device, or a latency-critical loop
that must stay off the allocator).  It keeps its scratch in a fixed device array inside
the library.  These tests call it through the C ABI (device buffers), several times in a
row, and compare every result with the log-overlaps the regular walker-set path reports;
they also check that a warm call leaves the device's free memory unchanged.  The shapes
reach each Gauss-Jordan variant the entry point can run: the one-CTA shared-memory kernel
(N <= 96), its two-CTA cluster form (97 <= N <= 128) and the general kernel for N > 128,
where no walker set exists to compare with and the reference is the log-determinant of
Psi^+ Phi itself."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu


def device_inputs(Psi, Phi0, W):
    import torch
    dev = torch.device("cuda", 0)
    Pu = torch.from_numpy(np.ascontiguousarray(Psi[0])).to(dev)
    Pd = torch.from_numpy(np.ascontiguousarray(Psi[1])).to(dev)
    Phi = torch.from_numpy(np.ascontiguousarray(
        np.concatenate([Phi0[0].reshape(W, -1), Phi0[1].reshape(W, -1)], axis=1))).to(dev)
    return Pu, Pd, Phi


def calls_match(Pu, Pd, Nup, Ndn, M, W, Phi, ref, ncalls=3):
    """ncalls calls in a row, each compared with ref; from the second call on, the device's
    free memory before and after the call must be the same."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(ncalls):
        out = torch.zeros(W, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        api.afqmc_log_overlap_noalloc(Pu, Pd, Nup, Ndn, M, W, Phi, out, stream=stream)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if call > 0:
            assert free1 == free0, (call, free0, free1)
        got = out.cpu().numpy()
        assert np.max(np.abs(got.real - ref.real)) < 1e-10 * np.max(np.abs(ref.real)) + 1e-12, call
        assert np.max(np.abs(np.exp(1j * (got.imag - ref.imag)) - 1)) < 1e-9, call


@pytest.mark.parametrize("M,Nup,Ndn,nch,W", [(40, 6, 5, 30, 7), (160, 120, 118, 16, 6)])
def test_noalloc_log_overlap_matches_energy_entry_point(M, Nup, Ndn, nch, W):
    from paper_2003_01831_gb300 import build
    build.build()
    rng = np.random.default_rng(12)
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = list(syn.make_trial(h, Nup, Ndn))
    Psi = [p + 0.1 * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)) for p in Psi]
    Phi0 = [syn.make_random_walkers(M, Nup, W, 1), syn.make_random_walkers(M, Ndn, W, 2)]
    Phi0 = [p + 0.5 * Psi[s][None] for s, p in enumerate(Phi0)]   # overlaps well conditioned
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi0) as g:
        _, _, ref, _ = g.energy()
    Pu, Pd, Phi = device_inputs(Psi, Phi0, W)
    calls_match(Pu, Pd, Nup, Ndn, M, W, Phi, ref)


def test_noalloc_log_overlap_beyond_walker_set_sizes():
    """N = 160 and 150 (above the walker sets' 128): the log-determinant of Psi^+ Phi."""
    rng = np.random.default_rng(13)
    M, Nup, Ndn, W = 200, 160, 150, 4
    Psi = [syn.make_random_walkers(M, n, 1, 5 + n)[0] for n in (Nup, Ndn)]
    Phi0 = [syn.make_random_walkers(M, Nup, W, 3), syn.make_random_walkers(M, Ndn, W, 4)]
    Phi0 = [p + 0.5 * Psi[s][None] for s, p in enumerate(Phi0)]   # overlaps well away from zero
    ref = np.zeros(W, dtype=np.complex128)
    for s in range(2):
        sign, la = np.linalg.slogdet(np.einsum("ka,wkb->wab", Psi[s].conj(), Phi0[s]))
        ref += la + 1j * np.angle(sign)
    Pu, Pd, Phi = device_inputs(Psi, Phi0, W)
    calls_match(Pu, Pd, Nup, Ndn, M, W, Phi, ref)


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
