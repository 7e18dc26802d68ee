"""GPU adjoint (afqmc_energy_backward) vs the oracle's adjoint and central differences."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.adjoint import energy_logdet_backward
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu


def instance(M, N, nch, W, seed, noise=0.1):
    rng = np.random.default_rng(seed)
    h, L, _ = syn.make_hamiltonian(M, nch, rng)
    E0 = 0.3
    Psi = [p + noise * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape))
           for p in syn.make_trial(h, N, N)]
    Phi = [syn.make_random_walkers(M, N, W, seed + 1), syn.make_random_walkers(M, N, W, seed + 2)]
    dE = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    dS = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    return h, L, E0, Psi, Phi, dE, dS


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("M,N,nch,W", [(16, 4, 80, 3), (40, 7, 60, 5)])
def test_backward_matches_oracle(M, N, nch, W):
    h, L, E0, Psi, Phi, dE, dS = instance(M, N, nch, W, 31)
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi) as g:
        dPu, dPd, dL = g.backward(dE, dS)
    ref = energy_logdet_backward(O.Hamiltonian(h, L, E0), Psi, Phi, dE, dS)
    assert rel(dPu, ref[0]) < 1e-10
    assert rel(dPd, ref[1]) < 1e-10
    assert rel(dL, ref[2]) < 1e-10


def test_backward_matches_central_differences():
    """M=16, N=4, Nchol=80: GPU gradient against central differences of the GPU energy."""
    M, N, nch, W = 16, 4, 80, 3
    h, L, E0, Psi, Phi, dE, dS = instance(M, N, nch, W, 44)

    def loss(Pu, Pd, LL):
        with AFQMC(h, LL, E0, Pu, Pd, W, 0.01, Phi0=Phi) as g:
            E, _, lS, _ = g.energy()
        return np.sum(np.real(np.conj(dE) * E + np.conj(dS) * lS))

    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi) as g:
        dPu, dPd, dL = g.backward(dE, dS)
    eps = 1e-6
    for (i, a) in [(0, 0), (5, 2), (15, 3)]:
        for unit in (1.0, 1j):
            P1 = Psi[0].copy(); P1[i, a] += eps * unit
            P2 = Psi[0].copy(); P2[i, a] -= eps * unit
            fd = (loss(P1, Psi[1], L) - loss(P2, Psi[1], L)) / (2 * eps)
            an = dPu[i, a].real if unit == 1.0 else dPu[i, a].imag
            assert abs(fd - an) < 1e-6 * max(1, abs(an)), (i, a, unit, fd, an)
    for (n, i, k) in [(0, 1, 2), (40, 7, 7), (79, 15, 0)]:
        L1 = L.copy(); L1[n, i, k] += eps; L1[n, k, i] += eps * (i != k)
        L2 = L.copy(); L2[n, i, k] -= eps; L2[n, k, i] -= eps * (i != k)
        fd = (loss(Psi[0], Psi[1], L1) - loss(Psi[0], Psi[1], L2)) / (2 * eps)
        an = dL[n, i, k] + (dL[n, k, i] if i != k else 0.0)   # symmetric perturbation
        assert abs(fd - an) < 1e-6 * max(1, abs(an)), (n, i, k, fd, an)


def test_backward_m256_workload_sampled():
    """Differentiation workload sizes (M=256, N=64+64, Nchol=1280) at 2 walkers vs the oracle."""
    wl = syn.WORKLOADS["m256"]
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng)
    Psi = [p + 0.1 * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape))
           for p in syn.make_trial(h, wl.Nup, wl.Ndn)]
    W = 2
    Phi = []
    for s in range(2):
        z = Psi[s][None] + 0.1 * (rng.standard_normal((W, wl.M, wl.Nup)) + 1j * rng.standard_normal((W, wl.M, wl.Nup)))
        Phi.append(np.linalg.qr(z)[0])
    dE = np.array([1.0 + 0.5j, -0.3 + 0.2j])
    dS = np.array([0.2 - 0.1j, 0.7 + 0.0j])
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, Phi0=Phi) as g:
        dPu, dPd, dL = g.backward(dE, dS)
    ref = energy_logdet_backward(O.Hamiltonian(h, L, E0), Psi, Phi, dE, dS)
    assert rel(dPu, ref[0]) < 1e-10 and rel(dPd, ref[1]) < 1e-10
    assert rel(dL, ref[2]) < 1e-10


def test_autograd_function_matches_oracle():
    import torch
    from paper_2003_01831_gb300.autograd import local_energy
    M, N, nch, W = 12, 3, 30, 4
    h, L, E0, Psi, Phi, dE, dS = instance(M, N, nch, W, 9)
    Pu = torch.tensor(Psi[0], requires_grad=True)
    Pd = torch.tensor(Psi[1], requires_grad=True)
    Lt = torch.tensor(L, requires_grad=True)
    E, lS = local_energy(Pu, Pd, Lt, torch.tensor(h), E0, torch.tensor(Phi[0]), torch.tensor(Phi[1]))
    loss = torch.sum(torch.real(torch.conj(torch.tensor(dE)) * E + torch.conj(torch.tensor(dS)) * lS))
    loss.backward()
    ref = energy_logdet_backward(O.Hamiltonian(h, L, E0), Psi, Phi, dE, dS)
    assert rel(Pu.grad.numpy(), ref[0]) < 1e-10
    assert rel(Pd.grad.numpy(), ref[1]) < 1e-10
    assert rel(Lt.grad.numpy(), ref[2]) < 1e-10
    E_ref = O.local_energy(O.Hamiltonian(h, L, E0), Psi, Phi)[0]
    assert rel(E.detach().numpy(), E_ref) < 1e-10


def test_autograd_on_device_tensors_reuses_the_hamiltonian():
    """CUDA tensors in, CUDA gradients out (no host round trip); two calls with the same L and h
    share one library Hamiltonian, and changing L in place builds a new one."""
    import torch
    from paper_2003_01831_gb300 import autograd as A
    M, N, nch, W = 12, 3, 30, 4
    h, L, E0, Psi, Phi, dE, dS = instance(M, N, nch, W, 11)
    dev = torch.device("cuda", 0)
    Lt = torch.tensor(L, device=dev, requires_grad=True)
    ht = torch.tensor(h, device=dev)
    Ph = [torch.tensor(p, device=dev) for p in Phi]
    ref = energy_logdet_backward(O.Hamiltonian(h, L, E0), Psi, Phi, dE, dS)
    hams = []
    for it in range(2):
        Pu = torch.tensor(Psi[0], device=dev, requires_grad=True)
        Pd = torch.tensor(Psi[1], device=dev, requires_grad=True)
        E, lS = A.local_energy(Pu, Pd, Lt, ht, E0, Ph[0], Ph[1])
        assert E.is_cuda and lS.is_cuda
        loss = torch.sum(torch.real(torch.conj(torch.tensor(dE, device=dev)) * E +
                                    torch.conj(torch.tensor(dS, device=dev)) * lS))
        Lt.grad = None
        loss.backward()
        assert Pu.grad.is_cuda and Lt.grad.is_cuda
        assert rel(Pu.grad.cpu().numpy(), ref[0]) < 1e-10
        assert rel(Lt.grad.cpu().numpy(), ref[2]) < 1e-10
        hams.append(A._cache["ham"])
    assert hams[0] is hams[1]
    with torch.no_grad():
        Lt.mul_(1.0)                                 # in-place: new version, new Hamiltonian
    A.local_energy(torch.tensor(Psi[0], device=dev), torch.tensor(Psi[1], device=dev), Lt, ht, E0, Ph[0], Ph[1])
    assert A._cache["ham"] is not hams[0]
