"""Pin the oracle's energy/log-overlap adjoint against central finite differences."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.adjoint import energy_logdet_backward
from paper_2003_01831_gb300 import synthetic as syn


def loss(ham, Psi, Phi, dE, dlogS):
    E, _, _ = O.local_energy(ham, Psi, Phi)
    lS = sum(O.log_det(O.overlap_matrix(Psi[s], Phi[s])) for s in range(2))
    return np.sum(np.real(np.conj(dE) * E + np.conj(dlogS) * lS))


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(44)
    M, N, nch, W = 16, 4, 80, 3
    h, L, _ = syn.make_hamiltonian(M, nch, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=0.1)
    Psi = syn.make_trial(h, N, N)
    Psi = [p + 0.1 * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)) for p in Psi]
    Phi = [syn.make_random_walkers(M, N, W, seed=s) for s in (1, 2)]
    dE = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    dlogS = rng.standard_normal(W) + 1j * rng.standard_normal(W)
    grads = energy_logdet_backward(ham, Psi, Phi, dE, dlogS)
    return ham, Psi, Phi, dE, dlogS, grads, rng


def test_psi_gradient_matches_central_differences(case):
    ham, Psi, Phi, dE, dlogS, grads, rng = case
    eps = 1e-6
    for s in range(2):
        g = grads[s]
        for (i, a) in [(0, 0), (3, 1), (7, 2), (15, 3), (9, 0)]:
            for part, unit in (("re", 1.0), ("im", 1j)):
                Pp = [p.copy() for p in Psi]
                Pm = [p.copy() for p in Psi]
                Pp[s][i, a] += eps * unit
                Pm[s][i, a] -= eps * unit
                fd = (loss(ham, Pp, Phi, dE, dlogS) - loss(ham, Pm, Phi, dE, dlogS)) / (2 * eps)
                an = g[i, a].real if part == "re" else g[i, a].imag
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (s, i, a, part, fd, an)


def test_L_gradient_matches_central_differences(case):
    ham, Psi, Phi, dE, dlogS, grads, rng = case
    dL = grads[2]
    eps = 1e-6
    for (n, i, k) in [(0, 0, 0), (0, 2, 5), (5, 7, 3), (40, 11, 11), (79, 15, 2)]:
        Lp = ham.L.copy(); Lp[n, i, k] += eps
        Lm = ham.L.copy(); Lm[n, i, k] -= eps
        fp = loss(O.Hamiltonian(ham.h, Lp, ham.E0), Psi, Phi, dE, dlogS)
        fm = loss(O.Hamiltonian(ham.h, Lm, ham.E0), Psi, Phi, dE, dlogS)
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - dL[n, i, k]) < 1e-6 * max(1.0, abs(fd)), (n, i, k, fd, dL[n, i, k])
    # one random direction over the whole tensor
    D = rng.standard_normal(ham.L.shape)
    fp = loss(O.Hamiltonian(ham.h, ham.L + eps * D, ham.E0), Psi, Phi, dE, dlogS)
    fm = loss(O.Hamiltonian(ham.h, ham.L - eps * D, ham.E0), Psi, Phi, dE, dlogS)
    fd = (fp - fm) / (2 * eps)
    assert abs(fd - np.sum(dL * D)) < 1e-6 * max(1.0, abs(fd))


def test_gradient_orthogonal_to_gauge_directions(case):
    """logS and E_L depend on Psi only through its column space up to det factors:
    a change Psi -> Psi (I + eps R) changes E_L by zero, so <grad_E, Psi R> = 0."""
    ham, Psi, Phi, dE, dlogS, grads, rng = case
    W = len(dE)
    g = energy_logdet_backward(ham, Psi, Phi, dE, np.zeros(W, complex))
    for s in range(2):
        R = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
        D = Psi[s] @ R
        inner = np.sum(np.real(np.conj(g[s]) * D))
        assert abs(inner) < 1e-9 * np.linalg.norm(g[s]) * np.linalg.norm(D)
