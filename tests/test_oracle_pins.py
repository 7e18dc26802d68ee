"""Pins of the CPU oracle against closed forms, brute force and library routines.

Each test checks one oracle function against something other than itself
(Sec. V, Eqs. (1), (3) and the phaseless algorithm the paper cites)."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import afqmc as O
from oracle.fock import four_index_from_cholesky
from oracle.philox import philox4x32_10, philox_fields
from paper_2003_01831_gb300 import synthetic as syn


def small_system(M=6, N=2, Nchol=12, seed=7):
    rng = np.random.default_rng(seed)
    h, L, _ = syn.make_hamiltonian(M, Nchol, rng, decay=6.0)
    ham = O.Hamiltonian(h=h, L=L, E0=0.37)
    Psi = syn.make_trial(h, N, N)
    return ham, Psi, rng


def random_complex(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_projector_idempotent_and_trace():
    ham, Psi, rng = small_system(M=9, N=3)
    Psi_c = Psi[0] + 0.3 * random_complex(rng, 9, 3)
    Phi = random_complex(rng, 4, 9, 3)
    Th = O.half_rotated_green(Psi_c, Phi)
    for w in range(4):
        P = Th[w] @ Psi_c.conj().T
        assert np.allclose(P @ P, P, atol=1e-12)
        assert abs(np.trace(P) - 3) < 1e-12


def test_hf_energy_matches_four_index_loops():
    """At Phi = Psi the mixed energy is the HF energy sum h P + 1/2 sum v (PP - PP_exch)."""
    ham, Psi, rng = small_system(M=6, N=2, Nchol=10)
    v = four_index_from_cholesky(ham.L)
    # spin density matrices P_s[k, i] = <c+_i c_k> for an orthonormal determinant
    Ps = [p @ p.conj().T for p in Psi]
    M = ham.M
    E = ham.E0
    for s in range(2):
        for i in range(M):
            for k in range(M):
                E += ham.h[i, k] * Ps[s][k, i]
    for s in range(2):
        for s2 in range(2):
            for i, j, k, l in itertools.product(range(M), repeat=4):
                E += 0.5 * v[i, j, k, l] * Ps[s][k, i] * Ps[s2][l, j]
                if s == s2:
                    E -= 0.5 * v[i, j, k, l] * Ps[s][l, i] * Ps[s][k, j]
    EL, _, _ = O.local_energy(ham, Psi, [p[None] for p in Psi])
    assert abs(EL[0] - E) < 1e-12 * max(1.0, abs(E))


def test_gauge_invariance_energy_and_logdet():
    ham, Psi, rng = small_system(M=7, N=3, Nchol=14)
    Phi = [random_complex(rng, 3, 7, 3) for _ in range(2)]
    R = [random_complex(rng, 3, 3, 3) for _ in range(2)]
    PhiR = [np.matmul(Phi[s], R[s]) for s in range(2)]
    E1, _, _ = O.local_energy(ham, Psi, Phi)
    E2, _, _ = O.local_energy(ham, Psi, PhiR)
    assert np.allclose(E1, E2, rtol=1e-11, atol=1e-11)
    for s in range(2):
        l1 = O.log_det(O.overlap_matrix(Psi[s], Phi[s]))
        l2 = O.log_det(O.overlap_matrix(Psi[s], PhiR[s]))
        lr = O.log_det(R[s])
        d = l2 - l1 - lr
        assert np.allclose(d.real, 0, atol=1e-11)
        assert np.allclose(np.exp(1j * d.imag), 1, atol=1e-11)


def test_force_bias_matches_full_green_function():
    """<L_n> = sum_s sum_ik L_ik G_s[k, i] with the full M x M mixed density."""
    ham, Psi, rng = small_system(M=8, N=3, Nchol=9)
    Phi = [random_complex(rng, 2, 8, 3) for _ in range(2)]
    _, t_sum, _ = O.local_energy(ham, Psi, Phi)
    for w in range(2):
        ref = np.zeros(ham.Nchol, dtype=complex)
        for s in range(2):
            S = Psi[s].conj().T @ Phi[s][w]
            G = Phi[s][w] @ np.linalg.inv(S) @ Psi[s].conj().T      # G[k, i] = <c+_i c_k>
            for n in range(ham.Nchol):
                ref[n] += np.sum(ham.L[n] * G.T)
        assert np.allclose(t_sum[w], ref, rtol=1e-12, atol=1e-12)
    tau, cap = 0.01, 0.05
    xb = O.force_bias(t_sum, tau, cap)
    raw = -1j * np.sqrt(tau) * t_sum
    assert np.all(np.abs(xb) <= cap + 1e-15)
    small = np.abs(raw) <= cap
    assert np.allclose(xb[small], raw[small])
    assert np.allclose(np.angle(xb[~small]), np.angle(raw[~small]))


def leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        term = (-1) ** inv
        for i in range(n):
            term = term * A[i, perm[i]]
        tot += term
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_log_det_matches_leibniz(n):
    rng = np.random.default_rng(n)
    S = random_complex(rng, 5, n, n)
    ld = O.log_det(S)
    for w in range(5):
        d = leibniz_det(S[w])
        assert abs(np.exp(ld[w]) - d) < 1e-12 * abs(d)


def test_taylor_matches_eigendecomposition_and_expm():
    """K = 16 Taylor of i sqrt(tau) A applied to Phi vs exact exponentials (||sqrt(tau) A|| < 1)."""
    ham, Psi, rng = small_system(M=10, N=3, Nchol=20)
    tau = 0.01
    x = rng.standard_normal((2, ham.Nchol))
    A = O.hs_potential(x.astype(complex), ham.L)          # real symmetric per walker
    Phi = random_complex(rng, 2, 10, 3)
    for w in range(2):
        assert np.linalg.norm(np.sqrt(tau) * A[w], 2) < 1.0
        got = O.taylor_exp_apply(1j * np.sqrt(tau) * A[w:w + 1], Phi[w:w + 1], 16)[0]
        e, V = np.linalg.eigh(A[w].real)
        ref = (V * np.exp(1j * np.sqrt(tau) * e)) @ V.T @ Phi[w]
        ref2 = scipy.linalg.expm(1j * np.sqrt(tau) * A[w]) @ Phi[w]
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(got - ref2)) < 1e-12 * np.max(np.abs(ref))


def test_zero_field_one_body_step_is_exp_minus_tau_h():
    """L = 0 and x = 0: one step maps Phi to exp(-tau h) Phi exactly and the weight to
    |<Psi|Phi'>/<Psi|Phi>| exp(tau (E_T - E0))."""
    rng = np.random.default_rng(3)
    M, N = 8, 3
    h, _, _ = syn.make_hamiltonian(M, 1, rng)
    ham = O.Hamiltonian(h=h, L=np.zeros((4, M, M)), E0=0.0)
    Psi = syn.make_trial(h, N, N)
    Phi0 = [syn.make_random_walkers(M, N, 3, seed=s) for s in (11, 12)]
    p = O.Params(tau=0.05, k_taylor=6, k_qr=0)
    B = O.half_one_body_propagator(ham, p.tau)
    wk = O.init_walkers(ham, Psi, 3, Phi0)
    logS0 = wk.logS.copy()
    O.step(ham, Psi, B, wk, np.zeros((3, 4)), p)
    E = scipy.linalg.expm(-p.tau * h)
    for s in range(2):
        assert np.allclose(wk.Phi[s], np.matmul(E, Phi0[s]), rtol=1e-13, atol=1e-14)
    dl = wk.logS - logS0
    expect = np.exp(dl.real + p.tau * wk.E_T) * np.maximum(0, np.cos(dl.imag))
    assert np.allclose(wk.w, expect, rtol=1e-13)


def test_hprime_against_loops():
    ham, _, _ = small_system(M=5, N=2, Nchol=7)
    hp = O.hprime(ham)
    v = four_index_from_cholesky(ham.L)
    ref = ham.h.copy()
    for i in range(5):
        for l in range(5):
            ref[i, l] -= 0.5 * sum(v[i, k, k, l] for k in range(5))
    assert np.allclose(hp, ref, atol=1e-14)


def test_qr_properties_and_energy_unchanged():
    ham, Psi, rng = small_system(M=9, N=4, Nchol=11)
    Phi = random_complex(rng, 3, 9, 4)
    Q, ldr = O.qr_reorthonormalise(Phi)
    for w in range(3):
        R = Q[w].conj().T @ Phi[w]
        assert np.allclose(Q[w].conj().T @ Q[w], np.eye(4), atol=1e-13)
        assert np.allclose(Q[w] @ R, Phi[w], atol=1e-12)
        assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
        d = np.diag(R)
        assert np.all(d.real > 0) and np.allclose(d.imag, 0, atol=1e-12)
        assert abs(np.sum(np.log(d.real)) - ldr[w]) < 1e-12
    E1, _, _ = O.local_energy(ham, Psi, [Phi, Phi])
    E2, _, _ = O.local_energy(ham, Psi, [Q, Q])
    assert np.allclose(E1, E2, rtol=1e-11)


def _load_kat():
    """Philox4x32-10 known-answer vectors from tests/golden (Random123, Salmon et al. SC'11)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((tuple(v[0:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


PHILOX_KAT = _load_kat()


@pytest.mark.parametrize("ctr,key,expect", PHILOX_KAT)
def test_philox_known_answers(ctr, key, expect):
    out = philox4x32_10(tuple(np.uint64(c) for c in ctr), tuple(np.uint64(k) for k in key))
    assert tuple(int(o) for o in out) == expect


def test_philox_fields_are_standard_normal():
    x = philox_fields(seed=5, step=3, W=64, Nchol=1001)
    assert x.shape == (64, 1001)
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 1) < 0.03
    # different steps / seeds give different fields; same arguments reproduce
    assert not np.allclose(x, philox_fields(5, 4, 64, 1001))
    assert np.array_equal(x, philox_fields(5, 3, 64, 1001))
