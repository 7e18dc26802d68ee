"""General complex Cholesky vectors (Sec. V, Eq. (3): v_ijkl = sum_n L^n_ik L^n*_lj with complex
L_n) in the oracle, through the Hermitian split A_n = (L_n + L_n^+)/2, B_n = (L_n - L_n^+)/(2i).

Pinned against brute-force Fock-space quantum mechanics built from the complex L itself:
* the split Cholesky vectors give the same Hamiltonian matrix;
* the oracle's local energy and force bias on the split vectors are the Fock-space mixed
  estimates;
* the Hubbard-Stratonovich average over the two fields of each split pair reproduces
  <Psi|exp(-tau (H - E0))|Phi> up to O(tau^2) (A_n and B_n do not commute), and dropping B_n
  leaves an O(tau) error."""
import numpy as np
import pytest
import scipy.linalg

from oracle import afqmc as O
from oracle.fock import FockSpace, four_index_from_cholesky
from paper_2003_01831_gb300 import synthetic as syn


def random_complex(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def complex_system(M, N, Nchol, seed, scale=0.6):
    rng = np.random.default_rng(seed)
    h, _, _ = syn.make_hamiltonian(M, 1, rng)
    L = scale * random_complex(rng, Nchol, M, M) / np.sqrt(M)    # neither Hermitian nor symmetric
    Psi = syn.make_trial(h, N, N)
    return h, L, Psi, rng


def test_split_is_the_same_two_body_operator():
    h, L, Psi, rng = complex_system(4, 2, 3, seed=1)
    Ms = O.hermitian_split(L)
    for m in Ms:
        assert np.allclose(m, m.conj().T)
    fs = FockSpace(4, 2, 2)
    H_L = fs.hamiltonian(h, four_index_from_cholesky(L), 0.3)
    H_M = fs.hamiltonian(h, four_index_from_cholesky(Ms), 0.3)
    assert np.max(np.abs(H_L - H_M)) < 1e-12 * np.max(np.abs(H_L))
    assert np.allclose(H_L, H_L.conj().T)
    # the squares of the split operators carry h' = h - 1/4 sum (L L^+ + L^+ L), which differs
    # from h - 1/2 sum L L^+ by the commutator term 1/4 sum [L, L^+]
    Ld = np.conj(np.swapaxes(L, 1, 2))
    expect = h - 0.25 * np.einsum("nik,nkj->ij", L, Ld) - 0.25 * np.einsum("nik,nkj->ij", Ld, L)
    assert np.allclose(O.hprime(O.Hamiltonian(h=h, L=Ms, E0=0.0)), expect, atol=1e-13)
    comm = 0.25 * (np.einsum("nik,nkj->ij", L, Ld) - np.einsum("nik,nkj->ij", Ld, L))
    assert np.allclose(O.hprime(O.Hamiltonian(h=h, L=L, E0=0.0)) + comm, expect, atol=1e-13)


@pytest.fixture(scope="module")
def sys6c():
    h, L, Psi, rng = complex_system(6, 2, 4, seed=7)
    Psi = [Psi[0] + 0.2 * random_complex(rng, 6, 2), Psi[1] + 0.2 * random_complex(rng, 6, 2)]
    fs = FockSpace(6, 2, 2)
    H = fs.hamiltonian(h, four_index_from_cholesky(L), 0.25)
    ham = O.Hamiltonian(h=h, L=O.hermitian_split(L), E0=0.25)
    return ham, Psi, fs, H, rng


def test_local_energy_matches_fock_with_complex_L(sys6c):
    ham, Psi, fs, H, rng = sys6c
    Phi = [random_complex(rng, 3, 6, 2) for _ in range(2)]
    EL, _, _ = O.local_energy(ham, Psi, Phi)
    vp = fs.slater_vector(Psi[0], Psi[1])
    for w in range(3):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ref = np.vdot(vp, H @ vf) / np.vdot(vp, vf)
        assert abs(EL[w] - ref) < 1e-11 * max(1, abs(ref))


def test_force_bias_matches_fock_with_complex_L(sys6c):
    ham, Psi, fs, H, rng = sys6c
    Phi = [random_complex(rng, 2, 6, 2) for _ in range(2)]
    _, t_sum, _ = O.local_energy(ham, Psi, Phi)
    vp = fs.slater_vector(Psi[0], Psi[1])
    for w in range(2):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ov = np.vdot(vp, vf)
        for m in range(ham.Nchol):
            Mm = fs.one_body_operator(ham.L[m])
            assert abs(t_sum[w, m] - np.vdot(vp, Mm @ vf) / ov) < 1e-11


def hs_pair_error(ham, Psi, Phi, fs, H, tau, nodes=32):
    """| E_{x_a, x_b} <Psi|B exp(i sqrt(tau) (x_a A + x_b B)) B|Phi> - <Psi|exp(-tau (H - E0))|Phi> |
    for one split pair (2-D Gauss-Hermite quadrature; high Taylor order)."""
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)
    ws = ws / np.sqrt(2 * np.pi)
    X = np.array([[xa, xb] for xa in xs for xb in xs], dtype=np.complex128)
    Wq = np.array([wa * wb for wa in ws for wb in ws])
    B = O.half_one_body_propagator(ham, tau)
    A = O.hs_potential(X, ham.L)
    acc = 0.0
    for s0 in range(0, len(X), 256):
        sl = slice(s0, s0 + 256)
        n = len(X[sl])
        ov = sum(O.log_det(O.overlap_matrix(Psi[s], O.propagate(np.repeat(Phi[s][None], n, 0), A[sl], B, tau, 40)))
                 for s in range(2))
        acc += np.sum(Wq[sl] * np.exp(ov))
    vp = fs.slater_vector(Psi[0], Psi[1])
    vf = fs.slater_vector(Phi[0], Phi[1])
    ref = np.vdot(vp, scipy.linalg.expm(-tau * (H - ham.E0 * np.eye(fs.dim))) @ vf)
    return abs(acc - ref), abs(ref)


def test_hs_with_a_split_pair_against_exact_propagation():
    h, L, Psi, rng = complex_system(5, 2, 1, seed=3, scale=1.0)
    Phi = [random_complex(rng, 5, 2) for _ in range(2)]
    fs = FockSpace(5, 2, 2)
    H = fs.hamiltonian(h, four_index_from_cholesky(L))
    ham = O.Hamiltonian(h=h, L=O.hermitian_split(L), E0=0.0)
    e1, r1 = hs_pair_error(ham, Psi, Phi, fs, H, 0.01)
    e2, r2 = hs_pair_error(ham, Psi, Phi, fs, H, 0.005)
    print(f"split-pair HS: error {e1 / r1:.2e} at tau 0.01, {e2 / r2:.2e} at 0.005, ratio {e1 / e2:.2f}")
    assert e1 / r1 < 2e-3
    assert 3.3 < e1 / e2 < 4.8          # O(tau^2) (A and B do not commute), not O(tau)
    # negative control: the A part alone misses half the interaction -- an O(tau) error
    half = O.Hamiltonian(h=h, L=O.hermitian_split(L)[0:1], E0=0.0)
    f1, q1 = hs_pair_error_single(half, Psi, Phi, fs, H, 0.01)
    f2, q2 = hs_pair_error_single(half, Psi, Phi, fs, H, 0.005)
    assert f1 / f2 < 2.5 and f2 / q2 > 10 * e2 / r2


def hs_pair_error_single(ham, Psi, Phi, fs, H, tau, nodes=40):
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)
    ws = ws / np.sqrt(2 * np.pi)
    B = O.half_one_body_propagator(ham, tau)
    A = O.hs_potential(xs[:, None].astype(np.complex128), ham.L)
    ov = sum(O.log_det(O.overlap_matrix(Psi[s], O.propagate(np.repeat(Phi[s][None], nodes, 0), A, B, tau, 40)))
             for s in range(2))
    acc = np.sum(ws * np.exp(ov))
    vp = fs.slater_vector(Psi[0], Psi[1])
    vf = fs.slater_vector(Phi[0], Phi[1])
    ref = np.vdot(vp, scipy.linalg.expm(-tau * (H - ham.E0 * np.eye(fs.dim))) @ vf)
    return abs(acc - ref), abs(ref)


def test_phaseless_step_runs_with_complex_L():
    """A short phaseless run on split complex Cholesky vectors: finite weights and energies."""
    h, L, Psi, rng = complex_system(6, 2, 3, seed=11, scale=0.4)
    ham = O.Hamiltonian(h=h, L=O.hermitian_split(L), E0=0.0)
    p = O.Params(tau=0.01, k_taylor=6, k_qr=2)
    x = rng.standard_normal((6, 4, ham.Nchol))
    out = O.run(ham, Psi, 4, x, p)
    assert np.all(np.isfinite(np.array(out["E_mix"])))
    assert np.all(out["walkers"].w > 0)
