"""Pins of the THC oracle (oracle/thc.py; Sec. V, Eqs. (4)-(6)).

* The four-index tensor of Eq. (5), by explicit loops, equals the one rebuilt from the
  structured Cholesky vectors L^n = X^* diag(U_n) X^T with M = U U^+ (Eq. (3) form).
* The direct THC local energy (Wick contraction over the interpolating points, no L^n formed)
  equals the Cholesky-form local energy and the Fock-space matrix element <Psi|H|Phi>/<Psi|Phi>
  of the Hamiltonian built from Eq. (5), for complex orbitals.
* The THC force bias and HS potential equal their Cholesky forms; real orbitals give real
  symmetric vectors, which the real-L paths take as they are."""
import numpy as np

from oracle import afqmc as O
from oracle import thc as T
from oracle.fock import FockSpace, four_index_from_cholesky
from paper_2003_01831_gb300 import synthetic as syn


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_four_index_tensor_from_the_thc_cholesky_vectors():
    rng = np.random.default_rng(1)
    X, Mmat = syn.make_thc(3, 5, rng, complex_orbitals=True)
    L = T.cholesky_from_thc(X, Mmat)
    assert L.shape == (5, 3, 3)
    for n in range(L.shape[0]):
        assert np.allclose(L[n], L[n].conj().T, atol=1e-15)          # Hermitian for a real kernel
    assert rel(four_index_from_cholesky(L), T.four_index_thc(X, Mmat)) < 1e-12
    # a rank-deficient kernel keeps only its non-zero directions
    B = rng.standard_normal((5, 2))
    assert T.cholesky_from_thc(X, B @ B.T).shape[0] == 2


def test_direct_local_energy_against_cholesky_form_and_fock_space():
    rng = np.random.default_rng(2)
    M, N, Nmu = 5, 2, 7
    h, _, _ = syn.make_hamiltonian(M, 1, rng)
    X, Mmat = syn.make_thc(M, Nmu, rng, complex_orbitals=True)
    E0 = 0.3
    Psi = [crandn(rng, M, N), crandn(rng, M, N)]
    Phi = [crandn(rng, 3, M, N), crandn(rng, 3, M, N)]
    E_thc = T.local_energy_thc(h, X, Mmat, E0, Psi, Phi)
    ham = O.Hamiltonian(h=h, L=T.cholesky_from_thc(X, Mmat), E0=E0)
    E_chol, t_chol, _ = O.local_energy(ham, Psi, Phi)
    assert rel(E_thc, E_chol) < 1e-12
    fs = FockSpace(M, N, N)
    H = fs.hamiltonian(h, T.four_index_thc(X, Mmat), E0)
    vp = fs.slater_vector(*Psi)
    for w in range(3):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ref = np.vdot(vp, H @ vf) / np.vdot(vp, vf)
        assert abs(E_thc[w] - ref) < 1e-11 * max(1.0, abs(ref)), w
    # the force bias of the factorised fields
    assert rel(T.force_bias_traces_thc(X, Mmat, Psi, Phi), t_chol) < 1e-12
    # negative control: conjugating the orbitals on the wrong side changes the energy
    assert rel(T.local_energy_thc(h, np.conj(X), Mmat, E0, Psi, Phi), E_chol) > 1e-3


def test_hs_potential_and_real_orbitals():
    rng = np.random.default_rng(3)
    M, Nmu = 6, 9
    X, Mmat = syn.make_thc(M, Nmu, rng, complex_orbitals=True)
    L = T.cholesky_from_thc(X, Mmat)
    c = crandn(rng, 4, L.shape[0])
    assert rel(T.hs_potential_thc(c, X, Mmat), O.hs_potential(c, L)) < 1e-12
    Xr, Mr = syn.make_thc(M, Nmu, rng)
    Lr = T.cholesky_from_thc(Xr, Mr)
    assert np.isrealobj(Lr)
    assert np.max(np.abs(Lr - np.swapaxes(Lr, 1, 2))) < 1e-15


def test_thc_factor_is_the_diagonally_pivoted_cholesky_factor():
    """U U^T = M; in the pivot order read off U (the row that stays zero in every later column),
    U is LAPACK's Cholesky factor of the permuted kernel, and every pivot is the row with the
    largest remaining diagonal at its step; a kernel of rank 3 stops after three columns."""
    import scipy.linalg
    rng = np.random.default_rng(4)
    _, Mmat = syn.make_thc(6, 10, rng)
    U = T.thc_factor(Mmat)
    assert U.shape == (10, 10)
    assert rel(U @ U.T, Mmat) < 1e-12
    piv = []
    for r in range(U.shape[1]):
        rest = [i for i in range(10) if i not in piv]
        later = np.max(np.abs(U[rest, r + 1:]), axis=1) if r + 1 < U.shape[1] else np.zeros(len(rest))
        cand = [i for i, z in zip(rest, later) if z < 1e-12 * np.max(np.abs(U))]
        assert len(cand) == 1
        piv.append(cand[0])
        d = np.array([Mmat[i, i] - np.sum(U[i, :r] ** 2) for i in rest])
        assert rest[int(np.argmax(d))] == piv[-1]
    L = scipy.linalg.cholesky(Mmat[np.ix_(piv, piv)], lower=True)
    assert np.max(np.abs(L - U[piv])) < 1e-12 * np.max(np.abs(L))
    B = rng.standard_normal((10, 3))
    U3 = T.thc_factor(B @ B.T)
    assert U3.shape == (10, 3) and rel(U3 @ U3.T, B @ B.T) < 1e-12
