"""Pins of the back-propagation oracle (oracle/backprop.py): the back-propagated one-body
density matrix the paper lists among the estimators (Sec. V), restated from the mathematics.

* The back-propagated trial is the adjoint of the forward propagators in the right order:
  Psi_bp^+ X = Psi^+ B(n) ... B(1) X for an arbitrary X, with B(k) applied by the forward
  propagator (negative controls: reversed order, no adjoint).
* A window of length zero gives the mixed one-body density, checked against Fock-space
  matrix elements <Psi| c+_i c_j |Phi> / <Psi|Phi>.
* A one-step window averaged over the field (Nchol = 1, Gauss-Hermite) gives
  <Psi| exp(-tau (H - E0)) c+_i c_j |Phi> / <Psi|Phi> from Fock-space exponentials up to the
  O(tau^3) symmetric Trotter error (negative control: the transposed density matrix).
* Invariances: walker relabelling, re-orthonormalisation of the back-propagated trial, and a
  comb that keeps every walker; a comb inside the window follows the ancestry."""
import numpy as np
import scipy.linalg

from oracle import afqmc as O
from oracle import backprop as BP
from oracle.fock import FockSpace, four_index_from_cholesky
from paper_2003_01831_gb300 import synthetic as syn


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def unit(M, i, j):
    E = np.zeros((M, M))
    E[i, j] = 1.0
    return E


def test_back_propagated_trial_is_the_adjoint_of_the_forward_steps():
    rng = np.random.default_rng(3)
    M, N, nch, W, n, tau, K = 7, 3, 4, 2, 3, 0.05, 10
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    B = O.half_one_body_propagator(O.Hamiltonian(h=h, L=L, E0=E0), tau)
    Psi = crandn(rng, M, N)
    coefs = [crandn(rng, W, nch) for _ in range(n)]     # complex: A is not Hermitian
    X = crandn(rng, W, M, 5)
    Y = X
    for c in coefs:                                      # B(n) ... B(1) X, forward
        Y = O.propagate(Y, O.hs_potential(c, L), B, tau, K)
    rhs = Psi.conj().T @ Y
    Q = BP.back_propagated_trial(L, Psi, B, coefs, tau, K)
    assert rel(np.conj(np.swapaxes(Q, 1, 2)) @ X, rhs) < 1e-12
    # negative controls: the steps in the wrong order, and the forward operators in place of
    # their adjoints
    Qr = BP.back_propagated_trial(L, Psi, B, coefs[::-1], tau, K)
    assert rel(np.conj(np.swapaxes(Qr, 1, 2)) @ X, rhs) > 1e-4
    Qf = np.repeat(Psi[None], W, axis=0)
    for c in reversed(coefs):
        Qf = O.propagate(Qf, O.hs_potential(c, L), B, tau, K)
    assert rel(np.conj(np.swapaxes(Qf, 1, 2)) @ X, rhs) > 1e-4


def fock_system(seed, M=5, Nup=2, Ndn=1):
    rng = np.random.default_rng(seed)
    h, L, _ = syn.make_hamiltonian(M, 1, rng)
    Psi = [crandn(rng, M, Nup), crandn(rng, M, Ndn)]
    Phi = [crandn(rng, M, Nup), crandn(rng, M, Ndn)]
    fs = FockSpace(M, Nup, Ndn)
    H = fs.hamiltonian(h, four_index_from_cholesky(L))
    return h, L, Psi, Phi, fs, H


def test_zero_length_window_is_the_mixed_density_matrix():
    h, L, Psi, Phi, fs, _ = fock_system(11)
    M = h.shape[0]
    G = BP.Window([p[None] for p in Phi]).estimate(L, Psi, np.eye(M), np.ones(1), 0.01, 6)
    vp = fs.slater_vector(*Psi)
    vf = fs.slater_vector(*Phi)
    ov = np.vdot(vp, vf)
    for i in range(M):
        for j in range(M):
            ref = np.vdot(vp, fs.one_body_operator(unit(M, i, j)) @ vf) / ov
            assert abs(G[0][i, j] + G[1][i, j] - ref) < 1e-12 * max(1.0, abs(ref)), (i, j)
    assert abs(np.trace(G[0]) - Psi[0].shape[1]) < 1e-12
    assert abs(np.trace(G[1]) - Psi[1].shape[1]) < 1e-12


def one_step_window_error(h, L, Psi, Phi, fs, H, tau, transpose=False, nodes=50):
    """max_ij | E_x[<Psi|B(x) c+_i c_j|Phi>] - <Psi|exp(-tau H) c+_i c_j|Phi> | / max |ref|.

    The integrand is the window estimate for one walker of weight 1 times the overlap
    <Psi_bp(x)|Phi> = <Psi|B(x)|Phi>."""
    M = h.shape[0]
    ham = O.Hamiltonian(h=h, L=L, E0=0.0)
    B = O.half_one_body_propagator(ham, tau)
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)
    ws = ws / np.sqrt(2 * np.pi)
    acc = np.zeros((M, M), dtype=np.complex128)
    for x, wq in zip(xs, ws):
        win = BP.Window([p[None] for p in Phi])
        win.record(np.array([[x + 0j]]))
        G = win.estimate(L, Psi, B, np.ones(1), tau, 30)
        Q = [BP.back_propagated_trial(L, Psi[s], B, win.coefs, tau, 30)[0] for s in range(2)]
        ov = np.prod([np.linalg.det(Q[s].conj().T @ Phi[s]) for s in range(2)])
        acc += wq * ov * (G[0] + G[1])
    vp = fs.slater_vector(*Psi)
    vf = fs.slater_vector(*Phi)
    U = scipy.linalg.expm(-tau * H)
    ref = np.array([[np.vdot(vp, U @ (fs.one_body_operator(unit(M, i, j)) @ vf)) for j in range(M)]
                    for i in range(M)])
    if transpose:
        ref = ref.T
    return np.max(np.abs(acc - ref)) / np.max(np.abs(ref))


def test_one_step_window_against_fock_imaginary_time():
    h, L, Psi, Phi, fs, H = fock_system(5)
    e1 = one_step_window_error(h, L, Psi, Phi, fs, H, 0.02)
    e2 = one_step_window_error(h, L, Psi, Phi, fs, H, 0.01)
    print(f"one-step window: relative error {e1:.2e} at tau 0.02, {e2:.2e} at 0.01, ratio {e1 / e2:.2f}")
    assert e1 < 1e-4
    assert 6.0 < e1 / e2 < 10.0               # symmetric Trotter error ~ tau^3
    # negative control: the transposed density matrix (c+_j c_i) misses by far more
    assert one_step_window_error(h, L, Psi, Phi, fs, H, 0.01, transpose=True) > 1e3 * e2


def random_window(seed, M=8, N=3, nch=5, W=4, n=3):
    rng = np.random.default_rng(seed)
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    tau = 0.02
    B = O.half_one_body_propagator(O.Hamiltonian(h=h, L=L, E0=E0), tau)
    Psi = [crandn(rng, M, N), crandn(rng, M, N - 1)]
    win = BP.Window([crandn(rng, W, M, N), crandn(rng, W, M, N - 1)])
    for _ in range(n):
        win.record(0.3 * crandn(rng, W, nch))
    w = rng.uniform(0.5, 1.5, W)
    w[1] = 0.0                                    # a dead walker contributes nothing
    return L, Psi, B, tau, win, w, rng


def test_estimate_is_invariant_under_relabelling_and_reorthonormalisation():
    L, Psi, B, tau, win, w, rng = random_window(7)
    G = win.estimate(L, Psi, B, w, tau, 6)
    perm = np.array([2, 0, 3, 1])
    pw = BP.Window([p[perm] for p in win.Phi0])
    for c in win.coefs:
        pw.record(c[perm])
    Gp = pw.estimate(L, Psi, B, w[perm], tau, 6)
    for s in range(2):
        assert rel(Gp[s], G[s]) < 1e-13
        Q = BP.back_propagated_trial(L, Psi[s], B, win.coefs, tau, 6)
        R = crandn(rng, Q.shape[0], Q.shape[2], Q.shape[2]) + 3 * np.eye(Q.shape[2])
        assert rel(BP.rdm1(Q @ R, win.Phi0[s], w), G[s]) < 1e-12
        assert abs(np.trace(G[s]) - Psi[s].shape[1]) < 1e-12
    # a comb on equal weights keeps every walker in place
    idx = O.comb(np.ones(4), 0.37)
    assert np.array_equal(idx, np.arange(4))
    win.comb(idx)
    Gc = win.estimate(L, Psi, B, w, tau, 6)
    assert rel(Gc[0], G[0]) == 0.0 and rel(Gc[1], G[1]) == 0.0


def test_comb_inside_the_window_follows_the_ancestry():
    L, Psi, B, tau, win, w, rng = random_window(9, n=2)
    Phi0 = [p.copy() for p in win.Phi0]
    before = [c.copy() for c in win.coefs]
    idx = O.comb(np.array([0.2, 2.5, 0.9, 0.4]), 0.61)
    assert len(set(idx.tolist())) < 4              # some walker is copied, some dropped
    win.comb(idx)
    after = 0.3 * crandn(rng, 4, L.shape[0])
    win.record(after)
    w_end = rng.uniform(0.5, 1.5, 4)
    G = win.estimate(L, Psi, B, w_end, tau, 6)
    for s in range(2):
        acc = 0.0
        for j in range(4):
            hist = [c[idx[j]][None] for c in before] + [after[j][None]]
            Q = BP.back_propagated_trial(L, Psi[s], B, hist, tau, 6)
            acc = acc + BP.rdm1(Q, Phi0[s][idx[j]][None], w_end[j:j + 1]) * w_end[j]
        assert rel(G[s], acc / np.sum(w_end)) < 1e-13
