"""Oracle pins against brute-force Fock-space quantum mechanics (Sec. V, Eq. (1)).

The Fock-space Hamiltonian is built operator by operator from the 4-index
tensor rebuilt from L by loops, so these tests check the oracle's Green's
function, Coulomb/exchange energy, force bias, h' correction and HS sign
convention without sharing any of its algebra."""
import numpy as np
import pytest
import scipy.linalg

from oracle import afqmc as O
from oracle.fock import FockSpace, four_index_from_cholesky
from paper_2003_01831_gb300 import synthetic as syn


def random_complex(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.fixture(scope="module")
def sys6():
    rng = np.random.default_rng(21)
    M, N = 6, 2
    h, L, _ = syn.make_hamiltonian(M, 8, rng, decay=5.0)
    L *= 3.0  # stronger interaction than the R1 scale so every term matters
    ham = O.Hamiltonian(h=h, L=L, E0=0.25)
    Psi = syn.make_trial(h, N, N)
    Psi = [Psi[0] + 0.2 * random_complex(rng, M, N), Psi[1] + 0.2 * random_complex(rng, M, N)]
    fs = FockSpace(M, N, N)
    H = fs.hamiltonian(h, four_index_from_cholesky(L), ham.E0)
    return ham, Psi, fs, H, rng


def test_fock_hamiltonian_is_hermitian(sys6):
    _, _, _, H, _ = sys6
    assert np.allclose(H, H.conj().T, atol=1e-12)


def test_overlap_matches_fock_inner_product(sys6):
    ham, Psi, fs, H, rng = sys6
    Phi = [random_complex(rng, 1, 6, 2) for _ in range(2)]
    vp = fs.slater_vector(Psi[0], Psi[1])
    vf = fs.slater_vector(Phi[0][0], Phi[1][0])
    ref = np.vdot(vp, vf)
    got = np.exp(sum(O.log_det(O.overlap_matrix(Psi[s], Phi[s]))[0] for s in range(2)))
    assert abs(got - ref) < 1e-12 * abs(ref)


def test_mixed_local_energy_matches_fock(sys6):
    ham, Psi, fs, H, rng = sys6
    Phi = [random_complex(rng, 3, 6, 2) for _ in range(2)]
    EL, _, _ = O.local_energy(ham, Psi, Phi)
    vp = fs.slater_vector(Psi[0], Psi[1])
    for w in range(3):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ref = np.vdot(vp, H @ vf) / np.vdot(vp, vf)
        assert abs(EL[w] - ref) < 1e-11 * max(1, abs(ref))


def test_force_bias_matches_fock(sys6):
    ham, Psi, fs, H, rng = sys6
    Phi = [random_complex(rng, 2, 6, 2) for _ in range(2)]
    _, t_sum, _ = O.local_energy(ham, Psi, Phi)
    vp = fs.slater_vector(Psi[0], Psi[1])
    for w in range(2):
        vf = fs.slater_vector(Phi[0][w], Phi[1][w])
        ov = np.vdot(vp, vf)
        for n in range(ham.Nchol):
            Ln = fs.one_body_operator(ham.L[n])
            assert abs(t_sum[w, n] - np.vdot(vp, Ln @ vf) / ov) < 1e-11


def test_one_body_exponential_is_thouless(sys6):
    """exp(i sqrt(tau) x L-hat) on a determinant = the determinant exp(i sqrt(tau) x L) Phi."""
    ham, Psi, fs, H, rng = sys6
    Phi = [random_complex(rng, 6, 2) for _ in range(2)]
    X = 1j * 0.3 * ham.L[0]
    op = scipy.linalg.expm(fs.one_body_operator(X))
    lhs = op @ fs.slater_vector(Phi[0], Phi[1])
    rhs = fs.slater_vector(scipy.linalg.expm(X) @ Phi[0], scipy.linalg.expm(X) @ Phi[1])
    assert np.max(np.abs(lhs - rhs)) < 1e-11 * np.max(np.abs(rhs))


def hs_quadrature_error(ham, Psi, Phi, fs, H, tau, nodes=60):
    """| sum_x GH-weight <Psi|B exp(i sqrt(tau) x L) B|Phi> - <Psi|exp(-tau H)|Phi> | (Nchol = 1).

    The one-body matrix exponential is exact here (the quadrature integrand is
    built with the oracle's propagator at a high Taylor order)."""
    xs, ws = np.polynomial.hermite_e.hermegauss(nodes)     # weight exp(-x^2/2)
    ws = ws / np.sqrt(2 * np.pi)
    B = O.half_one_body_propagator(ham, tau)
    acc = 0.0
    for x, wgt in zip(xs, ws):
        A = O.hs_potential(np.array([[x + 0j]]), ham.L)
        Pn = [O.propagate(Phi[s][None], A, B, tau, 40)[0] for s in range(2)]
        acc += wgt * np.exp(sum(O.log_det(O.overlap_matrix(Psi[s], Pn[s][None]))[0] for s in range(2)))
    vp = fs.slater_vector(Psi[0], Psi[1])
    vf = fs.slater_vector(Phi[0], Phi[1])
    ref = np.vdot(vp, scipy.linalg.expm(-tau * (H - ham.E0 * np.eye(fs.dim))) @ vf)
    return abs(acc - ref), abs(ref)


def test_hs_convention_against_exact_propagation():
    """Nchol = 1: the HS integral over the one-body propagator reproduces
    <Psi|exp(-tau H)|Phi> up to the O(tau^3) symmetric Trotter error.  A wrong
    sign/i convention or a missing h' correction leaves an O(tau) error."""
    rng = np.random.default_rng(5)
    M, N = 5, 2
    h, L, _ = syn.make_hamiltonian(M, 1, rng)
    ham = O.Hamiltonian(h=h, L=L, E0=0.0)
    Psi = syn.make_trial(h, N, N)
    Phi = [random_complex(rng, M, N) for _ in range(2)]
    fs = FockSpace(M, N, N)
    H = fs.hamiltonian(h, four_index_from_cholesky(L))
    e1, r1 = hs_quadrature_error(ham, Psi, Phi, fs, H, 0.02)
    e2, r2 = hs_quadrature_error(ham, Psi, Phi, fs, H, 0.01)
    assert e1 / r1 < 1e-4
    ratio = e1 / e2
    assert 6.0 < ratio < 10.0, ratio          # local error ~ tau^3


def test_wrong_hs_sign_is_detected():
    """Negative control for the test above: using h instead of h' breaks the tau^3 scaling."""
    rng = np.random.default_rng(5)
    M, N = 5, 2
    h, L, _ = syn.make_hamiltonian(M, 1, rng)
    Psi = syn.make_trial(h, N, N)
    Phi = [random_complex(rng, M, N) for _ in range(2)]
    fs = FockSpace(M, N, N)
    H = fs.hamiltonian(h, four_index_from_cholesky(L))
    # build a Hamiltonian object whose h' equals h (i.e. drop the correction)
    h_shift = h + 0.5 * np.einsum("nik,njk->ij", L, L)
    wrong = O.Hamiltonian(h=h_shift, L=L, E0=0.0)
    e1, r1 = hs_quadrature_error(wrong, Psi, Phi, fs, H, 0.02)
    e2, r2 = hs_quadrature_error(wrong, Psi, Phi, fs, H, 0.01)
    assert e1 / e2 < 3.0 and e1 / r1 > 1e-3


@pytest.fixture(scope="module")
def fci8():
    rng = np.random.default_rng(1008)
    M, N = 8, 2
    h, L, _ = syn.make_hamiltonian(M, 16, rng, decay=8.0)
    L *= 0.8
    ham = O.Hamiltonian(h=h, L=L, E0=0.0)
    Psi = syn.make_trial(h, N, N)
    fs = FockSpace(M, N, N)
    H = fs.hamiltonian(h, four_index_from_cholesky(L))
    e, V = np.linalg.eigh(H)
    return ham, Psi, fs, H, e, V


def blocking_error(series, nblocks=20):
    b = np.array_split(np.asarray(series), nblocks)
    m = np.array([x.mean() for x in b])
    return m.std(ddof=1) / np.sqrt(nblocks)


def test_phaseless_run_approaches_fci(fci8):
    """Long phaseless projection on the 8-orbital 2+2 system approaches E_FCI within
    3 sigma plus a 5 mHa phaseless-bias allowance (the allowance itself is unpinned)."""
    ham, Psi, fs, H, e, V = fci8
    W, nsteps, tau = 200, 1200, 0.02
    p = O.Params(tau=tau, k_taylor=6, k_qr=10, fb_cap=1.0)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W)
    rng = np.random.default_rng(99)
    trace = []
    for s in range(nsteps):
        E_L, E_mix = O.step(ham, Psi, B, wk, rng.standard_normal((W, ham.Nchol)), p)
        trace.append(E_mix.real)
        if (s + 1) % 20 == 0:            # rescale weights (E_mix is scale invariant)
            wk.w = wk.w / np.mean(wk.w[wk.w > 0])
    eq = np.array(trace[300:])
    est, err = eq.mean(), blocking_error(eq)
    E_hf = O.local_energy(ham, Psi, [p_[None] for p_ in Psi])[0][0].real
    assert E_hf - e[0] > 0.04                  # the test system is correlated
    assert abs(est - e[0]) < 3 * err + 5e-3, (est, err, e[0], E_hf)


def test_free_projection_matches_exact_imaginary_time(fci8):
    """Free projection (complex weights, no cap, no phase projection) reproduces
    E(beta) = <Psi|H e^{-beta H}|Psi> / <Psi|e^{-beta H}|Psi> within 3 sigma + O(tau^2)."""
    ham, Psi, fs, H, e, V = fci8
    W, nsteps, tau = 4000, 25, 0.02
    p = O.Params(tau=tau, k_taylor=8, k_qr=0, mode="free")
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W, complex_weights=True)
    rng = np.random.default_rng(7)
    for s in range(nsteps):
        O.step(ham, Psi, B, wk, rng.standard_normal((W, ham.Nchol)), p)
    E_L, _, _ = O.local_energy(ham, Psi, wk.Phi)
    num, den = wk.w * E_L, wk.w
    est = (num.sum() / den.sum()).real
    # jackknife over walker blocks
    nb = 40
    idx = np.array_split(np.arange(W), nb)
    jk = []
    for b in idx:
        mask = np.ones(W, bool)
        mask[b] = False
        jk.append((num[mask].sum() / den[mask].sum()).real)
    jk = np.array(jk)
    err = np.sqrt((nb - 1) * np.mean((jk - jk.mean()) ** 2))
    vp = fs.slater_vector(Psi[0], Psi[1])
    beta = tau * nsteps
    prop = (V * np.exp(-beta * (e - e[0]))) @ V.conj().T
    exact = (np.vdot(vp, H @ prop @ vp) / np.vdot(vp, prop @ vp)).real
    assert abs(est - exact) < 3 * err + 2e-3, (est, err, exact)
