"""Back-propagated one-body density matrix on the GPU (afqmc_bp_begin / afqmc_bp_rdm1)
against the oracle (oracle/backprop.py, pinned against forward propagators and Fock-space
imaginary-time evolution).

FP64 path: the window estimate equals the oracle's to 1e-10 relative, for real and for
general complex Cholesky vectors, with a walker killed before the window, QR inside it, and
a comb between its steps (the window follows the ancestry); a zero-length window gives the
mixed estimate.  BF16X3 walker sets record the same shifted fields from their tensor-core
step and carry the trial back on the tensor cores, so their estimate follows the FP64 one and
the oracle to the mixed path's accuracy.  The window's
error states are reported, not guessed around."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle import backprop as BP
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("complex_L", [False, True])
def test_bp_rdm1_matches_oracle(complex_L):
    rng = np.random.default_rng(31)
    M, Nu, Nd, nch, W, tau, K = 12, 3, 2, 5, 6, 0.01, 6
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    if complex_L:
        L = 0.5 * crandn(rng, nch, M, M) / np.sqrt(M)
    Lo = O.hermitian_split(L) if complex_L else L
    Psi = [p + 0.2 * crandn(rng, *p.shape) for p in syn.make_trial(h, Nu, Nd)]
    Phi0 = [syn.make_random_walkers(M, Nu, W, 3), syn.make_random_walkers(M, Nd, W, 4)]
    ham = O.Hamiltonian(h=h, L=Lo, E0=E0)
    p = O.Params(tau=tau, k_taylor=K, k_qr=2)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W, Phi0)
    x = rng.standard_normal((6, W, Lo.shape[0]))
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, Phi0=Phi0, k_taylor=K, k_qr=2) as g:
        for s in range(2):
            O.step(ham, Psi, B, wk, x[s], p)
        g.step(2, x[0:2])
        Pu, Pd, w, step = g.walkers()
        w = w.copy()
        w[4] = 0.0                              # a dead walker contributes nothing
        g.set_walkers(Pu, Pd, w, step)
        wk.w[4] = 0.0

        g.bp_begin(0)                           # zero-length window: the mixed estimate
        G0 = g.bp_rdm1()
        ref0 = BP.Window(wk.Phi).estimate(Lo, Psi, B, wk.w, tau, K)
        for s in range(2):
            assert rel(G0[s], ref0[s]) < RTOL, s

        g.bp_begin(4)                           # four steps: QR after the 2nd and 4th, comb between
        win = BP.Window(wk.Phi)
        for s in (2, 3):
            O.step(ham, Psi, B, wk, x[s], p, record=win.coefs)
        g.step(2, x[2:4])
        idx_g = g.population_control(0.43)
        idx_o = O.population_control(wk, 0.43)
        assert np.array_equal(idx_g, idx_o)
        assert len(set(idx_o.tolist())) < W     # the comb copied some walker
        win.comb(idx_o)
        for s in (4, 5):
            O.step(ham, Psi, B, wk, x[s], p, record=win.coefs)
        g.step(2, x[4:6])
        G = g.bp_rdm1()
        ref = win.estimate(Lo, Psi, B, wk.w, tau, K)
        for s, n in enumerate((Nu, Nd)):
            print(f"spin {s}: rel diff {rel(G[s], ref[s]):.2e}, trace {np.trace(G[s]):.12f}")
            assert rel(G[s], ref[s]) < RTOL, s
            assert abs(np.trace(G[s]) - n) < 1e-10
        assert np.array_equal(g.bp_rdm1()[0], G[0])     # the window stays open


def test_bp_rdm1_bf16x3_follows_fp64():
    rng = np.random.default_rng(6)
    M, N, nch, W = 64, 32, 64, 8
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    G = {}
    for prec in (api.PREC_FP64, api.PREC_BF16X3):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, precision=prec, k_qr=3) as g:
            g.step(2, seed=5)
            g.bp_begin(4)
            g.step(4, seed=5)
            G[prec] = g.bp_rdm1()
    for s in range(2):
        d = rel(G[api.PREC_BF16X3][s], G[api.PREC_FP64][s])
        print(f"spin {s}: BF16X3 vs FP64 back-propagated 1RDM, max rel diff {d:.2e}")
        assert d < 1e-5


def test_bp_rdm1_bf16x3_matches_oracle():
    """BF16X3 walker set (M=128, N=32+32): the forward steps and every back step run on the tensor
    cores (the back steps through the forward step's three-slice propagation with conjugated
    coefficients and -i sqrt(tau)); the estimate follows the oracle's window to the mixed path's
    accuracy (bar 1e-5 relative), with a QR inside the window."""
    rng = np.random.default_rng(8)
    M, N, nch, W, tau, K = 128, 32, 96, 4, 0.005, 6
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=tau, k_taylor=K, k_qr=2)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W)
    x = rng.standard_normal((5, W, nch))
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, k_taylor=K, k_qr=2, precision=api.PREC_BF16X3) as g:
        for s in range(2):
            O.step(ham, Psi, B, wk, x[s], p)
        g.step(2, x[0:2])
        g.bp_begin(3)
        win = BP.Window(wk.Phi)
        for s in (2, 3, 4):
            O.step(ham, Psi, B, wk, x[s], p, record=win.coefs)
        g.step(3, x[2:5])
        G = g.bp_rdm1()
    ref = win.estimate(L, Psi, B, wk.w, tau, K)
    for s in range(2):
        d = rel(G[s], ref[s])
        print(f"spin {s}: BF16X3 back-propagated 1RDM vs oracle, max rel diff {d:.2e}")
        assert d < 1e-5
        assert abs(np.trace(G[s]) - N) < 1e-6


def test_bp_window_errors():
    rng = np.random.default_rng(2)
    M, N, nch, W = 10, 2, 6, 3
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)

    def code(fn, *a):
        with pytest.raises(api.AfqmcError) as e:
            fn(*a)
        return e.value.code

    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01) as g:
        assert code(g.bp_rdm1) == -1                 # no window
        assert code(g.bp_begin, -1) == -1
        g.bp_begin(3)
        g.step(1, seed=1)
        assert code(g.bp_rdm1) == -1                 # 1 of 3 steps
        g.step(2, seed=1)
        g.bp_rdm1()
        g.step(1, seed=1)
        assert code(g.bp_rdm1) == -1                 # a step after the window was complete
        g.bp_begin(1)
        g.step(1, seed=1)
        g.bp_rdm1()
        Pu, Pd, w, step = g.walkers()
        g.set_walkers(Pu, Pd, w, step)
        assert code(g.bp_rdm1) == -1                 # set_walkers closed the window
