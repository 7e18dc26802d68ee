"""Tensor-hypercontraction Hamiltonians on the FP64 GPU path against the oracle (Sec. V, Eqs. (4)-(6)).

The GPU never forms Cholesky vectors: it contracts through the interpolating points.  The
oracle runs its phaseless step on the equivalent Cholesky vectors L^n = X diag(U[:, n]) X^T
built from the same modified-Cholesky factor U of the kernel, and its direct THC local energy
(no L^n) checks the energy on its own.  Fields are passed to both, so trajectories match to
the FP64 bar (1e-10 relative)."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle import thc as T
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu


def thc_system(M, N, Nmu, seed):
    rng = np.random.default_rng(seed)
    h, _, E0 = syn.make_hamiltonian(M, 1, rng)
    X, Mk = syn.make_thc(M, Nmu, rng)
    Psi = syn.make_trial(h, N, N)
    return h, X, Mk, E0, Psi


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("M,N,Nmu,W,steps", [(24, 5, 48, 6, 8), (64, 16, 256, 5, 6)])
def test_thc_trajectory_matches_oracle(M, N, Nmu, W, steps):
    h, X, Mk, E0, Psi = thc_system(M, N, Nmu, 100 + M)
    L = T.cholesky_from_thc(X, Mk)
    nch = L.shape[0]
    tau = 0.01
    x = syn.make_fields(steps, W, nch, seed=3)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=tau, k_taylor=6, k_qr=3)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W)
    ref = [O.step(ham, Psi, B, wk, x[s], p)[1] for s in range(steps)]
    with AFQMC(h, None, E0, Psi[0], Psi[1], W, tau, k_qr=3, thc=(X, Mk)) as g:
        assert api.afqmc_hamiltonian_info(g.ham) == (M, nch, Nmu)
        got = g.step(steps, x, measure_every=1)
        E_L, w, logS, _ = g.energy()
    print(f"THC M={M} Nmu={Nmu} Nchol={nch}: E_mix rel err {rel(got, np.array(ref)):.2e}")
    assert rel(got, np.array(ref)) < 1e-10
    E_ref = O.local_energy(ham, Psi, wk.Phi)[0]
    assert rel(E_L, E_ref) < 1e-10
    assert rel(w, wk.w) < 1e-10
    assert np.max(np.abs(logS.real - wk.logS.real)) < 1e-10 * np.max(np.abs(wk.logS.real)) + 1e-12


def test_thc_local_energy_matches_direct_contraction():
    """E_L at random walkers against the oracle's direct THC energy (Wick contraction through
    the interpolating points, no Cholesky vectors)."""
    M, N, Nmu, W = 40, 8, 120, 4
    h, X, Mk, E0, Psi = thc_system(M, N, Nmu, 7)
    Phi0 = [syn.make_random_walkers(M, N, W, 1) + 0.5 * Psi[0][None],
            syn.make_random_walkers(M, N, W, 2) + 0.5 * Psi[1][None]]
    with AFQMC(h, None, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi0, thc=(X, Mk)) as g:
        E_L = g.energy()[0]
    ref = T.local_energy_thc(h, X, Mk, E0, Psi, Phi0)
    assert rel(E_L, ref) < 1e-10


def test_thc_rank_and_unsupported_combinations():
    M, N, Nmu, W = 32, 8, 40, 2
    rng = np.random.default_rng(9)
    h, _, E0 = syn.make_hamiltonian(M, 1, rng)
    X = rng.normal(0.0, 1.0 / np.sqrt(M), size=(M, Nmu))
    Bf = rng.normal(size=(Nmu, 7))
    Mk = Bf @ Bf.T                                   # rank 7: seven fields per walker
    Psi = syn.make_trial(h, N, N)
    with AFQMC(h, None, E0, Psi[0], Psi[1], W, 0.01, thc=(X, Mk)) as g:
        assert g.Nchol == 7
        with pytest.raises(api.AfqmcError) as e:
            api.afqmc_bp_begin(g.wk, 2)
        assert e.value.code == -8
        with pytest.raises(api.AfqmcError) as e:
            g.backward(np.ones(W, dtype=np.complex128))
        assert e.value.code == -8
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, None, E0, Psi[0], Psi[1], W, 0.01, thc=(X, Mk), precision=api.PREC_BF16X3)
    assert e.value.code == -8
    bad = Mk.copy()
    bad[0, 1] += 1.0                                 # not symmetric
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, None, E0, Psi[0], Psi[1], W, 0.01, thc=(X, bad))
    assert e.value.code == -1
