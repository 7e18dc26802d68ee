"""Pins of the local-energy weights and of the comb population control in the oracle.

* The comb is checked against a worked example and against what it must do whatever the
  weights: copy counts floor or ceil of W w_j / W_tot, dead walkers never taken, equal weights
  left alone, and on average (over xi) exactly W w_j / W_tot copies.
* The local-energy weight factor exp(-tau (E_L - E_T)) is pinned to the hybrid importance
  function it approximates: averaged over the Hubbard-Stratonovich field (Gauss-Hermite
  quadrature, one Cholesky vector), the hybrid factor equals exp(-tau (E_L - E_T)) up to
  O(tau^2) -- the shift x -> x - xbar removes the force bias from the average, leaving
  <Psi|exp(-tau (H - E_T))|Phi> / <Psi|Phi> = 1 - tau (E_L - E_T) + O(tau^2)."""
import numpy as np
import pytest

from oracle import afqmc as O
from paper_2003_01831_gb300 import synthetic as syn


def counts(idx, W):
    return np.bincount(idx, minlength=W)


def test_comb_worked_example():
    # W_tot = 4, running sums 0.5, 2, 3, 4.  xi = 0.25: slots 0.25, 1.25, 2.25, 3.25;
    # xi = 0.75: slots 0.75, 1.75, 2.75, 3.75.
    w = np.array([0.5, 1.5, 1.0, 1.0])
    assert O.comb(w, 0.25).tolist() == [0, 1, 2, 3]
    assert O.comb(w, 0.75).tolist() == [1, 1, 2, 3]
    assert O.comb(np.array([0.0, 2.0, 0.0, 2.0]), 0.5).tolist() == [1, 1, 3, 3]


@pytest.mark.parametrize("xi", [0.01, 0.1, 0.5, 0.999])
def test_comb_equal_weights_is_identity(xi):
    # (xi = 0 puts every slot on an interval boundary, where the rounding of the running sum
    # decides; any xi clear of 0 gives the identity)
    assert np.array_equal(O.comb(np.full(37, 0.7), xi), np.arange(37))


@pytest.mark.parametrize("seed", range(6))
def test_comb_counts_and_dead_walkers(seed):
    rng = np.random.default_rng(seed)
    W = 200
    w = rng.exponential(1.0, W)
    w[rng.random(W) < 0.2] = 0.0
    for xi in rng.random(5) * 0.999:
        idx = O.comb(w, xi)
        c = counts(idx, W)
        expect = W * w / w.sum()
        assert c.sum() == W
        assert np.all(np.diff(idx) >= 0)
        assert np.all(c[w == 0] == 0)
        assert np.all((c >= np.floor(expect) - 1e-9) & (c <= np.ceil(expect) + 1e-9))


def test_comb_is_unbiased_over_xi():
    """Each copy count is a step function of xi; on a fine uniform grid its mean is
    W w_j / W_tot up to one grid step."""
    rng = np.random.default_rng(11)
    W = 24
    w = rng.exponential(1.0, W)
    grid = (np.arange(4000) + 0.5) / 4000
    mean = np.mean([counts(O.comb(w, xi), W) for xi in grid], axis=0)
    assert np.allclose(mean, W * w / w.sum(), atol=2.0 / 4000)


def test_population_control_moves_walkers_and_weights():
    ham, Psi = small_system()
    Phi0 = [syn.make_random_walkers(6, 2, 5, seed=s) for s in (1, 2)]
    wk = O.init_walkers(ham, Psi, 5, Phi0)
    wk.w = np.array([0.0, 3.0, 1.0, 0.5, 0.5])
    Phi_before = [p.copy() for p in wk.Phi]
    logS_before = wk.logS.copy()
    idx = O.population_control(wk, 0.3)
    assert idx.tolist() == O.comb(np.array([0.0, 3.0, 1.0, 0.5, 0.5]), 0.3).tolist()
    assert np.allclose(wk.w, 1.0)
    for s in range(2):
        assert np.array_equal(wk.Phi[s], Phi_before[s][idx])
    assert np.array_equal(wk.logS, logS_before[idx])


def small_system(M=6, N=2, Nchol=1, seed=5):
    rng = np.random.default_rng(seed)
    h, L, _ = syn.make_hamiltonian(M, Nchol, rng, decay=6.0)
    L = L * 4.0                      # a two-body term large enough to matter at this tau
    return O.Hamiltonian(h=h, L=L, E0=0.37), syn.make_trial(h, N, N)


def hybrid_average(ham, Psi, Phi, tau, nodes=60, K=16):
    """Field average of the hybrid importance factor for one walker (Nchol = 1)."""
    x, wq = np.polynomial.hermite_e.hermegauss(nodes)
    wq = wq / wq.sum()
    E_L, t_sum, _ = O.local_energy(ham, Psi, [p[None] for p in Phi])
    xbar = O.force_bias(t_sum, tau, 0.0)[0]                 # no cap
    E_T = O.local_energy(ham, Psi, [p[None] for p in Psi])[0][0].real
    B = O.half_one_body_propagator(ham, tau)
    c = x[:, None] - xbar[None, :]                            # [nodes, 1]
    A = O.hs_potential(c, ham.L)
    logS0 = sum(O.log_det(O.overlap_matrix(Psi[s], Phi[s][None]))[0] for s in range(2))
    logS1 = sum(O.log_det(O.overlap_matrix(Psi[s], O.propagate(np.repeat(Phi[s][None], nodes, 0), A, B, tau, K)))
                for s in range(2))
    I = np.exp(logS1 - logS0 + x * xbar[0] - 0.5 * xbar[0] ** 2 + tau * (E_T - ham.E0))
    return np.sum(wq * I), E_L[0], E_T


def test_local_energy_factor_is_the_field_averaged_hybrid_factor():
    ham, Psi = small_system()
    rng = np.random.default_rng(2)
    z = Psi[0] + 0.3 * (rng.standard_normal(Psi[0].shape) + 1j * rng.standard_normal(Psi[0].shape))
    Phi = [np.linalg.qr(z)[0], np.linalg.qr(Psi[1] + 0.2 * rng.standard_normal(Psi[1].shape))[0].astype(complex)]
    errs = []
    # a flipped sign would miss by twice the first-order term, a dropped E0 (0.37 here, against
    # E_L - E_T ~ 3.5) by ~10% of it; the O(tau^2) remainder is 2.6% and 1.3% at these tau
    for tau in (0.002, 0.001):
        avg, E_L, E_T = hybrid_average(ham, Psi, Phi, tau)
        target = np.exp(-tau * (E_L - E_T))
        first = abs(tau * (E_L - E_T))
        errs.append(abs(avg - target))
        assert first > 1e-3                                   # the first-order term is visible
        assert errs[-1] < 0.05 * first                        # and matched by the local factor
        # the oracle's local-energy factor is the real part of this exponent, bounded
        assert np.isclose(O.local_energy_factor(np.array([E_L]), E_T, tau)[0], np.exp(-tau * (E_L.real - E_T)))
    assert 3.0 < errs[0] / errs[1] < 5.0                      # the remainder is O(tau^2)


def test_energy_bound_clips_at_two_over_sqrt_tau():
    tau = 0.01
    E = np.array([-100.0, -12.0, -10.0, -8.0, 50.0]) + 0j
    got = O.energy_bound(E, -10.0, tau)
    assert got.tolist() == [-30.0, -12.0, -10.0, -8.0, 10.0]


def test_local_mode_step_weights():
    """One step in local mode: w' = w exp(-tau (E_b - E_T)) max(0, cos dtheta), E_b the bounded
    pre-step local energy (dtheta from the same overlaps as the hybrid mode)."""
    ham, Psi = small_system(M=8, N=3, Nchol=5, seed=9)
    Phi0 = [syn.make_random_walkers(8, 3, 4, seed=s) for s in (3, 4)]
    p = O.Params(tau=0.01, k_taylor=6, k_qr=0, mode="local")
    B = O.half_one_body_propagator(ham, p.tau)
    wk = O.init_walkers(ham, Psi, 4, Phi0)
    wk.w = np.array([1.0, 0.5, 2.0, 0.0])
    w0, logS0 = wk.w.copy(), wk.logS.copy()
    x = np.random.default_rng(1).standard_normal((4, 5))
    E_L, _ = O.step(ham, Psi, B, wk, x, p)
    dl = wk.logS - logS0
    expect = w0 * np.exp(-p.tau * (np.clip(E_L.real, wk.E_T - 20.0, wk.E_T + 20.0) - wk.E_T)) \
        * np.maximum(0.0, np.cos(dl.imag))
    assert np.allclose(wk.w, expect, rtol=1e-13)
    assert wk.w[3] == 0.0
