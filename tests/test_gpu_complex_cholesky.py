"""General complex Cholesky vectors on the FP64 GPU path (Sec. V, Eq. (3) with complex L_n:
v_ijkl = sum_n L^n_ik conj(L^n_lj)), through afqmc_create_hamiltonian_complex.

The library runs the Hermitian split A_n = (L_n + L_n^+)/2, B_n = (L_n - L_n^+)/(2i); the oracle
runs the same step on its own split (oracle.afqmc.hermitian_split, pinned against Fock-space
matrices built from the complex L).  Parity bar as for real L: local energies, weights and
log-overlaps to 1e-10 relative at every step, walkers to 1e-9.  Also: a real symmetric L given
as complex reproduces the real-L run (its B_n vanish), device Philox fields cover the 2 Nchol
split vectors, and the calls that need real L reject it."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.philox import philox_fields
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def phase_close(a, b, tol):
    return np.max(np.abs(np.exp(1j * (a.imag - b.imag)) - 1)) < tol


def crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def complex_system(M, Nu, Nd, nch, seed, scale=0.5, perturb=0.0):
    rng = np.random.default_rng(seed)
    h, _, _ = syn.make_hamiltonian(M, 1, rng)
    L = scale * crandn(rng, nch, M, M) / np.sqrt(M)      # neither Hermitian nor symmetric
    Psi = [np.asarray(p, dtype=np.complex128) for p in syn.make_trial(h, Nu, Nd)]
    if perturb:
        Psi = [p + perturb * crandn(rng, *p.shape) for p in Psi]
    return h, L, Psi, rng


def run_parity(h, L, E0, Psi, W, tau, nsteps, k_qr, x, Phi0=None, mode="phaseless", fb_cap=1.0):
    ham = O.Hamiltonian(h=h, L=O.hermitian_split(L), E0=E0)
    p = O.Params(tau=tau, k_taylor=6, k_qr=k_qr, fb_cap=fb_cap, mode=mode)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W, Phi0, complex_weights=(mode == "free"))
    wm = {"free": api.WEIGHT_FREE, "local": api.WEIGHT_LOCAL}.get(mode, api.WEIGHT_PHASELESS)
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, Phi0=Phi0, k_qr=k_qr, fb_cap=fb_cap, weight_mode=wm) as g:
        assert g.Nchol == ham.Nchol == 2 * L.shape[0]
        E_L, _, _, _ = g.energy()
        assert rel(E_L, O.local_energy(ham, Psi, wk.Phi)[0]) < RTOL
        for s in range(nsteps):
            _, Emix_ref = O.step(ham, Psi, B, wk, x[s], p)
            trace = g.step(1, x[s:s + 1], measure_every=1)
            assert abs(trace[0] - Emix_ref) < RTOL * abs(Emix_ref), (s, trace[0], Emix_ref)
            E_L, w, logS, _ = g.energy()
            assert rel(E_L, O.local_energy(ham, Psi, wk.Phi)[0]) < RTOL, s
            assert rel(w, wk.w) < RTOL, s
            assert rel(logS.real, wk.logS.real) < RTOL, s
            assert phase_close(logS, wk.logS, RTOL * 10), s
        Pu, Pd, _, step = g.walkers()
        assert step == nsteps
        assert rel(Pu, wk.Phi[0]) < 1e-9 and rel(Pd, wk.Phi[1]) < 1e-9
    return wk


def test_complex_L_ragged_trajectory_matches_oracle():
    """N_up != N_dn, sizes that are not tile multiples, complex trial, random walkers,
    force-bias cap active, QR every other step."""
    M, Nu, Nd, nch, W, steps = 13, 3, 2, 4, 5, 6
    h, L, Psi, rng = complex_system(M, Nu, Nd, nch, seed=21, perturb=0.2)
    Phi0 = [syn.make_random_walkers(M, Nu, W, 5), syn.make_random_walkers(M, Nd, W, 6)]
    x = rng.standard_normal((steps, W, 2 * nch))
    run_parity(h, L, 0.75, Psi, W, 0.01, steps, 2, x, Phi0=Phi0, fb_cap=0.05)


@pytest.mark.parametrize("mode", ["phaseless", "local", "free"])
def test_complex_L_weight_modes_match_oracle(mode):
    M, N, nch, W, steps = 16, 4, 6, 4, 5
    h, L, Psi, rng = complex_system(M, N, N, nch, seed=33)
    x = rng.standard_normal((steps, W, 2 * nch))
    run_parity(h, L, 0.0, Psi, W, 0.005, steps, 3, x, mode=mode)


def test_real_symmetric_L_given_as_complex_reproduces_real_run():
    """For real symmetric L the split gives A_n = L_n and B_n = 0, so the fields of the B_n
    change nothing and the run equals the real-L run fed the A_n fields."""
    rng = np.random.default_rng(4)
    M, N, nch, W, steps = 20, 4, 9, 4, 4
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    x = rng.standard_normal((steps, W, nch))
    xs = np.empty((steps, W, 2 * nch))
    xs[..., 0::2] = x
    xs[..., 1::2] = rng.standard_normal((steps, W, nch))
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, k_qr=2) as g1, \
            AFQMC(h, L.astype(np.complex128), E0, Psi[0], Psi[1], W, 0.01, k_qr=2) as g2:
        t1 = g1.step(steps, x, measure_every=1)
        t2 = g2.step(steps, xs, measure_every=1)
        assert rel(t2, t1) < 1e-12
        e1, e2 = g1.energy(), g2.energy()
        for a, b in zip(e1[:3], e2[:3]):
            assert rel(b, a) < 1e-12
        assert rel(g2.walkers()[0], g1.walkers()[0]) < 1e-12


def test_complex_L_philox_fields_cover_the_split_vectors():
    M, N, nch, W, steps, seed = 12, 3, 5, 6, 3, 99
    h, L, Psi, _ = complex_system(M, N, N, nch, seed=8)
    xs = np.stack([philox_fields(seed, s, W, 2 * nch) for s in range(steps)])
    with AFQMC(h, L, 0.0, Psi[0], Psi[1], W, 0.01) as g1, AFQMC(h, L, 0.0, Psi[0], Psi[1], W, 0.01) as g2:
        t1 = g1.step(steps, None, seed=seed, measure_every=1)
        t2 = g2.step(steps, xs, measure_every=1)
        assert rel(t1, t2) < 1e-12
        assert rel(g1.walkers()[0], g2.walkers()[0]) < 1e-12


def test_complex_L_rejections():
    M, N, nch, W = 64, 4, 8, 2
    h, L, Psi, _ = complex_system(M, N, N, nch, seed=2)
    Psi = [p.real.copy() for p in Psi]
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, L, 0.0, Psi[0], Psi[1], W, 0.01, precision=api.PREC_BF16X3)
    assert e.value.code == -8
    with AFQMC(h, L, 0.0, Psi[0], Psi[1], W, 0.01) as g:
        with pytest.raises(api.AfqmcError) as e:
            g.backward(np.ones(W, complex))
        assert e.value.code == -8
    bad = L.copy()
    bad[3, 1, 2] = complex(0.0, np.nan)
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, bad, 0.0, Psi[0], Psi[1], W, 0.01)
    assert e.value.code == -4
