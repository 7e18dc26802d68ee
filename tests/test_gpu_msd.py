"""Multi-determinant trials on the FP64 GPU path (afqmc_init_walkers_msd; Sec. V:
|psi_T> = sum_I c_I |D_I>, here non-orthogonal) against the oracle (oracle/msd.py, pinned
against Fock-space vectors).

Parity bar as for one determinant: local energies, weights and log-overlaps <psi_T|Phi> to
1e-10 relative at every step (phases modulo 2 pi), walkers to 1e-9, in the phaseless,
local-energy and free-projection modes; the trial energy enters every weight, so the
variational energy through S_IJ is checked with them.  A one-determinant expansion runs the
single-determinant path, and the calls that need one determinant reject an expansion."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.msd import MSDTrial
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


def msd_system(seed, M, Nu, Nd, nch, ND):
    """A non-orthogonal expansion around the lowest orbitals of h."""
    rng = np.random.default_rng(seed)
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    P = syn.make_trial(h, Nu, Nd)
    dets = [(P[0] + 0.3 * crandn(rng, M, Nu), P[1] + 0.3 * crandn(rng, M, Nd)) for _ in range(ND)]
    c = crandn(rng, ND)
    return h, L, E0, MSDTrial(dets, c), rng


def run_parity(h, L, E0, trial, W, tau, nsteps, k_qr, x, Phi0=None, mode="phaseless", fb_cap=1.0):
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=tau, k_taylor=6, k_qr=k_qr, fb_cap=fb_cap, mode=mode)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, trial, W, Phi0, complex_weights=(mode == "free"))
    wm = {"free": api.WEIGHT_FREE, "local": api.WEIGHT_LOCAL}.get(mode, api.WEIGHT_PHASELESS)
    Du = np.stack([d[0] for d in trial.dets])
    Dd = np.stack([d[1] for d in trial.dets])
    with AFQMC(h, L, E0, Du, Dd, W, tau, Phi0=Phi0, k_qr=k_qr, fb_cap=fb_cap, weight_mode=wm,
               coeffs=trial.c) as g:
        E_L, _, logS, _ = g.energy()
        assert rel(E_L, trial.local_energy(ham, wk.Phi)[0]) < RTOL
        ref_ls = trial.log_overlap(wk.Phi)
        assert rel(logS.real, ref_ls.real) < RTOL and phase_close(logS, ref_ls, RTOL * 10)
        for s in range(nsteps):
            _, Emix_ref = O.step(ham, trial, B, wk, x[s], p)
            trace = g.step(1, x[s:s + 1], measure_every=1)
            assert abs(trace[0] - Emix_ref) < RTOL * abs(Emix_ref), (s, trace[0], Emix_ref)
            E_L, w, logS, _ = g.energy()
            assert rel(E_L, trial.local_energy(ham, wk.Phi)[0]) < RTOL, s
            assert rel(w, wk.w) < RTOL, s
            assert rel(logS.real, wk.logS.real) < RTOL, s
            assert phase_close(logS, wk.logS, RTOL * 10), s
        Pu, Pd, _, step = g.walkers()
        assert step == nsteps
        assert rel(Pu, wk.Phi[0]) < 1e-9 and rel(Pd, wk.Phi[1]) < 1e-9
    return wk


def test_msd_ragged_trajectory_matches_oracle():
    """Three non-orthogonal determinants, N_up != N_dn, sizes off the tile grid, complex
    coefficients, random walkers, force-bias cap active, QR every other step."""
    M, Nu, Nd, nch, W, steps = 12, 3, 2, 7, 5, 5
    h, L, E0, trial, rng = msd_system(41, M, Nu, Nd, nch, 3)
    Phi0 = [syn.make_random_walkers(M, Nu, W, 7), syn.make_random_walkers(M, Nd, W, 8)]
    x = rng.standard_normal((steps, W, nch))
    run_parity(h, L, 0.5, trial, W, 0.01, steps, 2, x, Phi0=Phi0, fb_cap=0.05)


@pytest.mark.parametrize("mode", ["phaseless", "local", "free"])
def test_msd_weight_modes_from_the_largest_determinant(mode):
    """Walkers start at the determinant with the largest |c_I| (the second one here)."""
    M, N, nch, W, steps = 16, 4, 10, 4, 4
    h, L, E0, trial, rng = msd_system(43, M, N, N, nch, 4)
    trial.c[1] = 3.0 + 1.0j
    x = rng.standard_normal((steps, W, nch))
    run_parity(h, L, E0, trial, W, 0.005, steps, 3, x, mode=mode)
    assert trial.reference() is trial.dets[1]


def test_one_determinant_expansion_is_the_single_determinant_path():
    M, N, nch, W = 14, 3, 9, 4
    h, L, E0, trial, rng = msd_system(44, M, N, N, nch, 1)
    D = trial.dets[0]
    x = rng.standard_normal((3, W, nch))
    with AFQMC(h, L, E0, D[0], D[1], W, 0.01) as g1, \
            AFQMC(h, L, E0, D[0][None], D[1][None], W, 0.01, coeffs=[2.0 - 1.0j]) as g2:
        assert np.array_equal(g1.step(3, x, measure_every=1), g2.step(3, x, measure_every=1))


def test_msd_rejections():
    M, N, nch, W = 64, 32, 16, 2
    h, L, E0, trial, _ = msd_system(45, M, N, N, nch, 2)
    Du = np.stack([d[0].real.copy() for d in trial.dets]).astype(np.complex128)
    Dd = Du.copy()

    def code(**kw):
        with pytest.raises(api.AfqmcError) as e:
            AFQMC(h, L, E0, Du, Dd, W, 0.01, **kw)
        return e.value.code

    assert code(coeffs=trial.c, precision=api.PREC_BF16X3) == -8
    assert code(coeffs=[0.0, 0.0]) == -1
    assert code(coeffs=[1.0, np.nan]) == -4
    with AFQMC(h, L, E0, Du, Dd, W, 0.01, coeffs=trial.c) as g:
        with pytest.raises(api.AfqmcError) as e:
            g.backward(np.ones(W, complex))
        assert e.value.code == -8
        with pytest.raises(api.AfqmcError) as e:
            g.bp_begin(2)
        assert e.value.code == -8
    ham = api.afqmc_create_hamiltonian(h, L, E0, M, nch)
    try:
        with pytest.raises(api.AfqmcError) as e:
            api.afqmc_init_walkers_msd(ham, 0, Du, Dd, trial.c, N, N, W, None, 0.01)
        assert e.value.code == -2
    finally:
        api.afqmc_destroy_hamiltonian(ham)
