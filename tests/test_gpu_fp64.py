"""GPU FP64 path vs the CPU oracle: per-walker trajectories with identical fields.

Parity bar (FP64): local energies, weights and log-overlaps agree to 1e-10
relative at every step (phase of logS compared modulo 2 pi)."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.philox import philox_fields
from paper_2003_01831_gb300 import api, synthetic as syn

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_01831_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def make_system(wl, W=None):
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band, reading=wl.reading)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    return h, L, E0, Psi


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def phase_close(a, b, tol):
    return np.max(np.abs(np.exp(1j * (a.imag - b.imag)) - 1)) < tol


def run_parity(h, L, E0, Psi, W, tau, nsteps, k_qr, x, Phi0=None, fb_cap=1.0, mode="phaseless", K=6,
               check_every=1):
    from paper_2003_01831_gb300.walkers import AFQMC
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=tau, k_taylor=K, k_qr=k_qr, fb_cap=fb_cap, mode=mode)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, Psi, W, Phi0, complex_weights=(mode == "free"))
    wm = {"free": api.WEIGHT_FREE, "local": api.WEIGHT_LOCAL}.get(mode, api.WEIGHT_PHASELESS)
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, Phi0=Phi0, k_taylor=K, k_qr=k_qr, fb_cap=fb_cap,
               weight_mode=wm) as g:
        E_L, w, logS, Emix = g.energy()
        assert rel(E_L, O.local_energy(ham, Psi, wk.Phi)[0]) < RTOL
        for s in range(nsteps):
            E_ref, Emix_ref = O.step(ham, Psi, B, wk, x[s], p)
            trace = g.step(1, x[s:s + 1], measure_every=1)
            assert abs(trace[0] - Emix_ref) < RTOL * abs(Emix_ref), (s, trace[0], Emix_ref)
            if s % check_every == 0 or s == nsteps - 1:
                E_L, w, logS, Emix = g.energy()
                E_now = O.local_energy(ham, Psi, wk.Phi)[0]
                assert rel(E_L, E_now) < RTOL, s
                assert rel(w, wk.w) < RTOL, s
                assert rel(logS.real, wk.logS.real) < RTOL, s
                assert phase_close(logS, wk.logS, RTOL * 10), s
        Pu, Pd, wg, step = g.walkers()
        assert step == nsteps
        assert rel(Pu, wk.Phi[0]) < 1e-9 and rel(Pd, wk.Phi[1]) < 1e-9
    return wk


def test_m24_full_trajectory():
    """Molecule-like workload: M=24, N=5+5, Nchol=120, 16 walkers, tau=0.005, 50 steps, QR/5."""
    wl = syn.WORKLOADS["m24"]
    h, L, E0, Psi = make_system(wl)
    x = syn.make_fields(wl.nsteps, wl.W, wl.Nchol, seed=0)
    run_parity(h, L, E0, Psi, wl.W, wl.tau, wl.nsteps, wl.k_qr, x, check_every=5)


def test_m128_sampled_walkers():
    """M=128, N=32+32, Nchol=640 at reduced walkers/steps (oracle cost)."""
    wl = syn.WORKLOADS["m128"]
    h, L, E0, Psi = make_system(wl)
    W, ns = 6, 4
    x = syn.make_fields(ns, W, wl.Nchol, seed=0)
    run_parity(h, L, E0, Psi, W, wl.tau, ns, 2, x, check_every=1)


def test_ragged_uhf_complex_trial_random_walkers():
    """N_up != N_dn, sizes that are not tile multiples, complex trial, random walkers,
    force-bias cap active, QR every step."""
    rng = np.random.default_rng(77)
    M, Nu, Nd, nch, W = 37, 7, 3, 53, 5
    h, L, E0 = syn.make_hamiltonian(M, nch, rng, decay=10.0)
    E0 = 1.25
    Psi = list(syn.make_trial(h, Nu, Nd))
    Psi = [p + 0.2 * (rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)) for p in Psi]
    Phi0 = [syn.make_random_walkers(M, Nu, W, 3), syn.make_random_walkers(M, Nd, W, 4)]
    x = rng.standard_normal((6, W, nch))
    run_parity(h, L, E0, Psi, W, 0.01, 6, 1, x, Phi0=Phi0, fb_cap=0.05)


def test_free_projection_mode():
    rng = np.random.default_rng(5)
    M, N, nch, W = 16, 3, 30, 7
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    x = rng.standard_normal((5, W, nch))
    run_parity(h, L, E0, Psi, W, 0.02, 5, 3, x, mode="free")


def test_single_walker_and_high_taylor_order():
    rng = np.random.default_rng(9)
    M, N, nch, W = 20, 4, 40, 1
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    x = rng.standard_normal((3, W, nch))
    run_parity(h, L, E0, Psi, W, 0.01, 3, 0, x, K=12)


def test_zero_field_one_body_limit():
    """L = 0, x = 0: one step maps Phi to exp(-tau h) Phi."""
    import scipy.linalg
    from paper_2003_01831_gb300.walkers import AFQMC
    rng = np.random.default_rng(3)
    M, N, W = 12, 3, 4
    h, _, _ = syn.make_hamiltonian(M, 1, rng)
    L = np.zeros((2, M, M))
    Psi = syn.make_trial(h, N, N)
    Phi0 = [syn.make_random_walkers(M, N, W, 11), syn.make_random_walkers(M, N, W, 12)]
    with AFQMC(h, L, 0.0, Psi[0], Psi[1], W, 0.05, Phi0=Phi0, k_qr=0) as g:
        g.step(1, np.zeros((1, W, 2)))
        Pu, Pd, w, _ = g.walkers()
    E = scipy.linalg.expm(-0.05 * h)
    assert rel(Pu, np.matmul(E, Phi0[0])) < 1e-12
    assert rel(Pd, np.matmul(E, Phi0[1])) < 1e-12


def test_philox_fields_match_oracle_and_drive_steps():
    from paper_2003_01831_gb300.walkers import AFQMC
    W, nch = 9, 37
    for step in (0, 5, 123456):
        x = np.zeros((W, nch))
        api.afqmc_philox_fields(0xDEADBEEF12345, step, W, nch, x)
        assert rel(x, philox_fields(0xDEADBEEF12345, step, W, nch)) < 1e-13
    # a run with device-drawn fields equals a run fed the oracle's fields
    rng = np.random.default_rng(2)
    M, N, nch = 14, 3, 21
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    seed = 77
    xs = np.stack([philox_fields(seed, s, W, nch) for s in range(4)])
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01) as g1, AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01) as g2:
        t1 = g1.step(4, None, seed=seed, measure_every=1)
        t2 = g2.step(4, xs, measure_every=1)
        assert rel(t1, t2) < 1e-12
        assert rel(g1.walkers()[0], g2.walkers()[0]) < 1e-12


def test_checkpoint_resume_and_dead_walkers():
    from paper_2003_01831_gb300.walkers import AFQMC
    rng = np.random.default_rng(8)
    M, N, nch, W = 18, 4, 30, 6
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, k_qr=2) as g, \
            AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, k_qr=2) as g2:
        g.step(3, None, seed=5)
        Pu, Pd, w, step = g.walkers()
        w = w.copy()
        w[2] = 0.0                       # kill walker 2: it must stay frozen
        g.set_walkers(Pu, Pd, w, step)
        g2.set_walkers(Pu, Pd, w, step)
        a = g.step(4, None, seed=5, measure_every=2)
        b = g2.step(4, None, seed=5, measure_every=2)
        assert np.array_equal(a, b)      # resumed runs are bitwise reproducible
        Pu2, Pd2, w2, step2 = g.walkers()
        assert step2 == step + 4
        assert w2[2] == 0.0
        assert np.array_equal(Pu2[2], Pu[2]) and np.array_equal(Pd2[2], Pd[2])
        assert np.all(w2[[0, 1, 3, 4, 5]] > 0)


def test_error_paths():
    from paper_2003_01831_gb300.walkers import AFQMC
    rng = np.random.default_rng(1)
    M, N, nch, W = 10, 2, 6, 3
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    bad = L.copy()
    bad[1, 2, 3] += 0.5
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, bad, E0, Psi[0], Psi[1], W, 0.01)
    assert e.value.code == -8
    hn = h.copy()
    hn[0, 0] = np.nan
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(hn, L, E0, Psi[0], Psi[1], W, 0.01)
    assert e.value.code == -4
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01) as g:
        x = np.zeros((1, W, nch))
        x[0, 1, 2] = np.inf
        with pytest.raises(api.AfqmcError) as e:
            g.step(1, x)
        assert e.value.code == -4
    with pytest.raises(api.AfqmcError) as e:   # zero walkers: exactly singular overlap
        Z = np.zeros((W, M, N), complex)
        AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=[Z, Z])
    assert e.value.code == -5
