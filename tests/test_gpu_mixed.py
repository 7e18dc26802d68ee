"""Mixed-precision (BF16X3 tensor-core) walker step vs the FP64 GPU path and the oracle.

Bar: |E_mix(BF16X3) - E_mix(FP64)| <= 1 mHa per measured step with identical fields and
initial walkers; per-walker local energies and weights close to the FP64 ones."""
import numpy as np
import pytest

from oracle import afqmc as O
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

MHA = 1e-3


def system(M, N, nch, seed, band=None, decay=20.0):
    rng = np.random.default_rng(seed)
    h, L, E0 = syn.make_hamiltonian(M, nch, rng, decay=decay, band=band)
    Psi = syn.make_trial(h, N, N)
    return h, L, E0, Psi


def pair(h, L, E0, Psi, W, tau, k_qr, Phi0=None):
    a = AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, Phi0=Phi0, k_qr=k_qr, precision=api.PREC_FP64)
    b = AFQMC(h, L, E0, Psi[0], Psi[1], W, tau, Phi0=Phi0, k_qr=k_qr, precision=api.PREC_BF16X3)
    return a, b


@pytest.mark.parametrize("M,N,nch,W", [(128, 32, 640, 16), (128, 64, 256, 8), (256, 128, 512, 4)])
def test_energy_at_start_matches_fp64(M, N, nch, W):
    """Walkers near the trial (trial + 0.1 x complex Gaussian, orthonormalised), the regime a
    phaseless run lives in; the overlap matrices are well conditioned there."""
    h, L, E0, Psi = system(M, N, nch, 11)
    rng = np.random.default_rng(5)
    Phi0 = []
    amp = 0.8 / np.sqrt(M)       # perturbation norm ~1 per column: overlap condition numbers O(10)
    for s in range(2):
        z = Psi[s][None] + amp * (rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N)))
        Phi0.append(np.linalg.qr(z)[0])
    a, b = pair(h, L, E0, Psi, W, 0.005, 5, Phi0)
    with a, b:
        Ea, wa, la, Ema = a.energy()
        Eb, wb, lb, Emb = b.energy()
    assert np.max(np.abs(Ea - Eb)) < MHA, np.max(np.abs(Ea - Eb))
    assert abs(Ema - Emb) < MHA
    assert np.max(np.abs(la.real - lb.real)) < 1e-3
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    Eo = O.local_energy(ham, Psi, Phi0)[0]
    assert np.max(np.abs(Eb - Eo)) < MHA


def test_single_product_tail_matches_rounded_three():
    """The default energy products (rounded three, with single-product tiles for the Cholesky
    vectors whose squared norms make up at most 2^-15 of the total) against the rounded three on
    every tile, on the same walkers of the molecule-like M = 128 shape, where the tail is most of
    the tiles: the mean product count drops below 2, and the local energies and force-bias-driven
    log-overlaps agree far inside the 1 mHa bar."""
    import ctypes
    M, N, nch, W = 128, 32, 640, 16
    h, L, E0, Psi = system(M, N, nch, 11)
    rng = np.random.default_rng(5)
    amp = 0.8 / np.sqrt(M)
    Phi0 = [np.linalg.qr(Psi[s][None] + amp * (rng.standard_normal((W, M, N))
                                                 + 1j * rng.standard_normal((W, M, N))))[0] for s in range(2)]
    lib = api.lib()
    lib.afqmc_debug_energy_products.restype = ctypes.c_int
    lib.afqmc_debug_energy_products.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    x = syn.make_fields(3, W, nch, seed=4)
    out = {}
    for terms in (0, 2):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.005, Phi0=Phi0, k_qr=5, precision=api.PREC_BF16X3,
                   energy_terms=terms) as g:
            mean = ctypes.c_double(0.0)
            assert lib.afqmc_debug_energy_products(g.wk, ctypes.addressof(mean)) == 0
            E0_L = g.energy()[0]
            tr = g.step(3, x, measure_every=1)
            out[terms] = (mean.value, E0_L, tr, g.energy())
    print("mean products:", out[0][0], out[2][0])
    assert out[2][0] == 3.0 and 1.0 <= out[0][0] < 2.0
    dE = np.max(np.abs(out[0][1] - out[2][1]))
    dmix = np.max(np.abs(out[0][2] - out[2][2]))
    dlog = np.max(np.abs(out[0][3][2].real - out[2][3][2].real))
    print(f"single tail vs rounded three: E_L {dE:.2e} Ha, E_mix over 3 steps {dmix:.2e} Ha, log-overlap {dlog:.2e}")
    assert dE < 2e-5 and dmix < 5e-5 and dlog < 1e-5


@pytest.mark.parametrize("M,N,nch,W,steps,me", [(128, 32, 640, 32, 12, 1), (128, 64, 256, 8, 8, 3),
                                                 (256, 128, 512, 4, 6, 1), (128, 24, 320, 12, 8, 1)])
def test_trajectory_matches_fp64_within_1mha(M, N, nch, W, steps, me):
    h, L, E0, Psi = system(M, N, nch, 21)
    x = syn.make_fields(steps, W, nch, seed=0)
    a, b = pair(h, L, E0, Psi, W, 0.005, 5)
    with a, b:
        ta = a.step(steps, x, measure_every=me)
        tb = b.step(steps, x, measure_every=me)
        assert np.max(np.abs(ta - tb)) < MHA, np.abs(ta - tb)
        Ea, wa, la, _ = a.energy()
        Eb, wb, lb, _ = b.energy()
        assert np.max(np.abs(Ea - Eb)) < 10 * MHA
        # E_mix depends on relative weights only; a common factor per step (the split
        # representation of B = exp(-tau h'/2) is the same for every walker) cancels
        ra, rb = wa / np.mean(wa), wb / np.mean(wb)
        print(f"M={M} N={N} every {me}: |dE_mix| {np.max(np.abs(ta - tb)):.2e}, |dE_L| {np.max(np.abs(Ea - Eb)):.2e}, "
              f"relative weights {np.max(np.abs(ra - rb) / np.abs(ra)):.2e}")
        assert np.max(np.abs(ra - rb) / np.abs(ra)) < 1e-3
        Pa = a.walkers()
        Pb = b.walkers()
        assert Pa[3] == Pb[3] == steps


def test_mixed_vs_oracle_m128():
    """M=128, N=32+32, Nchol=640 at 4 walkers: BF16X3 trajectory within 1 mHa of the oracle."""
    wl = syn.WORKLOADS["m128"]
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    W, ns = 4, 3
    x = syn.make_fields(ns, W, wl.Nchol, seed=0)
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=wl.tau, k_taylor=6, k_qr=2)
    B = O.half_one_body_propagator(ham, wl.tau)
    wk = O.init_walkers(ham, Psi, W)
    ref = [O.step(ham, Psi, B, wk, x[s], p)[1] for s in range(ns)]
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=2, precision=api.PREC_BF16X3) as g:
        got = g.step(ns, x, measure_every=1)
        E_L, w, logS, _ = g.energy()
    assert np.max(np.abs(got - np.array(ref))) < MHA
    assert np.max(np.abs(E_L - O.local_energy(ham, Psi, wk.Phi)[0])) < MHA
    assert np.max(np.abs(w / w.mean() - wk.w / wk.w.mean()) / (wk.w / wk.w.mean())) < 1e-3


def test_unsupported_shapes_rejected():
    h, L, E0, Psi = system(96, 24, 40, 3)
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, L, E0, Psi[0], Psi[1], 2, 0.01, precision=api.PREC_BF16X3)
    assert e.value.code == -8


def test_spin_unrestricted_trial_rejected():
    """The tensor-core path forms one trial operand for both spins, so a real trial with
    Psi_up != Psi_dn (same N) is refused rather than run with Psi_dn replaced by Psi_up; the FP64
    path takes it."""
    h, L, E0, Psi = system(128, 32, 64, 5)
    _, v = np.linalg.eigh(h)
    Pdn = np.ascontiguousarray(v[:, 1:33].astype(np.complex128))   # a different real determinant
    with pytest.raises(api.AfqmcError) as e:
        AFQMC(h, L, E0, Psi[0], Pdn, 4, 0.01, precision=api.PREC_BF16X3)
    assert e.value.code == -8 and "Psi_up == Psi_dn" in str(e.value)
    with AFQMC(h, L, E0, Psi[0], Pdn, 4, 0.01, precision=api.PREC_FP64) as g:
        assert np.isfinite(g.energy()[3])


@pytest.mark.parametrize("M,N,nch,W", [(128, 32, 64, 4), (256, 128, 96, 3)])
def test_qr_matches_fp64_path(M, N, nch, W):
    """One step with a QR at its end (k_qr = 1): the mixed path's Cholesky QR (tensor-core Gram
    and R^-1 product) leaves orthonormal walkers, equal to the FP64 path's Q (R has a positive
    real diagonal, so Q is unique) up to the step's mixed-precision error."""
    h, L, E0, Psi = system(M, N, nch, 31)
    x = syn.make_fields(1, W, nch, seed=4)
    a, b = pair(h, L, E0, Psi, W, 0.01, 1)
    with a, b:
        a.step(1, x, measure_every=0)
        b.step(1, x, measure_every=0)
        Qa = a.walkers()
        Qb = b.walkers()
    for s in range(2):
        G = np.einsum("wki,wkj->wij", Qb[s].conj(), Qb[s])
        orth = np.max(np.abs(G - np.eye(N)))
        diff = np.max(np.abs(Qb[s] - Qa[s]))
        print(f"M={M} N={N} spin {s}: |Q^H Q - I| {orth:.2e}, |Q - Q_fp64| {diff:.2e}")
        assert orth < 1e-7
        assert diff < 1e-6
