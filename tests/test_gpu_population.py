"""Local-energy weights and comb population control on the GPU against the oracle.

* Local-energy mode (FP64 path): per-walker E_L, weights and log-overlaps to 1e-10 of the
  oracle's local mode at every step; mixed precision against FP64 within 1 mHa in E_mix.
* Comb: the indices are an integer decision taken from FP64 running sums in the same order
  on both sides, so they must agree exactly; the copied walkers and the equal weights follow.
  After the comb the FP64 trajectory continues to match the oracle's."""
import numpy as np
import pytest

from oracle import afqmc as O
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC
from test_gpu_fp64 import make_system, rel, run_parity

pytestmark = pytest.mark.gpu

MHA = 1e-3


def test_local_energy_mode_matches_oracle_fp64():
    wl = syn.WORKLOADS["m24"]
    h, L, E0, Psi = make_system(wl)
    x = syn.make_fields(20, wl.W, wl.Nchol, seed=3)
    wk = run_parity(h, L, E0, Psi, wl.W, wl.tau, 20, wl.k_qr, x, mode="local", check_every=4)
    assert np.std(wk.w) > 1e-4          # the weights did move


def test_local_energy_mode_mixed_vs_fp64():
    rng = np.random.default_rng(21)
    M, N, nch, W, steps = 128, 32, 640, 16, 8
    h, L, E0 = syn.make_hamiltonian(M, nch, rng, decay=20.0)
    Psi = syn.make_trial(h, N, N)
    x = syn.make_fields(steps, W, nch, seed=5)
    traces = []
    for prec in (api.PREC_FP64, api.PREC_BF16X3):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.005, k_qr=5, precision=prec,
                   weight_mode=api.WEIGHT_LOCAL) as g:
            traces.append(g.step(steps, x, measure_every=1))
            w = g.walkers()[2]
    d = np.max(np.abs(traces[0] - traces[1]))
    print("local-energy mode, max |dE_mix| mixed vs FP64 (Ha):", d)
    assert d < MHA


def weights_after(g, steps, x):
    g.step(steps, x, measure_every=0)
    return g.walkers()


@pytest.mark.parametrize("prec,M,N,nch", [(api.PREC_FP64, 24, 5, 120), (api.PREC_BF16X3, 64, 16, 128)])
def test_comb_indices_and_walkers(prec, M, N, nch):
    rng = np.random.default_rng(4)
    W = 64
    h, L, E0 = syn.make_hamiltonian(M, nch, rng, decay=20.0)
    Psi = syn.make_trial(h, N, N)
    x = syn.make_fields(6, W, nch, seed=9) * 3.0      # wide fields: weights spread out
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.05, k_qr=0, precision=prec) as g:
        Pu, Pd, w, step = weights_after(g, 6, x)
        assert np.std(w) > 0.05 * np.mean(w)
        for xi in (0.137, 0.8):
            idx = g.population_control(xi)
            ref = O.comb(w, xi)
            assert np.array_equal(idx, ref), (idx, ref)
            Pu2, Pd2, w2, _ = g.walkers()
            assert np.allclose(w2, np.sum(w) / W, rtol=1e-14)
            assert rel(Pu2, Pu[ref]) < 1e-12 and rel(Pd2, Pd[ref]) < 1e-12
            Pu, Pd, w = Pu2, Pd2, w2


def test_trajectory_after_comb_matches_oracle():
    """FP64 path: steps, comb (same xi on both sides), more steps; per-walker parity at 1e-10."""
    wl = syn.WORKLOADS["m24"]
    h, L, E0, Psi = make_system(wl)
    W = wl.W
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=0.02, k_taylor=6, k_qr=5)
    B = O.half_one_body_propagator(ham, p.tau)
    wk = O.init_walkers(ham, Psi, W)
    x = syn.make_fields(12, W, wl.Nchol, seed=13) * 2.0
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, p.tau, k_qr=5) as g:
        for s in range(6):
            O.step(ham, Psi, B, wk, x[s], p)
        g.step(6, x[:6], measure_every=0)
        idx = g.population_control(0.42)
        ref = O.population_control(wk, 0.42)
        assert np.array_equal(idx, ref)
        for s in range(6, 12):
            E_ref, Emix_ref = O.step(ham, Psi, B, wk, x[s], p)
            tr = g.step(1, x[s:s + 1], measure_every=1)
            assert abs(tr[0] - Emix_ref) < 1e-10 * abs(Emix_ref), s
        E_L, w, logS, _ = g.energy()
        assert rel(w, wk.w) < 1e-10
        assert rel(E_L, O.local_energy(ham, Psi, wk.Phi)[0]) < 1e-10


def test_population_control_rejects_bad_input():
    rng = np.random.default_rng(1)
    h, L, E0 = syn.make_hamiltonian(16, 8, rng, decay=5.0)
    Psi = syn.make_trial(h, 3, 3)
    with AFQMC(h, L, E0, Psi[0], Psi[1], 4, 0.01) as g:
        for xi in (1.0, -0.1, float("nan")):
            with pytest.raises(RuntimeError):
                g.population_control(xi)
        g.set_walkers(*g.walkers()[:2], np.zeros(4), 0)
        with pytest.raises(RuntimeError):
            g.population_control(0.5)                     # no live walker
    with AFQMC(h, L, E0, Psi[0], Psi[1], 4, 0.01, weight_mode=api.WEIGHT_FREE) as g:
        with pytest.raises(RuntimeError):
            g.population_control(0.5)                     # complex weights


def test_standalone_comb_indices_match_oracle():
    """afqmc_comb_indices: the same kernel and rule on any weight vector."""
    rng = np.random.default_rng(9)
    w = rng.uniform(0.2, 2.0, 37)
    w[[3, 17]] = 0.0
    for xi in (0.13, 0.5, 0.91):
        idx, total = api.afqmc_comb_indices(w, xi)
        assert np.array_equal(idx, O.comb(w, xi))
        assert abs(total - np.sum(w)) < 1e-12 * np.sum(w)
    with pytest.raises(api.AfqmcError) as e:
        api.afqmc_comb_indices(np.zeros(4), 0.5)
    assert e.value.code == -1


def test_population_wide_comb_on_one_rank_equals_the_walker_set_comb():
    """distributed.population_control (gathered weights, library comb, walker exchange, then
    set_walkers) on a one-rank gloo group gives the walkers, weights and trajectory of
    afqmc_population_control."""
    import os
    import socket
    import torch.distributed as dist
    from paper_2003_01831_gb300 import distributed as D
    rng = np.random.default_rng(10)
    M, N, nch, W = 12, 3, 10, 9
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.02) as g1, AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.02) as g2:
            g1.step(3, seed=4)
            g2.step(3, seed=4)
            idx1 = g1.population_control(0.29)
            idx2 = D.population_control(g2, 0.29)
            assert np.array_equal(idx1, idx2)
            a, b = g1.walkers(), g2.walkers()
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
            t1 = g1.step(2, seed=4, measure_every=1)
            t2 = g2.step(2, seed=4, measure_every=1)
            assert np.max(np.abs(t1 - t2)) <= 1e-13 * np.max(np.abs(t1))
    finally:
        dist.destroy_process_group()
