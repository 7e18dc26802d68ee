"""Batches of independent uneven systems (one CUDA-graph launch per step).

* FP64 batch, unpadded and padded to the tensor-core shapes, against the oracle run on each
  unpadded system with the same Philox fields: per-walker E_L, w, logS to 1e-10 relative
  (the padding is exact: decoupled orbitals, one extra electron per extra orbital, zero
  Cholesky vectors).
* The replayed graph reproduces afqmc_step on each system alone (FP64 and BF16X3).
* BF16X3 batch (padded where needed) against the FP64 batch: E_mix within 1 mHa per step.
* The autotuner restores the walkers it advanced."""
import numpy as np
import pytest

from oracle import afqmc as O
from oracle.philox import philox_fields
from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC, Batch

pytestmark = pytest.mark.gpu

RTOL = 1e-10
MHA = 1e-3
MASK64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2003_01831_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available()


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def systems(dims, seed=7):
    out = []
    for i, d in enumerate(dims):
        h, L, E0, Psi = syn.make_uneven_system(d, i, seed=seed)
        out.append((h, L, E0, Psi[0], Psi[1], d.W))
    return out


SMALL = [syn.UnevenSystem(M=12, N=3, Nchol=30, W=4), syn.UnevenSystem(M=17, N=4, Nchol=43, W=3),
         syn.UnevenSystem(M=9, N=2, Nchol=21, W=5)]


def oracle_run(sysdef, s, seed, nsteps, tau, k_qr):
    h, L, E0, Pu, Pd, W = sysdef
    ham = O.Hamiltonian(h=h, L=L, E0=E0)
    p = O.Params(tau=tau, k_taylor=6, k_qr=k_qr)
    B = O.half_one_body_propagator(ham, tau)
    wk = O.init_walkers(ham, (Pu, Pd), W)
    key = (seed + s * api.SEED_STRIDE) & MASK64
    emix = []
    for t in range(nsteps):
        x = philox_fields(key, t, W, L.shape[0])
        emix.append(O.step(ham, (Pu, Pd), B, wk, x, p)[1])
    E_now = O.local_energy(ham, (Pu, Pd), wk.Phi)[0]
    return np.array(emix), wk, E_now


@pytest.mark.parametrize("pad", [api.PAD_AUTO, api.PAD_ALWAYS])
def test_fp64_batch_matches_oracle(pad):
    sysdefs = systems(SMALL)
    tau, k_qr, nsteps, seed = 0.01, 3, 7, 11
    with Batch(sysdefs, tau, k_qr=k_qr, pad_mode=pad) as b:
        if pad == api.PAD_ALWAYS:
            shape, _ = b.info(0)
            assert tuple(shape[:3]) == (64, 8, 32)    # M' >= 12 + 5, N' = 8, Nchol' = 32
        trace = b.step(nsteps, seed=seed, measure_every=1)
        for s, sd in enumerate(sysdefs):
            emix, wk, E_now = oracle_run(sd, s, seed, nsteps, tau, k_qr)
            assert rel(trace[:, s], emix) < RTOL, s
            E_L, w, logS, _ = b.energy(s)
            assert rel(E_L, E_now) < RTOL, s
            assert rel(w, wk.w) < RTOL, s
            assert rel(logS.real, wk.logS.real) < RTOL, s
            Pu, Pd, wg, step = b.walkers(s)
            assert step == nsteps
            assert rel(Pu, wk.Phi[0]) < 1e-9 and rel(Pd, wk.Phi[1]) < 1e-9


@pytest.mark.parametrize("prec", [api.PREC_FP64, api.PREC_BF16X3])
def test_graph_replay_matches_single_system_steps(prec):
    """No padding needed (M % 64 == 0, N = 32): the batch graph and afqmc_step run the same
    kernels, so the trajectories agree to rounding (QR every 4 steps, 9 steps)."""
    dims = [syn.UnevenSystem(M=64, N=32, Nchol=64, W=6), syn.UnevenSystem(M=128, N=32, Nchol=96, W=5)]
    sysdefs = systems(dims, seed=3)
    tau, k_qr, nsteps, seed = 0.01, 4, 9, 5
    with Batch(sysdefs, tau, precision=prec, k_qr=k_qr) as b:
        trace = b.step(nsteps, seed=seed, measure_every=1)
        for s, (h, L, E0, Pu, Pd, W) in enumerate(sysdefs):
            with AFQMC(h, L, E0, Pu, Pd, W, tau, precision=prec, k_qr=k_qr) as g:
                tr = g.step(nsteps, seed=(seed + s * api.SEED_STRIDE) & MASK64, measure_every=1)
                assert rel(trace[:, s], tr) < 1e-12, s
                assert rel(b.energy(s)[0], g.energy()[0]) < 1e-12, s


def test_mixed_batch_within_1mha_of_fp64():
    """Uneven shapes padded for the tensor cores (M, N, Nchol not tileable)."""
    dims = [syn.UnevenSystem(M=40, N=10, Nchol=200, W=16), syn.UnevenSystem(M=100, N=25, Nchol=500, W=12),
            syn.UnevenSystem(M=72, N=18, Nchol=360, W=20)]
    sysdefs = systems(dims, seed=9)
    tau, k_qr, nsteps, seed = 0.01, 10, 12, 2
    traces = {}
    for prec in (api.PREC_FP64, api.PREC_BF16X3):
        with Batch(sysdefs, tau, precision=prec, k_qr=k_qr) as b:
            traces[prec] = b.step(nsteps, seed=seed, measure_every=1)
            if prec == api.PREC_BF16X3:
                shape, nk = b.info(1)
                assert tuple(shape[:3]) == (128, 32, 504) and nk > 0
    d = np.abs(traces[api.PREC_FP64] - traces[api.PREC_BF16X3])
    print("max |dE_mix| per system (Ha):", d.max(axis=0))
    assert d.max() < MHA


def test_energy_launch_forms_agree():
    """One persistent energy launch over every system's tiles (K chunks of 32 or 16) and one
    launch per system: the same tiles, the same arithmetic, the same trajectories.  The systems
    pad to three different tile shapes (N' = 16 and 104: the generic epilogue, 8 and 1
    walker-spins per tile; N' = 32: a fixed-N' epilogue), so one launch mixes them."""
    import ctypes
    dims = [syn.UnevenSystem(M=40, N=10, Nchol=200, W=9), syn.UnevenSystem(M=160, N=32, Nchol=96, W=7),
            syn.UnevenSystem(M=400, N=100, Nchol=64, W=3)]
    sysdefs = systems(dims, seed=13)
    tau, k_qr, nsteps, seed = 0.01, 4, 6, 3
    lib = api.lib()
    lib.afqmc_debug_set_batch_energy.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    traces, energies = [], []
    for multi, bk in ((1, 32), (1, 16), (0, 32)):
        with Batch(sysdefs, tau, precision=api.PREC_BF16X3, k_qr=k_qr) as b:
            assert lib.afqmc_debug_set_batch_energy(b.b, multi, bk) == 0
            assert [int(b.info(s)[0][1]) for s in range(3)] == [16, 32, 104]
            traces.append(b.step(nsteps, seed=seed, measure_every=1))
            energies.append([b.energy(s)[0] for s in range(3)])
            shape, _ = b.info(0)
            assert int(shape[6]) == multi and int(shape[7]) == bk
    for t, e in zip(traces[1:], energies[1:]):
        assert rel(t, traces[0]) < 1e-12
        for s in range(3):
            assert rel(e[s], energies[0][s]) < 1e-12


def test_autotune_restores_walkers():
    dims = [syn.UnevenSystem(M=64, N=32, Nchol=64, W=8), syn.UnevenSystem(M=45, N=11, Nchol=225, W=7),
            syn.UnevenSystem(M=33, N=8, Nchol=165, W=9)]
    sysdefs = systems(dims, seed=4)
    tau, nsteps, seed = 0.01, 4, 8
    with Batch(sysdefs, tau, precision=api.PREC_BF16X3, k_qr=10) as ref:
        t_ref = ref.step(nsteps, seed=seed, measure_every=1)
    with Batch(sysdefs, tau, precision=api.PREC_BF16X3, k_qr=10) as b:
        ms = b.autotune(reps=1)
        assert ms > 0
        shape, _ = b.info(0)
        assert shape[3] >= 1 and shape[4] in (128, 256)
        t = b.step(nsteps, seed=seed, measure_every=1)
    # the tuned launch shape changes no arithmetic order inside a tile
    assert rel(t, t_ref) < 1e-12


def test_batch_errors():
    sd = systems([syn.UnevenSystem(M=12, N=3, Nchol=30, W=4)])
    with pytest.raises(api.AfqmcError):
        Batch(sd, -0.1)
    h, L, E0, Pu, Pd, W = sd[0]
    with pytest.raises(api.AfqmcError):   # padding needs Nup == Ndn
        Batch([(h, L, E0, Pu, Pd[:, :2], W)], 0.01, precision=api.PREC_BF16X3)
    with Batch(sd, 0.01) as b:
        with pytest.raises(api.AfqmcError):
            api.afqmc_batch_energy(b.b, 3)
        with pytest.raises(api.AfqmcError):
            api.afqmc_batch_step(b.b, -1)
