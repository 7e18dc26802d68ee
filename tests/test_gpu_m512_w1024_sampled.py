"""The throughput configuration at full size: M=512, N=128+128, Nchol=2560, W=1024 walkers,
BF16X3, Philox fields drawn on the device, energy measured every step, QR every 5 steps
(six steps, so one QR falls inside), checked on sampled walkers.

The oracle needs minutes per walker-step at this size (its rotated Cholesky tensor alone is
~1e11 multiply-adds), so the full-size checks use properties that hold at any size, and tie
the sampled walkers to the paths that are compared with the oracle at smaller sizes:
- walker independence: walkers j..j+3 of the 1024-walker run equal a set of 4 walkers at
  walker_offset j (Philox keys the fields by the global walker index).  Offsets 0, 126 (a
  128-walker tile edge inside) and 1020 (the last walkers).
- the FP64 GPU path on the same sampled walkers (same offset and seed) gives the same local
  energies within the 1 mHa bar of the mixed path; weights and log-overlaps agree to 1e-4.
- every returned E_L, weight and log-overlap is finite, weights are non-negative, and the
  returned E_mix equals sum w E_L / sum w of the returned arrays."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

MHA = 1e-3
SEED, STEPS, K = 1234, 6, 4
OFFSETS = (0, 126, 1020)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_m512_w1024_sampled_walkers():
    wl = syn.WORKLOADS["m512"]
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, wl.rng(), decay=wl.decay, band=wl.band, reading=wl.reading)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)

    def run(W, prec, off):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=wl.k_qr, precision=prec,
                   walker_offset=off) as g:
            trace = g.step(STEPS, seed=SEED, measure_every=1)
            E_L, w, logS, Emix = g.energy()
            Pu, Pd, _, step = g.walkers()
            assert step == STEPS
            picks = np.concatenate([np.arange(o, o + K) for o in OFFSETS]) if W == wl.W else np.arange(W)
            return dict(trace=trace, E_L=E_L, w=w, logS=logS, Emix=Emix,
                        Pu=Pu[picks].copy(), Pd=Pd[picks].copy())

    full = run(wl.W, api.PREC_BF16X3, 0)
    assert np.all(np.isfinite(full["E_L"])) and np.all(np.isfinite(full["logS"]))
    assert np.all(np.isfinite(full["w"])) and np.all(full["w"] >= 0) and np.any(full["w"] > 0)
    assert np.all(np.isfinite(full["trace"]))
    Emix = np.sum(full["w"] * full["E_L"]) / np.sum(full["w"])
    assert abs(Emix - full["Emix"]) <= 1e-12 * abs(Emix)

    for i, off in enumerate(OFFSETS):
        sl = slice(off, off + K)
        part = run(K, api.PREC_BF16X3, off)
        assert rel(part["E_L"], full["E_L"][sl]) <= 1e-12, off
        assert rel(part["w"], full["w"][sl]) <= 1e-12, off
        assert rel(part["logS"], full["logS"][sl]) <= 1e-12, off
        assert rel(part["Pu"], full["Pu"][i * K:(i + 1) * K]) <= 1e-12, off
        assert rel(part["Pd"], full["Pd"][i * K:(i + 1) * K]) <= 1e-12, off

        ref = run(K, api.PREC_FP64, off)
        dE = np.max(np.abs(ref["E_L"] - part["E_L"]))
        print(f"walkers {off}..{off + K - 1}: max |dE_L| vs FP64 {dE:.3e} Ha, "
              f"weights rel {rel(part['w'], ref['w']):.2e}, "
              f"max |dlogS| {np.max(np.abs(part['logS'] - ref['logS'])):.2e}")
        assert dE < MHA, off
        assert rel(part["w"], ref["w"]) < 1e-4, off
        assert np.max(np.abs(part["logS"].real - ref["logS"].real)) < 1e-4, off
        assert np.max(np.abs(np.exp(1j * (part["logS"].imag - ref["logS"].imag)) - 1)) < 1e-4, off
