"""Mixed precision against FP64 over whole runs at the stated workload sizes.

The mixed-precision (BF16X3) step and the plain FP64 GPU step run the same walkers with the
same fields from the trial; the mixed-estimator energy of every measured step must agree to
1 mHa, the bar for the tensor-core path.  Errors of the mixed path enter the phaseless weights
through the overlap ratio at every step and compound over the run, which is why the whole run
is compared and not only its first steps.

* molecule-like system (M=128, N=32+32, Nchol=640): the stated 512 walkers, 200 steps, QR
  every 10 steps;
* solid-like throughput system (M=512, N=128+128, Nchol=2560, h banded): 16 walkers for the
  stated 100 steps, QR every 5 steps (the FP64 path's energy contraction costs ~1.8e11 flops
  per walker-step, so the walker count is kept small).
"""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

MHA = 1e-3


def run_pair(wl, W, steps):
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    x = syn.make_fields(steps, W, wl.Nchol, seed=0)
    out = {}
    for name, prec in (("fp64", api.PREC_FP64), ("mixed", api.PREC_BF16X3)):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=wl.k_qr, precision=prec) as g:
            out[name] = g.step(steps, x, measure_every=1)
            out[name + "_w"] = g.energy()[1]
    return out


@pytest.mark.parametrize("name,W,steps", [("m128", 512, 200), ("m512", 16, 100)])
def test_mixed_matches_fp64_over_whole_run(name, W, steps):
    wl = syn.WORKLOADS[name]
    assert wl.k_qr in (5, 10)
    out = run_pair(wl, W, steps)
    d = np.abs(out["fp64"] - out["mixed"])
    ra = out["fp64_w"] / np.mean(out["fp64_w"])
    rb = out["mixed_w"] / np.mean(out["mixed_w"])
    print(f"{name}: W={W} steps={steps}: max |dE_mix| {d.max():.3e} Ha (step {int(d.argmax())}), "
          f"last {d[-1]:.3e} Ha; E_mix fp64 first/last {out['fp64'][0].real:.6f} / {out['fp64'][-1].real:.6f}; "
          f"final relative weights max |d| {np.max(np.abs(ra - rb)):.2e}")
    assert np.all(np.isfinite(out["mixed"]))
    assert d.max() < MHA, d
