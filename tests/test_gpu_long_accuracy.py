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
  per walker-step, so the walker count is kept small).  On this system the phaseless cos
  projection removes walkers quickly: without population control all 16 are dead (weight 0,
  E_mix undefined) by step ~97 on both paths, and with a comb every 10 steps (same uniform
  number on both paths, which must pick the same walkers) the copied population still dies
  inside one window near step 94.  The estimator is compared at every step where it is defined,
  and both paths must lose the population at the same step.
"""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

MHA = 1e-3


def run_pair(wl, W, steps, comb_every=0):
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    x = syn.make_fields(steps, W, wl.Nchol, seed=0)
    xi = np.random.default_rng(7).random(steps)
    seg = comb_every or steps
    out = {}
    for name, prec in (("fp64", api.PREC_FP64), ("mixed", api.PREC_BF16X3)):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=wl.k_qr, precision=prec) as g:
            tr, idx = [], []
            for s0 in range(0, steps, seg):
                tr.append(g.step(min(seg, steps - s0), x[s0:s0 + seg], measure_every=1))
                if comb_every and s0 + seg < steps and np.isfinite(tr[-1][-1]):   # no comb of a dead population
                    idx.append(g.population_control(xi[s0]))
            out[name] = np.concatenate(tr)
            out[name + "_idx"] = idx
            out[name + "_w"] = g.energy()[1]
    return out


@pytest.mark.parametrize("name,W,steps,comb_every", [("m128", 512, 200, 0), ("m512", 16, 100, 10)])
def test_mixed_matches_fp64_over_whole_run(name, W, steps, comb_every):
    wl = syn.WORKLOADS[name]
    assert wl.k_qr in (5, 10)
    out = run_pair(wl, W, steps, comb_every)
    for a, b in zip(out["fp64_idx"], out["mixed_idx"]):
        assert np.array_equal(a, b)
    live = np.isfinite(out["fp64"])
    assert np.array_equal(live, np.isfinite(out["mixed"]))       # the population dies at the same step
    assert live[: int(0.9 * steps)].all()
    d = np.abs(out["fp64"] - out["mixed"])[live]
    print(f"{name}: W={W} steps={steps}: E_mix defined at {live.sum()} steps; max |dE_mix| {d.max():.3e} Ha "
          f"(step {int(np.argmax(np.where(live, np.abs(out['fp64'] - out['mixed']), -1)))}), "
          f"E_mix fp64 first/last defined {out['fp64'][0].real:.6f} / {out['fp64'][live][-1].real:.6f}")
    assert d.max() < MHA, d
