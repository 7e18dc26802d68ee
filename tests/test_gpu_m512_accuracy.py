"""Throughput workload accuracy: BF16X3 vs FP64 GPU paths at M=512, N=128+128, Nchol=2560.

Same walkers, same fields; the mixed-estimator energy of every measured step must agree to
1 mHa (the bar for the tensor-core path), for the default energy products (three, with the
rounded Ltilde plane), for four products everywhere and for the adaptive four/three choice.
Sampled at 16 walkers x 10 steps (two QRs) to keep the FP64 path's run short (its energy
contraction costs ~1.7e11 flops per walker-step)."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

MHA = 1e-3


def test_m512_mixed_matches_fp64_within_1mha():
    wl = syn.WORKLOADS["m512"]
    rng = wl.rng()
    h, L, E0 = syn.make_hamiltonian(wl.M, wl.Nchol, rng, decay=wl.decay, band=wl.band)
    Psi = syn.make_trial(h, wl.Nup, wl.Ndn)
    W, steps = 16, 10
    x = syn.make_fields(steps, W, wl.Nchol, seed=0)
    traces = {}
    for name, prec, terms in (("fp64", api.PREC_FP64, 0), ("bf16x3", api.PREC_BF16X3, 0),
                              ("bf16x3_4", api.PREC_BF16X3, 4), ("bf16x3_3", api.PREC_BF16X3, 3),
                              ("bf16x3_adaptive", api.PREC_BF16X3, 1)):
        with AFQMC(h, L, E0, Psi[0], Psi[1], W, wl.tau, k_qr=wl.k_qr, precision=prec, energy_terms=terms) as g:
            traces[name] = g.step(steps, x, measure_every=1)
            traces[name + "_E"] = g.energy()[0]
    for name in ("bf16x3", "bf16x3_4", "bf16x3_3", "bf16x3_adaptive"):
        d = np.abs(traces["fp64"] - traces[name])
        print(name, "E_mix fp64", traces["fp64"].real, "max |dE_mix| (Ha)", d.max(),
              "max per-walker |dE_L| (Ha)", np.max(np.abs(traces["fp64_E"] - traces[name + "_E"])))
    # the bar applies to the library default (three products with the rounded Ltilde plane), to
    # four products for every vector and to the adaptive choice; three plain products everywhere
    # is reported only (~1.3 mHa here)
    assert np.max(np.abs(traces["fp64"] - traces["bf16x3"])) < MHA
    assert np.max(np.abs(traces["fp64"] - traces["bf16x3_4"])) < MHA
    assert np.max(np.abs(traces["fp64"] - traces["bf16x3_adaptive"])) < MHA
    # the default and the adaptive choice stay within a small fraction of the four-product
    # trajectory's error
    for name in ("bf16x3", "bf16x3_adaptive"):
        d0 = np.max(np.abs(traces[name] - traces["bf16x3_4"]))
        print(name, "vs four products: max |dE_mix| (Ha)", d0)
        assert d0 < 0.25 * MHA
