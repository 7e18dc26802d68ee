"""walker_offset: walker sets holding consecutive ranges of a population draw the Philox
fields of the whole population, so their trajectories equal those of one walker set; the
library's device partial sums (afqmc_mixed_sums) combine their mixed estimates into the whole
population's."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300 import distributed as D
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [api.PREC_FP64, api.PREC_BF16X3])
def test_shards_reproduce_whole_population(prec):
    d = syn.UnevenSystem(M=64, N=32, Nchol=64, W=9)
    h, L, E0, Psi = syn.make_uneven_system(d, 0, seed=12)
    W, steps, seed = 9, 6, 77
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, precision=prec, k_qr=3) as g:
        g.step(steps, seed=seed, measure_every=1)
        E_all, w_all, _, Emix_all = g.energy()
    E_parts, partial, trace_sums = [], np.zeros(4), np.zeros((steps, 4))
    for r in range(3):
        off, cnt = D.shard(W, r, 3)
        with AFQMC(h, L, E0, Psi[0], Psi[1], cnt, 0.01, precision=prec, k_qr=3, walker_offset=off) as g:
            g.step(steps, seed=seed, measure_every=1)
            # the step's per-measurement partial sums, formed by the library on the device
            trace_sums += D.device_partial_sums(g, steps).cpu().numpy()
            E, w, _, _ = g.energy()
            E_parts.append(E)
            dev = D.device_partial_sums(g, 1).cpu().numpy()[0]
            ref = D.partial_sums(w, E)
            assert np.max(np.abs(dev - ref)) <= 1e-13 * np.max(np.abs(ref))
            partial += dev
            with pytest.raises(api.AfqmcError):     # nmeas must match the last call
                D.device_partial_sums(g, 2)
    E_sh = np.concatenate(E_parts)
    assert np.max(np.abs(E_sh - E_all)) <= 1e-12 * np.max(np.abs(E_all))
    Emix = D.emix_from_sums(partial)[0]
    assert abs(Emix - Emix_all) <= 1e-12 * abs(Emix_all)
    # the shards' combined step trace equals the whole population's
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, precision=prec, k_qr=3) as g:
        whole = g.step(steps, seed=seed, measure_every=1)
    assert np.max(np.abs(D.emix_from_sums(trace_sums) - whole)) <= 1e-12 * np.max(np.abs(whole))
