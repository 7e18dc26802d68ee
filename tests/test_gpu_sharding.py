"""walker_offset: walker sets holding consecutive ranges of a population draw the Philox
fields of the whole population, so their trajectories equal those of one walker set."""
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
    E_parts, partial = [], np.zeros(4)
    for r in range(3):
        off, cnt = D.shard(W, r, 3)
        with AFQMC(h, L, E0, Psi[0], Psi[1], cnt, 0.01, precision=prec, k_qr=3, walker_offset=off) as g:
            g.step(steps, seed=seed, measure_every=1)
            E, w, _, _ = g.energy()
            E_parts.append(E)
            partial += D.partial_sums(w, E)
    E_sh = np.concatenate(E_parts)
    assert np.max(np.abs(E_sh - E_all)) <= 1e-12 * np.max(np.abs(E_all))
    Emix = complex(partial[0], partial[1]) / complex(partial[2], partial[3])
    assert abs(Emix - Emix_all) <= 1e-12 * abs(Emix_all)
