"""Failure detection without a GPU fault.

The tensor-core kernels wait on mbarriers with a bounded poll (try_wait against a clock64
budget), after which they record FLAG_TIMEOUT, drain and return instead of hanging.  Here a
warp waits the same way on a barrier phase that nothing completes: the wait runs out within
its budget, the host reads TIMEOUT from the status word, and the context stays usable -- a
walker step runs afterwards.  The positive control (one thread arrives) completes at once."""
import ctypes

import numpy as np
import pytest

from paper_2003_01831_gb300 import api, synthetic as syn
from paper_2003_01831_gb300.walkers import AFQMC

pytestmark = pytest.mark.gpu

FLAG_TIMEOUT = 4


def probe(limit_cycles, release):
    lib = api.lib()
    lib.afqmc_debug_wait_probe.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    status = ctypes.c_uint(0)
    ms = ctypes.c_float(0.0)
    assert lib.afqmc_debug_wait_probe(limit_cycles, release, ctypes.byref(status), ctypes.byref(ms)) == 0
    return status.value, ms.value


def test_bounded_wait_runs_out_reports_timeout_and_the_context_survives():
    status, ms = probe(200_000_000, 0)          # ~0.1 s of SM clock
    print(f"unreleased wait: status {status}, {ms:.1f} ms")
    assert status == FLAG_TIMEOUT
    assert 10.0 < ms < 5000.0
    status, ms_ok = probe(200_000_000, 1)
    print(f"released wait: status {status}, {ms_ok:.3f} ms")
    assert status == 0 and ms_ok < ms
    rng = np.random.default_rng(3)
    h, L, E0 = syn.make_hamiltonian(10, 6, rng)
    Psi = syn.make_trial(h, 2, 2)
    with AFQMC(h, L, E0, Psi[0], Psi[1], 3, 0.01) as g:
        assert np.all(np.isfinite(g.step(2, seed=1, measure_every=1)))
