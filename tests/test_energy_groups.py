"""Host-side choice of the adaptive energy products (afqmc_opts.energy_terms = 1): which groups
of Cholesky vectors form the lo*lo split product.  Checked against the rule written out in
numpy (drop the smallest vectors, by norm, while their norms add up to at most eta of the
total; a group keeps four products if any of its vectors does).  No device work."""
import ctypes

import numpy as np
import pytest

from paper_2003_01831_gb300 import api, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    L = api.lib()
    L.afqmc_debug_select_energy_groups.restype = ctypes.c_int
    L.afqmc_debug_select_energy_groups.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_void_p]
    L.afqmc_debug_select_single_groups.restype = ctypes.c_int
    L.afqmc_debug_select_single_groups.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                   ctypes.c_void_p]
    return L


def select(lib, nrm, G, eta):
    nrm = np.ascontiguousarray(nrm, dtype=np.float64)
    ng = (nrm.size + G - 1) // G if G > 0 else nrm.size
    flags = np.full(ng, 7, dtype=np.uint8)
    rc = lib.afqmc_debug_select_energy_groups(nrm.ctypes.data, nrm.size, G, eta, flags.ctypes.data)
    return rc, flags


def rule(nrm, G, eta):
    order = np.argsort(nrm, kind="stable")
    three = np.zeros(nrm.size, bool)
    acc, budget = 0.0, eta * nrm.sum()
    for n in order:
        if acc + nrm[n] > budget:
            break
        acc += nrm[n]
        three[n] = True
    ng = (nrm.size + G - 1) // G
    return np.array([0 if three[g * G:(g + 1) * G].all() else 1 for g in range(ng)], dtype=np.uint8)


def test_exponential_decay_splits_at_the_budget(lib):
    """Norms exp(-n/200) (the m512 workload's decay): the tail beyond n0 with exp(-n0/200) ~ eta
    skips lo*lo."""
    n = np.arange(2560)
    nrm = np.exp(-n / 200.0)
    rc, f = select(lib, nrm, 1, 0.01)
    assert rc == 0
    assert np.array_equal(f, rule(nrm, 1, 0.01))
    n0 = int(np.argmin(f))                           # first vector without lo*lo
    assert f[:n0].all() and not f[n0:].any()
    tail = nrm[n0:].sum() / nrm.sum()
    assert tail <= 0.01 < nrm[n0 - 1:].sum() / nrm.sum()
    assert abs(n0 - 200 * np.log(100)) < 3           # exp(-n0/200) = 1%: n0 ~ 921


@pytest.mark.parametrize("G", [1, 2, 4])
@pytest.mark.parametrize("eta", [0.0, 0.01, 0.3, 0.999])
def test_unsorted_norms_and_groups(lib, G, eta):
    rng = np.random.default_rng(G * 100 + int(eta * 1000))
    nrm = rng.exponential(1.0, 301) ** 3
    nrm[[5, 77, 200]] = 0.0                          # zero vectors: always droppable
    nrm[10:14] = nrm[9]                              # ties
    rc, f = select(lib, nrm, G, eta)
    assert rc == 0
    assert np.array_equal(f, rule(nrm, G, eta))


def test_eta_zero_keeps_every_nonzero_vector(lib):
    nrm = np.array([0.0, 1.0, 2.0, 0.0, 3.0, 0.0, 0.0, 0.0])
    rc, f = select(lib, nrm, 2, 0.0)
    assert rc == 0
    assert f.tolist() == [1, 1, 1, 0]


def test_bad_arguments_rejected(lib):
    nrm = np.ones(4)
    assert select(lib, nrm, 0, 0.01)[0] == -1
    assert select(lib, nrm, 1, 1.0)[0] == -1
    assert select(lib, np.array([1.0, np.nan]), 1, 0.01)[0] == -1
    assert select(lib, np.array([1.0, -1.0]), 1, 0.01)[0] == -1


# ---- single-product tail of the default energy products (energy_terms = 0)

def select_single(lib, sq, G, eta):
    sq = np.ascontiguousarray(sq, dtype=np.float64)
    ng = (sq.size + G - 1) // G if G > 0 else sq.size
    flags = np.full(ng, 7, dtype=np.uint8)
    rc = lib.afqmc_debug_select_single_groups(sq.ctypes.data, sq.size, G, eta, flags.ctypes.data)
    return rc, flags


def single_rule(sq, G, eta):
    """The tail written out: the smallest vectors by squared norm (lower index first on ties)
    while their squared norms add up to at most eta of the total; a group is single when all
    of its vectors are in the tail."""
    order = np.argsort(sq, kind="stable")
    tail = np.zeros(sq.size, bool)
    acc, budget = 0.0, eta * sq.sum()
    for n in order:
        if acc + sq[n] > budget:
            break
        acc += sq[n]
        tail[n] = True
    ng = (sq.size + G - 1) // G
    return np.array([1 if tail[g * G:(g + 1) * G].all() else 0 for g in range(ng)], dtype=np.uint8)


def test_single_tail_of_the_throughput_system(lib):
    """Squared norms exp(-n/100) (the m512 decay exp(-n/200) squared), eta = 2^-15: the tail
    starts where exp(-n0/100) ~ 2^-15, at n0 ~ 1040 of 2560 vectors, and holds at most that share
    of the total."""
    n = np.arange(2560)
    sq = np.exp(-n / 100.0)
    eta = 2.0 ** -15
    rc, f = select_single(lib, sq, 1, eta)
    assert rc == 0
    assert np.array_equal(f, single_rule(sq, 1, eta))
    n0 = int(np.argmax(f))                           # first single vector
    assert not f[:n0].any() and f[n0:].all()
    assert sq[n0:].sum() <= eta * sq.sum() < sq[n0 - 1:].sum()
    assert abs(n0 - 100 * np.log(2.0 ** 15)) < 3


@pytest.mark.parametrize("G", [1, 2, 4, 16])
@pytest.mark.parametrize("eta", [0.0, 2.0 ** -15, 0.01, 0.5])
def test_single_groups_match_rule(lib, G, eta):
    """Random squared norms with ties and zeros, ragged last group."""
    rng = np.random.default_rng(int(G * 1000 + eta * 1e4))
    sq = np.round(rng.exponential(1.0, size=203), 2) ** 2
    sq[rng.integers(0, 203, size=9)] = 0.0
    rc, f = select_single(lib, sq, G, eta)
    assert rc == 0
    assert np.array_equal(f, single_rule(sq, G, eta))


def test_single_groups_reject_bad_arguments(lib):
    sq = np.ones(8)
    assert select_single(lib, sq, 0, 0.01)[0] == -1
    assert select_single(lib, sq, 2, 1.0)[0] == -1
    sq[3] = -1.0
    assert select_single(lib, sq, 2, 0.01)[0] == -1
