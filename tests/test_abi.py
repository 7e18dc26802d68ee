"""Host-side checks of the C-ABI library: it builds, loads, exports every symbol
include/afqmc.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2003_01831_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return api.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(afqmc_\w+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "afqmc_step" in names and "afqmc_energy_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(api.EXPORTED) <= names


def test_default_opts(lib):
    o = api.afqmc_default_opts()
    assert (o.precision, o.k_taylor, o.k_qr, o.weight_mode, o.fb_cap) == (0, 6, 5, 0, 1.0)
    assert o.walker_offset == 0 and o.energy_terms == 0 and list(o.reserved) == [0] * 6


def test_opts_struct_layout_matches_header():
    # int, int, int, int, double, int[8]
    assert ctypes.sizeof(api.Opts) == 4 * 4 + 8 + 8 * 4


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    out = ctypes.c_void_p()
    h = np.zeros((4, 4))
    L = np.zeros((2, 4, 4))
    assert lib.afqmc_create_hamiltonian(h.ctypes.data, L.ctypes.data, 0.0, 4, 2, None, None) == -1
    assert lib.afqmc_create_hamiltonian(None, L.ctypes.data, 0.0, 4, 2, None, ctypes.byref(out)) == -1
    assert lib.afqmc_create_hamiltonian(h.ctypes.data, L.ctypes.data, 0.0, 0, 2, None, ctypes.byref(out)) == -2
    assert lib.afqmc_create_hamiltonian(h.ctypes.data, L.ctypes.data, float("nan"), 4, 2, None,
                                        ctypes.byref(out)) == -4
    assert b"E0" in lib.afqmc_last_error()
    Lc = np.zeros((2, 4, 4), dtype=np.complex128)
    mk = lib.afqmc_create_hamiltonian_complex
    assert mk(h.ctypes.data, Lc.ctypes.data, 0.0, 4, 2, None, None) == -1
    assert mk(h.ctypes.data, None, 0.0, 4, 2, None, ctypes.byref(out)) == -1
    assert mk(h.ctypes.data, Lc.ctypes.data, 0.0, 4, 0, None, ctypes.byref(out)) == -2
    assert mk(h.ctypes.data, Lc.ctypes.data, float("inf"), 4, 2, None, ctypes.byref(out)) == -4
    assert lib.afqmc_step(None, 1, None, 0, 0, None, None) == -1
    assert lib.afqmc_bp_begin(None, 3, None) == -1
    lib.afqmc_debug_wait_probe.argtypes = [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    st = ctypes.c_uint(0)
    assert lib.afqmc_debug_wait_probe(1000, 0, None, None) == -1
    assert lib.afqmc_debug_wait_probe(0, 0, ctypes.byref(st), None) == -1
    assert lib.afqmc_debug_wait_probe(5_000_000_000, 0, ctypes.byref(st), None) == -1
    D = np.zeros((2, 4, 2), dtype=np.complex128)
    cf = np.ones(2, dtype=np.complex128)
    init = lib.afqmc_init_walkers_msd
    assert init(None, 2, D.ctypes.data, D.ctypes.data, cf.ctypes.data, 2, 2, 3, None, 0.01, None, None,
                ctypes.byref(out)) == -1                      # no Hamiltonian
    assert init(None, 2, D.ctypes.data, D.ctypes.data, None, 2, 2, 3, None, 0.01, None, None,
                ctypes.byref(out)) == -1                      # no coefficients
    wv = np.ones(3)
    iv = np.zeros(3, dtype=np.int32)
    assert lib.afqmc_comb_indices(None, 3, 0.5, iv.ctypes.data, None, None) == -1
    assert lib.afqmc_comb_indices(wv.ctypes.data, 0, 0.5, iv.ctypes.data, None, None) == -2
    assert lib.afqmc_comb_indices(wv.ctypes.data, 3, 1.0, iv.ctypes.data, None, None) == -1
    assert lib.afqmc_bp_rdm1(None, None, None, None) == -1
    assert lib.afqmc_energy(None, None, None, None, None, None) == -1
    assert lib.afqmc_destroy_walkers(None) == -1
    assert lib.afqmc_destroy_hamiltonian(None) == -1
    assert lib.afqmc_philox_fields(0, 0, 0, 4, None, None) == -1
    assert lib.afqmc_init_walkers(None, None, None, 1, 1, 1, None, 0.01, None, None, ctypes.byref(out)) == -1


def test_python_binding_raises(lib):
    with pytest.raises(api.AfqmcError) as e:
        api.afqmc_create_hamiltonian(np.zeros((2, 2)), np.zeros((1, 2, 2)), 0.0, 0, 1)
    assert e.value.code == -2


def test_system_struct_layout_matches_header():
    # void* h, void* L, double E0, int M, int Nchol, void* Psi_up, void* Psi_dn, int Nup, int Ndn,
    # int W, (pad), void* Phi0
    assert ctypes.sizeof(api.System) == 8 + 8 + 8 + 4 + 4 + 8 + 8 + 4 + 4 + 4 + 4 + 8
    assert api.System.Phi0.offset == 64


def test_batch_bad_arguments_without_a_gpu(lib):
    out = ctypes.c_void_p()
    h = np.zeros((4, 4))
    L = np.zeros((2, 4, 4))
    P = np.zeros((4, 1), dtype=np.complex128)
    ok = api.System(h=h.ctypes.data, L=L.ctypes.data, E0=0.0, M=4, Nchol=2, Psi_up=P.ctypes.data,
                    Psi_dn=P.ctypes.data, Nup=1, Ndn=1, W=2, Phi0=None)
    arr = (api.System * 1)(ok)
    assert lib.afqmc_create_batch(1, arr, 0.01, None, 0, None, None) == -1          # out NULL
    assert lib.afqmc_create_batch(0, arr, 0.01, None, 0, None, ctypes.byref(out)) == -1
    assert lib.afqmc_create_batch(1, arr, -1.0, None, 0, None, ctypes.byref(out)) == -1
    assert lib.afqmc_create_batch(1, arr, 0.01, None, 7, None, ctypes.byref(out)) == -1   # pad mode
    bad = (api.System * 1)(api.System(h=h.ctypes.data, L=L.ctypes.data, E0=0.0, M=4, Nchol=2,
                                      Psi_up=P.ctypes.data, Psi_dn=P.ctypes.data, Nup=5, Ndn=1, W=2, Phi0=None))
    assert lib.afqmc_create_batch(1, bad, 0.01, None, 0, None, ctypes.byref(out)) == -2
    assert b"system 0" in lib.afqmc_last_error()
    o = api.afqmc_default_opts()
    o.precision = api.PREC_BF16X3
    uneven = (api.System * 1)(api.System(h=h.ctypes.data, L=L.ctypes.data, E0=0.0, M=4, Nchol=2,
                                         Psi_up=P.ctypes.data, Psi_dn=P.ctypes.data, Nup=1, Ndn=2, W=2,
                                         Phi0=None))
    assert lib.afqmc_create_batch(1, uneven, 0.01, ctypes.byref(o), 0, None, ctypes.byref(out)) == -8
    assert lib.afqmc_batch_step(None, 1, 0, 0, None, None) == -1
    assert lib.afqmc_batch_energy(None, 0, None, None, None, None, None) == -1
    assert lib.afqmc_batch_get_walkers(None, 0, None, None, None, None) == -1
    assert lib.afqmc_batch_info(None, 0, None, None) == -1
    assert lib.afqmc_batch_autotune(None, 1, None, None) == -1
    assert lib.afqmc_destroy_batch(None) == -1
