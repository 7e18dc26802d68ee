"""Thin ctypes binding of ``include/afqmc.h`` (argument marshalling only).

Every function keeps the C name and argument order.  Array arguments may be
numpy arrays (host memory) or torch tensors (host or CUDA); they must be
C-contiguous with the dtype the header states (float64, or complex128 for
"complex").  ``stream`` defaults to torch's current CUDA stream when torch is
importable with CUDA, else the legacy default stream.

There is no fallback: if the shared library is missing this module raises
at import of the first function call, and the library itself returns an error
on a machine without a GPU.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libafqmc_gb300.so")

AFQMC_OK = 0
ERRORS = {
    -1: "BADARG", -2: "SHAPE", -3: "OOM", -4: "NONFINITE", -5: "SINGULAR",
    -6: "TIMEOUT", -7: "CUDA", -8: "UNSUPPORTED",
}
PREC_FP64, PREC_BF16X3 = 0, 1
WEIGHT_PHASELESS, WEIGHT_FREE, WEIGHT_LOCAL = 0, 1, 2

EXPORTED = [
    "afqmc_default_opts", "afqmc_create_hamiltonian", "afqmc_create_hamiltonian_complex",
    "afqmc_destroy_hamiltonian",
    "afqmc_init_walkers", "afqmc_init_walkers_msd", "afqmc_destroy_walkers", "afqmc_step", "afqmc_energy",
    "afqmc_energy_backward", "afqmc_get_walkers", "afqmc_set_walkers",
    "afqmc_philox_fields", "afqmc_last_step_stats", "afqmc_last_error", "afqmc_log_overlap_noalloc",
    "afqmc_create_batch", "afqmc_destroy_batch", "afqmc_batch_step", "afqmc_batch_energy",
    "afqmc_batch_get_walkers", "afqmc_batch_info", "afqmc_batch_autotune", "afqmc_population_control",
    "afqmc_bp_begin", "afqmc_bp_rdm1", "afqmc_comb_indices", "afqmc_mixed_sums",
    "afqmc_create_hamiltonian_thc", "afqmc_hamiltonian_info",
]
PAD_AUTO, PAD_ALWAYS = 0, 1
SEED_STRIDE = 0x9E3779B97F4A7C15   # system s of a batch draws with key seed + s * SEED_STRIDE


class AfqmcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"AFQMC_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("k_taylor", ctypes.c_int),
        ("k_qr", ctypes.c_int),
        ("weight_mode", ctypes.c_int),
        ("fb_cap", ctypes.c_double),
        ("walker_offset", ctypes.c_int),
        ("energy_terms", ctypes.c_int),
        ("reserved", ctypes.c_int * 6),
    ]


class System(ctypes.Structure):
    _fields_ = [
        ("h", ctypes.c_void_p),
        ("L", ctypes.c_void_p),
        ("E0", ctypes.c_double),
        ("M", ctypes.c_int),
        ("Nchol", ctypes.c_int),
        ("Psi_up", ctypes.c_void_p),
        ("Psi_dn", ctypes.c_void_p),
        ("Nup", ctypes.c_int),
        ("Ndn", ctypes.c_int),
        ("W", ctypes.c_int),
        ("Phi0", ctypes.c_void_p),
    ]


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load the in-tree shared library (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, u64, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
    sig = {
        "afqmc_default_opts": (None, [ctypes.POINTER(Opts)]),
        "afqmc_create_hamiltonian": (i, [vp, vp, d, i, i, vp, ctypes.POINTER(vp)]),
        "afqmc_create_hamiltonian_complex": (i, [vp, vp, d, i, i, vp, ctypes.POINTER(vp)]),
        "afqmc_destroy_hamiltonian": (i, [vp]),
        "afqmc_create_hamiltonian_thc": (i, [vp, vp, vp, d, i, i, vp, ctypes.POINTER(vp)]),
        "afqmc_hamiltonian_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "afqmc_init_walkers": (i, [vp, vp, vp, i, i, i, vp, d, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]),
        "afqmc_init_walkers_msd": (i, [vp, i, vp, vp, vp, i, i, i, vp, d, ctypes.POINTER(Opts), vp,
                                       ctypes.POINTER(vp)]),
        "afqmc_destroy_walkers": (i, [vp]),
        "afqmc_step": (i, [vp, i, vp, u64, i, vp, vp]),
        "afqmc_energy": (i, [vp, vp, vp, vp, vp, vp]),
        "afqmc_mixed_sums": (i, [vp, i, vp, vp]),
        "afqmc_energy_backward": (i, [vp, vp, vp, vp, vp, vp, vp]),
        "afqmc_get_walkers": (i, [vp, vp, vp, ctypes.POINTER(i64), vp]),
        "afqmc_set_walkers": (i, [vp, vp, vp, i64, vp]),
        "afqmc_philox_fields": (i, [u64, i64, i, i, vp, vp]),
        "afqmc_last_step_stats": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(i)]),
        "afqmc_last_error": (ctypes.c_char_p, []),
        "afqmc_log_overlap_noalloc": (i, [vp, vp, i, i, i, i, vp, vp, vp]),
        "afqmc_create_batch": (i, [i, ctypes.POINTER(System), d, ctypes.POINTER(Opts), i, vp, ctypes.POINTER(vp)]),
        "afqmc_destroy_batch": (i, [vp]),
        "afqmc_batch_step": (i, [vp, i, u64, i, vp, vp]),
        "afqmc_batch_energy": (i, [vp, i, vp, vp, vp, vp, vp]),
        "afqmc_batch_get_walkers": (i, [vp, i, vp, vp, ctypes.POINTER(i64), vp]),
        "afqmc_batch_info": (i, [vp, i, vp, ctypes.POINTER(i)]),
        "afqmc_batch_autotune": (i, [vp, i, ctypes.POINTER(d), vp]),
        "afqmc_population_control": (i, [vp, d, vp, vp]),
        "afqmc_bp_begin": (i, [vp, i, vp]),
        "afqmc_comb_indices": (i, [vp, i, d, vp, vp, vp]),
        "afqmc_bp_rdm1": (i, [vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a) -> Optional[int]:
    """Data pointer of a numpy array / torch tensor (None stays None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


def _check(rc: int):
    if rc != AFQMC_OK:
        raise AfqmcError(rc, lib().afqmc_last_error().decode())


def afqmc_default_opts() -> Opts:
    o = Opts()
    lib().afqmc_default_opts(ctypes.byref(o))
    return o


def afqmc_create_hamiltonian(h, L, E0: float, M: int, Nchol: int, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().afqmc_create_hamiltonian(_ptr(h), _ptr(L), float(E0), int(M), int(Nchol),
                                          _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_create_hamiltonian_complex(h, L, E0: float, M: int, Nchol: int, stream=None) -> int:
    """L: complex128 [Nchol, M, M]; the walker sets see its 2 Nchol Hermitian-split vectors."""
    out = ctypes.c_void_p()
    _check(lib().afqmc_create_hamiltonian_complex(_ptr(h), _ptr(L), float(E0), int(M), int(Nchol),
                                                  _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_create_hamiltonian_thc(h, X, Mk, E0: float, M: int, Nmu: int, stream=None) -> int:
    """THC Hamiltonian (Eq. (5)): real orbital values X [M, Nmu] and kernel Mk [Nmu, Nmu]."""
    out = ctypes.c_void_p()
    _check(lib().afqmc_create_hamiltonian_thc(_ptr(h), _ptr(X), _ptr(Mk), float(E0), int(M), int(Nmu),
                                              _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_hamiltonian_info(ham: int):
    """(M, Nchol, Nmu) of a Hamiltonian."""
    m, n, q = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().afqmc_hamiltonian_info(ham, ctypes.byref(m), ctypes.byref(n), ctypes.byref(q)))
    return m.value, n.value, q.value


def afqmc_destroy_hamiltonian(ham: int):
    _check(lib().afqmc_destroy_hamiltonian(ham))


def afqmc_init_walkers(ham: int, Psi_up, Psi_dn, Nup: int, Ndn: int, W: int, Phi0, tau: float,
                       opts: Optional[Opts] = None, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().afqmc_init_walkers(ham, _ptr(Psi_up), _ptr(Psi_dn), int(Nup), int(Ndn), int(W), _ptr(Phi0),
                                    float(tau), ctypes.byref(opts) if opts is not None else None,
                                    _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_init_walkers_msd(ham: int, ND: int, D_up, D_dn, c, Nup: int, Ndn: int, W: int, Phi0, tau: float,
                           opts: Optional[Opts] = None, stream=None) -> int:
    """Walker set on the trial sum_I c_I |D_I>: D_up [ND, M, Nup], D_dn [ND, M, Ndn], c [ND] complex."""
    out = ctypes.c_void_p()
    _check(lib().afqmc_init_walkers_msd(ham, int(ND), _ptr(D_up), _ptr(D_dn), _ptr(c), int(Nup), int(Ndn), int(W),
                                        _ptr(Phi0), float(tau), ctypes.byref(opts) if opts is not None else None,
                                        _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_destroy_walkers(wk: int):
    _check(lib().afqmc_destroy_walkers(wk))


def afqmc_step(wk: int, nsteps: int, x=None, seed: int = 0, measure_every: int = 0, E_mix_trace=None,
               stream=None):
    _check(lib().afqmc_step(wk, int(nsteps), _ptr(x), int(seed), int(measure_every), _ptr(E_mix_trace),
                            _stream(stream)))


def afqmc_energy(wk: int, E_L=None, w=None, logS=None, E_mix=None, stream=None):
    _check(lib().afqmc_energy(wk, _ptr(E_L), _ptr(w), _ptr(logS), _ptr(E_mix), _stream(stream)))


def afqmc_mixed_sums(wk: int, nmeas: int, sums, stream=None):
    """Partial sums (Re, Im of sum w E_L; Re, Im of sum w) of the last call's measurements
    into sums (float64 [nmeas, 4], host or device)."""
    _check(lib().afqmc_mixed_sums(wk, int(nmeas), _ptr(sums), _stream(stream)))


def afqmc_energy_backward(wk: int, dE=None, dlogS=None, dPsi_up=None, dPsi_dn=None, dL=None, stream=None):
    _check(lib().afqmc_energy_backward(wk, _ptr(dE), _ptr(dlogS), _ptr(dPsi_up), _ptr(dPsi_dn), _ptr(dL),
                                       _stream(stream)))


def afqmc_get_walkers(wk: int, Phi=None, w=None, stream=None) -> int:
    step = ctypes.c_int64()
    _check(lib().afqmc_get_walkers(wk, _ptr(Phi), _ptr(w), ctypes.byref(step), _stream(stream)))
    return step.value


def afqmc_set_walkers(wk: int, Phi=None, w=None, step: int = 0, stream=None):
    _check(lib().afqmc_set_walkers(wk, _ptr(Phi), _ptr(w), int(step), _stream(stream)))


def afqmc_population_control(wk: int, xi: float, idx=None, stream=None):
    """Comb population control with the uniform number xi in [0, 1); idx (int32 [W]) receives
    the source walker of every new walker."""
    _check(lib().afqmc_population_control(wk, float(xi), _ptr(idx), _stream(stream)))


def afqmc_comb_indices(w, xi: float, stream=None):
    """The comb's selection on the real weights w: (idx int32 [W], total)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    idx = np.zeros(w.size, dtype=np.int32)
    total = np.zeros(1, dtype=np.float64)
    _check(lib().afqmc_comb_indices(_ptr(w), int(w.size), float(xi), _ptr(idx), _ptr(total), _stream(stream)))
    return idx, float(total[0])


def afqmc_bp_begin(wk: int, nbp: int, stream=None):
    """Open a back-propagation window of nbp steps at the current walkers."""
    _check(lib().afqmc_bp_begin(wk, int(nbp), _stream(stream)))


def afqmc_bp_rdm1(wk: int, rdm_up=None, rdm_dn=None, stream=None):
    """Back-propagated one-body density matrices (complex128 [M, M] per spin) of the window."""
    _check(lib().afqmc_bp_rdm1(wk, _ptr(rdm_up), _ptr(rdm_dn), _stream(stream)))


def afqmc_philox_fields(seed: int, step: int, W: int, Nchol: int, x, stream=None):
    _check(lib().afqmc_philox_fields(int(seed), int(step), int(W), int(Nchol), _ptr(x), _stream(stream)))


def afqmc_last_step_stats(wk: int):
    ms = ctypes.c_double()
    k = ctypes.c_int()
    _check(lib().afqmc_last_step_stats(wk, ctypes.byref(ms), ctypes.byref(k)))
    return ms.value, k.value


def afqmc_last_error() -> str:
    return lib().afqmc_last_error().decode()


def afqmc_log_overlap_noalloc(Psi_up, Psi_dn, Nup: int, Ndn: int, M: int, W: int, Phi, logS, stream=None):
    _check(lib().afqmc_log_overlap_noalloc(_ptr(Psi_up), _ptr(Psi_dn), int(Nup), int(Ndn), int(M), int(W), _ptr(Phi),
                                           _ptr(logS), _stream(stream)))


def afqmc_create_batch(systems, tau: float, opts: Optional[Opts] = None, pad_mode: int = PAD_AUTO,
                       stream=None) -> int:
    """systems: sequence of System structures (their arrays must stay alive for the call)."""
    arr = (System * len(systems))(*systems)
    out = ctypes.c_void_p()
    _check(lib().afqmc_create_batch(len(systems), arr, float(tau), ctypes.byref(opts) if opts is not None else None,
                                    int(pad_mode), _stream(stream), ctypes.byref(out)))
    return out.value


def afqmc_destroy_batch(b: int):
    _check(lib().afqmc_destroy_batch(b))


def afqmc_batch_step(b: int, nsteps: int, seed: int = 0, measure_every: int = 0, E_mix_trace=None, stream=None):
    _check(lib().afqmc_batch_step(b, int(nsteps), int(seed), int(measure_every), _ptr(E_mix_trace), _stream(stream)))


def afqmc_batch_energy(b: int, sys: int, E_L=None, w=None, logS=None, E_mix=None, stream=None):
    _check(lib().afqmc_batch_energy(b, int(sys), _ptr(E_L), _ptr(w), _ptr(logS), _ptr(E_mix), _stream(stream)))


def afqmc_batch_get_walkers(b: int, sys: int, Phi=None, w=None, stream=None) -> int:
    step = ctypes.c_int64()
    _check(lib().afqmc_batch_get_walkers(b, int(sys), _ptr(Phi), _ptr(w), ctypes.byref(step), _stream(stream)))
    return step.value


def afqmc_batch_info(b: int, sys: int):
    shape = np.zeros(8, dtype=np.int32)
    k = ctypes.c_int()
    _check(lib().afqmc_batch_info(b, int(sys), _ptr(shape), ctypes.byref(k)))
    return shape, k.value


def afqmc_batch_autotune(b: int, reps: int = 2, stream=None) -> float:
    ms = ctypes.c_double()
    _check(lib().afqmc_batch_autotune(b, int(reps), ctypes.byref(ms), _stream(stream)))
    return ms.value
