"""Isolated parity of the tcgen05 split-bf16 kernels (diagnostic C ABI, include/afqmc_debug.h).

The reference emulates the operand split exactly (hi = bf16(x), lo = bf16(x - hi), both
round-to-nearest-even) and forms hi*hi + hi*lo + lo*hi in float64, so the only difference
left is the fp32 accumulation order inside the tensor cores (bound ~ K * 2^-24)."""
import ctypes

import numpy as np
import pytest

from paper_2003_01831_gb300 import api

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round float64 values to the nearest bf16 value (ties to even), returned as float64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    shift = np.uint64(45)                       # keep 7 explicit mantissa bits
    lsb = (b >> shift) & np.uint64(1)
    bias = (np.uint64(1) << np.uint64(44)) - np.uint64(1) + lsb
    r = ((b + bias) >> shift) << shift
    return r.view(np.float64)


def split(x):
    hi = bf16_round(x)
    lo = bf16_round(x - hi)
    return hi, lo


def emul(A, B):
    Ah, Al = split(A)
    Bh, Bl = split(B)
    mm = lambda a, b: np.matmul(a, np.swapaxes(b, -1, -2))
    return mm(Ah, Bh) + mm(Ah, Bl) + mm(Al, Bh)


@pytest.fixture(scope="module")
def dbg():
    from paper_2003_01831_gb300 import build
    build.build()
    L = api.lib()
    d = ctypes.c_double
    vp = ctypes.c_void_p
    L.afqmc_debug_split_gemm.restype = ctypes.c_int
    L.afqmc_debug_split_gemm.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, vp]
    L.afqmc_debug_energy.restype = ctypes.c_int
    L.afqmc_debug_energy.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    return L


@pytest.mark.parametrize("nb,rows,cols,K,BN", [
    (1, 128, 256, 64, 256),
    (1, 256, 512, 512, 256),
    (1, 200, 300, 72, 256),     # ragged rows, columns and K tail
    (3, 130, 100, 136, 128),    # batched, ragged
    (2, 64, 128, 1024, 128),
])
def test_split_gemm_matches_split_emulation(dbg, nb, rows, cols, K, BN):
    rng = np.random.default_rng(rows + cols + K)
    A = rng.standard_normal((nb, rows, K))
    B = rng.standard_normal((nb, cols, K))
    C = np.zeros((nb, rows, cols))
    rc = dbg.afqmc_debug_split_gemm(A.ctypes.data, B.ctypes.data, nb, rows, cols, K, BN, C.ctypes.data)
    assert rc == 0, api.afqmc_last_error()
    ref = emul(A, B)
    exact = np.matmul(A, np.swapaxes(B, -1, -2))
    big = np.max(np.abs(ref))
    d = (C - ref) * np.sign(ref)
    print(f"split gemm K={K}: max |err|/max|C| {np.max(np.abs(C - ref)) / big:.2e}, "
          f"mean signed err/|C| {np.mean(d / np.maximum(np.abs(ref), 1e-30)):.2e}")
    # against the split emulation: only the fp32 accumulation inside the tensor cores differs
    # (a dropped cross product would leave ~2^-9 relative)
    assert np.max(np.abs(C - ref)) < 1e-5 * big, np.max(np.abs(C - ref)) / big
    # against exact float64: split error ~ 2^-16 per operand
    assert np.max(np.abs(C - exact)) < 3e-5 * big


@pytest.mark.parametrize("Np,Nchol,nws,M", [(128, 3, 2, 128), (64, 5, 3, 192), (32, 9, 5, 128), (128, 2, 3, 512)])
def test_energy_traces_match_reference(dbg, Np, Nchol, nws, M):
    rng = np.random.default_rng(Np * 7 + Nchol)
    Lt = rng.standard_normal((Nchol, Np, M)) * 0.1
    Th = rng.standard_normal((nws, 2, Np, M)) * 0.1
    t = np.zeros((nws, Nchol), dtype=np.complex128)
    X = np.zeros((nws, Nchol), dtype=np.complex128)
    rc = dbg.afqmc_debug_energy(Lt.ctypes.data, Th.ctypes.data, Np, Nchol, nws, M, t.ctypes.data, X.ctypes.data)
    assert rc == 0, api.afqmc_last_error()
    Tr = np.stack([emul(Lt, np.broadcast_to(Th[w, 0], (Nchol, Np, M))) for w in range(nws)])
    Ti = np.stack([emul(Lt, np.broadcast_to(Th[w, 1], (Nchol, Np, M))) for w in range(nws)])
    T = Tr + 1j * Ti                                     # [nws, Nchol, Np, Np]: T[a][b] = Lt[a] . Th^T[b]
    t_ref = np.trace(T, axis1=2, axis2=3)
    X_ref = np.einsum("wnab,wnba->wn", T, T)
    assert np.max(np.abs(t - t_ref)) < 1e-5 * np.max(np.abs(t_ref)) + 1e-6
    assert np.max(np.abs(X - X_ref)) < 1e-5 * np.max(np.abs(X_ref)) + 1e-6
