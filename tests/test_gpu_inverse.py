"""Batched FP64 inverse and log-determinant (the LU / inverse / log-det row of the walker
step, Sec. V): the register-resident Gauss-Jordan kernel and the shared-memory one against
the oracle's log-determinant, the defining identity S X = I and each other.  Sizes cover one
CTA (N <= 64), the two-CTA cluster (64 < N <= 128), partial column groups and ragged rows."""
import ctypes

import numpy as np
import pytest

from oracle import afqmc as O
from paper_2003_01831_gb300 import api

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2003_01831_gb300 import build
    build.build()
    L = api.lib()
    vp = ctypes.c_void_p
    L.afqmc_debug_inverse.restype = ctypes.c_int
    L.afqmc_debug_inverse.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    return L


def run(lib, S, variant, with_inverse=True):
    S = np.ascontiguousarray(S, dtype=np.complex128)
    count, N, _ = S.shape
    X = np.zeros_like(S)
    ld = np.zeros(count, dtype=np.complex128)
    ms = ctypes.c_float(0.0)
    rc = lib.afqmc_debug_inverse(S.ctypes.data, N, count, variant, int(with_inverse), X.ctypes.data,
                                 ld.ctypes.data, ctypes.addressof(ms))
    return rc, X, ld, ms.value


def walker_like(rng, count, N):
    """Overlap-like matrices: identity-dominated plus noise, condition numbers ~10-100."""
    return np.eye(N) + 0.35 * (rng.standard_normal((count, N, N)) + 1j * rng.standard_normal((count, N, N))) \
        / np.sqrt(N) * 2.0


def phase_close(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


@pytest.mark.parametrize("N", [33, 40, 63, 64, 65, 96, 100, 127, 128])
@pytest.mark.parametrize("variant", [1, 2, 3])
def test_inverse_and_logdet_match_oracle(lib, N, variant):
    rng = np.random.default_rng(N * 10 + variant)
    S = walker_like(rng, 5, N)
    rc, X, ld, _ = run(lib, S, variant)
    assert rc == 0, api.afqmc_last_error()
    ref = O.log_det(S)
    I = np.eye(N)
    res = np.max(np.abs(S @ X - I))
    kappa = max(np.linalg.cond(s) for s in S)
    print(f"N={N} variant={variant}: |SX-I| {res:.2e}, kappa {kappa:.0f}, "
          f"logdet err {np.max(np.abs(ld.real - ref.real)):.2e}")
    assert res < 1e-13 * N * kappa
    assert np.max(np.abs(X - np.linalg.inv(S))) < 1e-13 * N * kappa * np.max(np.abs(X))
    assert np.max(np.abs(ld.real - ref.real)) < 1e-12 * N
    assert np.max(phase_close(ld.imag, ref.imag)) < 1e-12 * N


@pytest.mark.parametrize("N", [48, 128])
def test_register_and_shared_kernels_agree(lib, N):
    rng = np.random.default_rng(7 + N)
    S = walker_like(rng, 7, N)
    _, X1, l1, _ = run(lib, S, 1)
    _, X2, l2, _ = run(lib, S, 2)
    _, X3, l3, _ = run(lib, S, 3)
    # same pivots (max |re|+|im|, lowest row on ties), different update order: rounding only
    assert np.max(np.abs(X1 - X2)) < 1e-12 * np.max(np.abs(X1))
    assert np.max(np.abs(l1 - l2)) < 1e-12 * N
    # float-pair elimination: ~2^-44 per operation, times the condition number
    kappa = max(np.linalg.cond(s) for s in S)
    print(f"N={N}: float-pair vs FP64 |dX| / |X| {np.max(np.abs(X1 - X3)) / np.max(np.abs(X1)):.2e}, "
          f"|d logdet| {np.max(np.abs(l1 - l3)):.2e}, kappa {kappa:.0f}")
    assert np.max(np.abs(X1 - X3)) < 1e-12 * kappa * np.max(np.abs(X1))
    assert np.max(np.abs(l1 - l3)) < 1e-11 * N


@pytest.mark.parametrize("N", [40, 64, 100, 128])
def test_permutation_matrices(lib, N):
    """Pivots are exactly 1 with ties at 0: inverse = transpose, det = sign of the permutation."""
    rng = np.random.default_rng(N)
    perms = [rng.permutation(N) for _ in range(4)] + [np.arange(N), np.arange(N)[::-1].copy()]
    S = np.stack([np.eye(N)[p] for p in perms]).astype(np.complex128)
    S[1] *= np.exp(0.7j)        # a phase on every entry: det picks up exp(0.7 i N)
    for variant in (1, 2, 3):
        rc, X, ld, _ = run(lib, S, variant)
        assert rc == 0, api.afqmc_last_error()
        assert np.array_equal(X[0], S[0].T)
        assert np.max(np.abs(X - np.linalg.inv(S))) < 1e-15 * N
        ref = O.log_det(S)
        assert np.max(np.abs(ld.real - ref.real)) < 1e-12
        assert np.max(phase_close(ld.imag, ref.imag)) < 1e-12 * N


@pytest.mark.parametrize("N", [64, 128])
def test_singular_and_nonfinite(lib, N):
    rng = np.random.default_rng(3)
    S = walker_like(rng, 3, N)
    S[1][:, 5] = 0.0                # a zero column: singular at some step
    for variant in (1, 2, 3):
        rc, X, ld, _ = run(lib, S, variant)
        assert rc == -5, rc                     # AFQMC_ERR_SINGULAR
        assert ld[1].real == -np.inf
        ref = O.log_det(S[[0, 2]])
        assert np.max(np.abs(ld[[0, 2]].real - ref.real)) < 1e-12 * N
    T = walker_like(rng, 2, N)
    T[0][3, 3] = np.nan
    for variant in (1, 2, 3):
        rc, X, ld, _ = run(lib, T, variant)
        assert rc == -4, rc                     # AFQMC_ERR_NONFINITE
        assert ld[0].real == -np.inf
    U = walker_like(rng, 2, N)
    U[1][:, 0] = np.inf                         # an infinite pivot column in the first step
    for variant in (2, 3):
        rc, X, ld, _ = run(lib, U, variant)
        assert rc == -4, rc
        assert ld[1].real == -np.inf


def test_logdet_only_path(lib):
    rng = np.random.default_rng(11)
    S = walker_like(rng, 4, 128)
    rc, _, ld, _ = run(lib, S, 0, with_inverse=False)
    assert rc == 0, api.afqmc_last_error()
    ref = O.log_det(S)
    assert np.max(np.abs(ld.real - ref.real)) < 1e-12 * 128
    assert np.max(phase_close(ld.imag, ref.imag)) < 1e-12 * 128


def test_inverse_timing_report(lib):
    """Times both kernels on 2048 matrices of N = 128 (one m512 step's inverses at W = 1024)."""
    rng = np.random.default_rng(5)
    S = walker_like(rng, 2048, 128)
    out = {}
    for variant in (1, 2, 3, 1, 2, 3):
        rc, _, _, ms = run(lib, S, variant)
        assert rc == 0
        out[variant] = ms
    flops = 2048 * 128 ** 3 * 8.0
    for v, ms in out.items():
        print(f"inverse N=128 x2048 variant {v}: {ms:.2f} ms, {flops / ms / 1e6:.0f} GFLOP/s FP64")
