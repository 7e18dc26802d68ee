"""Isolated parity of the tcgen05 split-operand kernels (diagnostic C ABI, include/afqmc_debug.h).

Two operand splits are covered.  The plain GEMM mode splits each operand into a bf16 pair
(hi = bf16(x), lo = bf16(x - hi), both round-to-nearest-even) and forms hi*hi + hi*lo + lo*hi.
The exact mode used by the walker step splits each row into row-scaled fp16 slices (hi an
integer with row 2-norm <= 2^11, lo = fp16 of the remainder), sums hi*hi exactly in one
accumulator and the remainder products in a second.  The reference emulates each split
exactly and forms the same products in float64, so the only difference left is the fp32
accumulation inside the tensor cores (bound ~ K * 2^-24 of the accumulated magnitude)."""
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


def split_rows(x, rounded=False):
    """Row-scaled split: scale = 2^(e-11) with ||x_row||_2 < 2^e, hi = rint(x/scale) (an
    integer, |hi| <= 2048), lo = fp16(x/scale - hi).  Returns (hi*scale, lo*scale), and with
    rounded=True also r*scale for the rounded plane r = fp16(x/scale)."""
    nrm = np.sqrt(np.sum(x * x, axis=-1, keepdims=True))
    e = np.frexp(np.where(nrm > 0, nrm, 1.0))[1]
    sc = np.where(nrm > 0, np.ldexp(1.0, e - 11), 1.0)
    y = x / sc
    hi = np.rint(y)
    lo = (y - hi).astype(np.float16).astype(np.float64)
    if rounded:
        return hi * sc, lo * sc, y.astype(np.float16).astype(np.float64) * sc
    return hi * sc, lo * sc


def emul(A, B, exact=False, lolo=None, rounded=False):
    """What the tensor cores form: hi*hi + hi*lo + lo*hi (plain) or + lo*lo (exact mode;
    lolo=False drops that fourth product); rounded=True (exact mode): hi*hi + r*lo + lo*hi
    with the rounded plane r of A."""
    mm = lambda a, b: np.matmul(a, np.swapaxes(b, -1, -2))
    if rounded:
        Ah, Al, Ar = split_rows(A, rounded=True)
        Bh, Bl = split_rows(B)
        return mm(Ah, Bh) + mm(Ar, Bl) + mm(Al, Bh)
    sp = split_rows if exact else split
    Ah, Al = sp(A)
    Bh, Bl = sp(B)
    C = mm(Ah, Bh) + mm(Ah, Bl) + mm(Al, Bh)
    if lolo is None:
        lolo = exact
    return C + mm(Al, Bl) if lolo else C


@pytest.fixture(scope="module")
def dbg():
    from paper_2003_01831_gb300 import build
    build.build()
    L = api.lib()
    d = ctypes.c_double
    vp = ctypes.c_void_p
    L.afqmc_debug_split_gemm.restype = ctypes.c_int
    L.afqmc_debug_split_gemm.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, vp]
    L.afqmc_debug_energy.restype = ctypes.c_int
    L.afqmc_debug_energy.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     vp, vp]
    L.afqmc_debug_set_energy_variant.restype = ctypes.c_int
    L.afqmc_debug_set_energy_variant.argtypes = [ctypes.c_int]
    return L


def energy_call(dbg, Lt, Th, Np, Nchol, nws, M, terms, pair):
    t = np.zeros((nws, Nchol), dtype=np.complex128)
    X = np.zeros((nws, Nchol), dtype=np.complex128)
    assert dbg.afqmc_debug_set_energy_variant(pair) == 0
    try:
        rc = dbg.afqmc_debug_energy(Lt.ctypes.data, Th.ctypes.data, Np, Nchol, nws, M, terms, t.ctypes.data,
                                    X.ctypes.data)
    finally:
        dbg.afqmc_debug_set_energy_variant(1)   # the library default: CTA pairs
    assert rc == 0, api.afqmc_last_error()
    return t, X


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
    rc = dbg.afqmc_debug_split_gemm(A.ctypes.data, B.ctypes.data, nb, rows, cols, K, BN, 0, C.ctypes.data)
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


@pytest.mark.parametrize("nb,rows,cols,K", [(1, 256, 384, 512), (3, 130, 100, 136), (2, 64, 128, 1024)])
def test_exact_mode_is_unbiased(dbg, nb, rows, cols, K):
    """Row-scaled operands: the hi*hi sum is exact, so the only accumulation error left is
    the rounding of the 2^-8 smaller cross terms -- no systematic bias toward zero."""
    rng = np.random.default_rng(rows * 3 + K)
    A = rng.standard_normal((nb, rows, K)) * np.exp(rng.uniform(-3, 3, (nb, rows, 1)))
    B = rng.standard_normal((nb, cols, K)) * np.exp(rng.uniform(-3, 3, (nb, cols, 1)))
    C = np.zeros((nb, rows, cols))
    rc = dbg.afqmc_debug_split_gemm(A.ctypes.data, B.ctypes.data, nb, rows, cols, K, 128, 1, C.ctypes.data)
    assert rc == 0, api.afqmc_last_error()
    ref = emul(A, B, exact=True)
    scale = np.linalg.norm(A, axis=-1)[:, :, None] * np.linalg.norm(B, axis=-1)[:, None, :]
    err = (C - ref) / scale
    exact = np.matmul(A, np.swapaxes(B, -1, -2))
    print(f"exact gemm K={K}: max err/(|a||b|) {np.max(np.abs(err)):.2e}, mean signed "
          f"{np.mean((C - ref) * np.sign(ref) / scale):.2e}, vs float64 {np.max(np.abs(C - exact) / scale):.2e}")
    assert np.max(np.abs(err)) < 5e-8
    assert abs(np.mean((C - ref) * np.sign(ref) / scale)) < 1e-10
    assert np.max(np.abs(C - exact) / scale) < 1e-6


def test_exact_mode_integer_products_are_exact(dbg):
    """Integer rows with 2-norm in [1024, 2048): scale 1, lo = 0, results must be exact."""
    rng = np.random.default_rng(3)
    K = 1024
    A = rng.integers(-60, 61, (1, 128, K)).astype(np.float64)
    B = rng.integers(-60, 61, (1, 128, K)).astype(np.float64)
    for Z in (A, B):
        n = np.sqrt((Z * Z).sum(-1))
        assert np.all((n >= 1024) & (n < 2048))
    C = np.zeros((1, 128, 128))
    rc = dbg.afqmc_debug_split_gemm(A.ctypes.data, B.ctypes.data, 1, 128, 128, K, 128, 1, C.ctypes.data)
    assert rc == 0, api.afqmc_last_error()
    assert np.array_equal(C, np.matmul(A, np.swapaxes(B, -1, -2)))


@pytest.mark.parametrize("pair", [0, 1])
@pytest.mark.parametrize("terms", [3, 4, 5])
@pytest.mark.parametrize("Np,Nchol,nws,M", [(128, 3, 2, 128), (64, 5, 3, 192), (32, 9, 5, 128), (128, 2, 3, 512),
                                            (128, 41, 9, 256),
                                            (8, 37, 21, 64), (24, 11, 7, 128), (40, 7, 4, 192), (56, 5, 3, 128),
                                            (120, 3, 2, 256), (16, 600, 33, 64)])
def test_energy_traces_match_reference(dbg, Np, Nchol, nws, M, terms, pair):
    """Both kernel forms (one CTA per tile; CTA pairs with M = 256 MMAs) and all three product
    sets against their exact float64 emulation.  The shapes include an odd number of Cholesky
    groups (the last pair's second CTA has no rows), ragged walker-spin groups, and more pair
    tiles than the GPU holds at once (persistent loop, barrier phases wrapping).  Np = 32, 64
    and 128 run the fixed-Np epilogues; the other multiples of 8 the generic one, whose tiles
    hold floor(128 / Np) Cholesky vectors by floor(128 / Np) walker-spins with padding rows and
    columns (Np = 40: 120 of 128)."""
    rng = np.random.default_rng(Np * 7 + Nchol)
    Lt = rng.standard_normal((Nchol, Np, M)) * 0.1
    Th = rng.standard_normal((nws, 2, Np, M)) * 0.1
    t, X = energy_call(dbg, Lt, Th, Np, Nchol, nws, M, terms, pair)
    lolo, rnd = terms == 4, terms == 5
    Tr = np.stack([emul(Lt, np.broadcast_to(Th[w, 0], (Nchol, Np, M)), exact=True, lolo=lolo, rounded=rnd)
                   for w in range(nws)])
    Ti = np.stack([emul(Lt, np.broadcast_to(Th[w, 1], (Nchol, Np, M)), exact=True, lolo=lolo, rounded=rnd)
                   for w in range(nws)])
    T = Tr + 1j * Ti                                     # [nws, Nchol, Np, Np]: T[a][b] = Lt[a] . Th^T[b]
    t_ref = np.trace(T, axis1=2, axis2=3)
    X_ref = np.einsum("wnab,wnba->wn", T, T)
    print(f"energy Np={Np} terms={terms} pair={pair}: t err {np.max(np.abs(t - t_ref)) / np.max(np.abs(t_ref)):.2e}, "
          f"X err {np.max(np.abs(X - X_ref)) / np.max(np.abs(X_ref)):.2e}")
    assert np.max(np.abs(t - t_ref)) < 2e-6 * np.max(np.abs(t_ref)) + 1e-9
    assert np.max(np.abs(X - X_ref)) < 2e-6 * np.max(np.abs(X_ref)) + 1e-9


@pytest.mark.parametrize("terms", [6, 7])
@pytest.mark.parametrize("Np,Nchol,nws,M", [(128, 9, 3, 512), (128, 41, 9, 256), (64, 13, 5, 192), (32, 37, 4, 128),
                                            (40, 23, 5, 192), (8, 37, 21, 64)])
def test_single_product_tiles_match_emulation(dbg, Np, Nchol, nws, M, terms):
    """Single-product tiles of the CTA-pair kernel (r*r': both operands rounded to fp16 after row
    scaling, one MMA per K slice into the first accumulator, two K chunks per operand stage), on
    every tile (terms 7) and alternating pair by pair with rounded-three tiles in one persistent
    launch (terms 6: stages of both kinds pass through one ring, and the epilogue leaves out the
    second accumulator only on the single tiles), against their float64 emulation.  The kernel
    must match the single-product emulation far better than the rounded-three one on those
    tiles, and the rounded-three emulation on the others."""
    rng = np.random.default_rng(Np * 11 + Nchol + terms)
    Lt = rng.standard_normal((Nchol, Np, M)) * 0.1
    Th = rng.standard_normal((nws, 2, Np, M)) * 0.1
    t, X = energy_call(dbg, Lt, Th, Np, Nchol, nws, M, terms, 1)
    G = 128 // Np
    single = np.array([terms == 7 or ((n // G) // 2) % 2 == 1 for n in range(Nchol)])
    mm = lambda a, b: np.matmul(a, np.swapaxes(b, -1, -2))
    Ar = split_rows(Lt, rounded=True)[2]
    T1, T3 = [], []
    for w in range(nws):
        parts1, parts3 = [], []
        for c in range(2):
            B = np.broadcast_to(Th[w, c], (Nchol, Np, M))
            parts1.append(mm(Ar, split_rows(Th[w, c], rounded=True)[2][None]))
            parts3.append(emul(Lt, B, exact=True, rounded=True))
        T1.append(parts1[0] + 1j * parts1[1])
        T3.append(parts3[0] + 1j * parts3[1])
    T1, T3 = np.stack(T1), np.stack(T3)                 # [nws, Nchol, Np, Np]

    def traces(T):
        return np.trace(T, axis1=2, axis2=3), np.einsum("wnab,wnba->wn", T, T)

    t1, X1 = traces(T1)
    t3, X3 = traces(T3)
    sel = single[None, :]
    t_ref, X_ref = np.where(sel, t1, t3), np.where(sel, X1, X3)
    st, sx = np.max(np.abs(t_ref)), np.max(np.abs(X_ref))
    e1 = max(np.max(np.abs((t - t1)[:, single])) / st, np.max(np.abs((X - X1)[:, single])) / sx)
    gap = max(np.max(np.abs((t1 - t3)[:, single])) / st, np.max(np.abs((X1 - X3)[:, single])) / sx)
    print(f"single tiles Np={Np} terms={terms}: err vs r*r' {e1:.2e}, r*r' vs rounded three {gap:.2e}")
    assert e1 < 5e-5 and e1 < 0.2 * gap
    if not single.all():
        e3 = max(np.max(np.abs((t - t3)[:, ~single])) / st, np.max(np.abs((X - X3)[:, ~single])) / sx)
        print(f"   rounded-three tiles: err {e3:.2e}")
        assert e3 < 2e-6


@pytest.mark.parametrize("M,N,nch,W", [(128, 32, 96, 3), (256, 128, 64, 2)])
def test_mixed_intermediates_match_numpy(dbg, M, N, nch, W):
    """Theta^T, the traces and the one-body energy of a BF16X3 walker set against numpy."""
    from paper_2003_01831_gb300 import synthetic as syn
    from paper_2003_01831_gb300.walkers import AFQMC
    rng = np.random.default_rng(17)
    h, L, E0 = syn.make_hamiltonian(M, nch, rng)
    Psi = syn.make_trial(h, N, N)
    Phi0 = []
    for s in range(2):
        z = Psi[s][None] + 0.1 * (rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N)))
        Phi0.append(np.linalg.qr(z)[0])
    dbg.afqmc_debug_mixed_terms.restype = ctypes.c_int
    dbg.afqmc_debug_mixed_terms.argtypes = [ctypes.c_void_p] * 7
    with AFQMC(h, L, E0, Psi[0], Psi[1], W, 0.01, Phi0=Phi0, precision=api.PREC_BF16X3) as g:
        ST = np.zeros((W, 2, 2, N, N))
        Si = np.zeros((W, 2, N, N), complex)
        ThT = np.zeros((W, 2, 2, N, M))
        t = np.zeros((W, 2, nch), complex)
        X = np.zeros((W, 2, nch), complex)
        E1 = np.zeros(W, complex)
        rc = dbg.afqmc_debug_mixed_terms(g.wk, ST.ctypes.data, Si.ctypes.data, ThT.ctypes.data, t.ctypes.data,
                                         X.ctypes.data, E1.ctypes.data)
        assert rc == 0, api.afqmc_last_error()
    P = Psi[0].real
    for w in range(W):
        e1 = 0
        for s in range(2):
            S = P.T @ Phi0[s][w]
            Sg = (ST[w, s, 0] + 1j * ST[w, s, 1]).T
            print(f"M={M} N={N} w={w} s={s}: S err {np.max(np.abs(Sg - S)) / np.max(np.abs(S)):.2e}, "
                  f"Sinv err {np.max(np.abs(Si[w, s] - np.linalg.inv(S))) / np.max(np.abs(np.linalg.inv(S))):.2e}, "
                  f"cond {np.linalg.cond(S):.1f}")
            if w == 0 and s == 0:
                A = np.ascontiguousarray(np.concatenate([Phi0[s][w].real.T, Phi0[s][w].imag.T])[None])
                B = np.ascontiguousarray(P.T[None])
                for ex in (0, 1):
                    C = np.zeros((1, 2 * N, N))
                    assert dbg.afqmc_debug_split_gemm(A.ctypes.data, B.ctypes.data, 1, 2 * N, N, M, 128, ex,
                                                      C.ctypes.data) == 0
                    Sd = (C[0, :N] + 1j * C[0, N:]).T
                    print(f"   standalone exact={ex}: S err {np.max(np.abs(Sd - S)) / np.max(np.abs(S)):.2e}, "
                          f"vs pipeline {np.max(np.abs(Sd - Sg)) / np.max(np.abs(S)):.2e}")
            Th = Phi0[s][w] @ np.linalg.inv(S)                                  # [M, N]
            got = ThT[w, s, 0] + 1j * ThT[w, s, 1]                               # [N, M]
            err = np.max(np.abs(got - Th.T)) / np.max(np.abs(Th))
            print(f"M={M} N={N} w={w} s={s}: Theta err {err:.2e}")
            assert err < 2e-7 * np.linalg.cond(S) + 1e-6
            Lt = np.einsum("ka,nkl->nal", P, L)
            T = np.matmul(Lt, Th)
            tr = np.trace(T, axis1=1, axis2=2)
            Xr = np.einsum("nab,nba->n", T, T)
            et = np.max(np.abs(t[w, s] - tr)) / np.max(np.abs(tr))
            ex = np.max(np.abs(X[w, s] - Xr)) / np.max(np.abs(Xr))
            print(f"   t err {et:.2e}  X err {ex:.2e}")
            assert et < 5e-7 * np.linalg.cond(S) + 2e-6 and ex < 5e-7 * np.linalg.cond(S) + 2e-6
            e1 += np.sum((P.T @ h) * Th.T)
        assert abs(E1[w] - e1) < 1e-5 * abs(e1)


def test_energy_tile_window_does_not_change_results(dbg):
    """The L2 window only reorders independent tiles: every window gives bit-identical traces."""
    dbg.afqmc_debug_set_energy_window.argtypes = [ctypes.c_int]
    Np, Nchol, nws, M = 128, 5, 7, 128
    rng = np.random.default_rng(99)
    Lt = rng.standard_normal((Nchol, Np, M)) * 0.1
    Th = rng.standard_normal((nws, 2, Np, M)) * 0.1
    outs = []
    try:
        for ws in (0, 1, 2, 3, 64):
            assert dbg.afqmc_debug_set_energy_window(ws) == 0
            t = np.zeros((nws, Nchol), dtype=np.complex128)
            X = np.zeros((nws, Nchol), dtype=np.complex128)
            rc = dbg.afqmc_debug_energy(Lt.ctypes.data, Th.ctypes.data, Np, Nchol, nws, M, 4, t.ctypes.data,
                                        X.ctypes.data)
            assert rc == 0, api.afqmc_last_error()
            outs.append((t, X))
    finally:
        dbg.afqmc_debug_set_energy_window(0)
    for t, X in outs[1:]:
        assert np.array_equal(t, outs[0][0]) and np.array_equal(X, outs[0][1])


@pytest.mark.parametrize("terms", [4, 5])
def test_energy_pair_kernel_matches_one_cta_kernel(dbg, terms):
    """The CTA-pair form issues the same split products in the same K order into the same
    accumulators: its traces agree with the one-CTA kernel's to the last bits."""
    Np, Nchol, nws, M = 128, 37, 11, 512
    rng = np.random.default_rng(123)
    Lt = rng.standard_normal((Nchol, Np, M)) * np.exp(-np.arange(Nchol) / 20.0)[:, None, None]
    Th = rng.standard_normal((nws, 2, Np, M)) * 0.05
    t1, X1 = energy_call(dbg, Lt, Th, Np, Nchol, nws, M, terms, 0)
    t2, X2 = energy_call(dbg, Lt, Th, Np, Nchol, nws, M, terms, 1)
    dt = np.max(np.abs(t1 - t2)) / np.max(np.abs(t1))
    dX = np.max(np.abs(X1 - X2)) / np.max(np.abs(X1))
    print(f"pair vs one-CTA (terms={terms}): t {dt:.2e}, X {dX:.2e}, identical {np.array_equal(t1, t2) and np.array_equal(X1, X2)}")
    assert dt < 1e-12 and dX < 1e-12


def test_rounded_products_match_four_product_accuracy(dbg):
    """The rounded three products (r*lo + lo*hi with r = fp16 of the scaled Ltilde) against exact
    float64 traces, beside three and four plain products: the rounded form has the accuracy of
    four products, an order of magnitude better than dropping lo*lo."""
    from paper_2003_01831_gb300 import synthetic as syn
    M, N, nch, nws = 512, 128, 16, 4
    h, L, E0 = syn.make_hamiltonian(M, nch, np.random.default_rng(1005), decay=200.0, band=64)
    P = syn.make_trial(h, N, N)[0].real
    Lt = np.ascontiguousarray(np.einsum("ka,nkl->nal", P, L))
    rng = np.random.default_rng(6)
    Th = np.zeros((nws, 2, N, M))
    for w in range(nws):
        Phi = P + 0.05 * (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N)))
        Theta = Phi @ np.linalg.inv(P.T @ Phi)
        Th[w, 0], Th[w, 1] = Theta.real.T, Theta.imag.T
    T = np.einsum("nak,wbk->wnab", Lt, Th[:, 0]) + 1j * np.einsum("nak,wbk->wnab", Lt, Th[:, 1])
    X_ref = np.einsum("wnab,wnba->wn", T, T)
    err = {}
    for terms in (3, 4, 5):
        t, X = energy_call(dbg, Lt, Th, N, nch, nws, M, terms, 0)
        err[terms] = np.max(np.abs(X - X_ref)) / np.max(np.abs(X_ref))
    print("max |dX| / max |X| for 3, 4, rounded 3:", err)
    assert err[5] < 2.0 * err[4]
    assert err[5] < 0.25 * err[3]
