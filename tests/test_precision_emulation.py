"""Accuracy of the energy contraction's split products, emulated exactly in float64 (no GPU).

The tensor-core energy kernel forms T_n = Ltilde_n Theta from row-scaled fp16 slices: with
y = x / scale (scale = 2^(e-11), ||row||_2 < 2^e), hi = rint(y), lo = fp16(y - hi) and the rounded
plane r = fp16(y), the head of the Cholesky spectrum takes the three products hi*hi + r*lo' + lo*hi'
(primes: Theta's slices) and the tail -- the smallest vectors whose squared norms add up to at
most 2^-15 of the total -- the one product r*r'.  Here the same arithmetic runs in float64 on a
molecule-like system (exact sums; the kernel's fp32 accumulation is checked against this
emulation by the GPU tests), and the two-body energy 1/2 sum_n [(sum_s t_n)^2 - sum_s X_n] of a
walker near the trial is compared with its exact value: the tail adds a small share of the
three-product error, inside the 2^-11 x 2^-15 x |E2| bound the selection rule is built on, while
one product on every vector would be orders of magnitude worse (negative control)."""
import numpy as np
import pytest

from paper_2003_01831_gb300 import synthetic as syn


def split(x):
    nrm = np.sqrt(np.sum(x * x, axis=-1, keepdims=True))
    e = np.frexp(np.where(nrm > 0, nrm, 1.0))[1]
    sc = np.where(nrm > 0, np.ldexp(1.0, e - 11), 1.0)
    y = x / sc
    hi = np.rint(y)
    lo = (y - hi).astype(np.float16).astype(np.float64)
    r = y.astype(np.float16).astype(np.float64)
    return sc, hi, lo, r


def tail_vectors(sq, eta):
    order = np.argsort(sq, kind="stable")
    tail = np.zeros(sq.size, bool)
    acc = 0.0
    for n in order:
        if acc + sq[n] > eta * sq.sum():
            break
        acc += sq[n]
        tail[n] = True
    return tail


@pytest.mark.parametrize("amp", [0.02, 0.05])
def test_single_product_tail_adds_a_small_share_of_the_error(amp):
    M, N, nch = 128, 32, 640
    h, L, _ = syn.make_hamiltonian(M, nch, np.random.default_rng(77), decay=100.0, band=16)
    P = syn.make_trial(h, N, N)[0].real
    Lt = np.matmul(P.T[None], L)                     # [n][a][k]
    sA, hA, lA, rA = split(Lt)
    tail = tail_vectors(np.sum(Lt ** 2, axis=(1, 2)), 2.0 ** -15)
    assert 0.1 * nch < tail.sum() < 0.5 * nch
    rng = np.random.default_rng(5)
    Phi = P + amp * (rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N)))
    Theta = Phi @ np.linalg.inv(P.T @ Phi)
    E2 = {}
    for form in ("exact", "three", "one"):
        T = np.zeros((nch, N, N), complex)
        for part, unit in ((Theta.real.T, 1.0), (Theta.imag.T, 1j)):
            sB, hB, lB, rB = split(part)
            if form == "exact":
                C = np.matmul(Lt, part.T[None])
            elif form == "three":
                C = (np.matmul(hA, hB.T[None]) + np.matmul(rA, lB.T[None]) + np.matmul(lA, hB.T[None])) \
                    * sA * sB.T[None]
            else:
                C = np.matmul(rA, rB.T[None]) * sA * sB.T[None]
            T += unit * C
        t = np.einsum("naa->n", T)
        X = np.einsum("nab,nba->n", T, T)
        E2[form] = 0.5 * ((2 * t) ** 2 - 2 * X)       # both spins at the same Theta
    exact = E2["exact"].sum()
    err_three = abs(E2["three"].sum() - exact)
    default = np.where(tail, E2["one"], E2["three"]).sum()
    added = abs(default - exact) - err_three
    err_one_everywhere = abs(E2["one"].sum() - exact)
    tail_share = abs(E2["exact"][tail].sum()) / abs(exact)
    print(f"amp {amp}: E2 {exact.real:.4f} Ha, three products {err_three:.2e}, default {abs(default - exact):.2e}, "
          f"tail share {tail_share:.1e}, one product everywhere {err_one_everywhere:.2e}")
    assert tail_share < 2.0 ** -15 * 4
    assert added < 0.2 * err_three + 1e-12
    assert abs(default - exact) < err_three + 2.0 ** -11 * 2.0 ** -15 * abs(exact)
    assert err_one_everywhere > 50 * err_three
