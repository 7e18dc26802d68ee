"""Tensor-hypercontraction (THC) Hamiltonians, complex128 CPU oracle (test infrastructure only).

Only the test suite may import this module.  It shares no code with the CUDA path.

Sec. V approximates the orbital products at N_mu interpolating points r_mu (Eq. (4)) and
writes the two-electron tensor as a product of rank-2 tensors (Eq. (5)),

    v_ijkl ~ sum_{mu nu} X*_{i mu} X_{k mu} M_{mu nu} X*_{j nu} X_{l nu},   X_{i mu} = phi_i(r_mu),

with M_{mu nu} the Coulomb kernel between the interpolating vectors (Eq. (6)), Hermitian and
positive semidefinite.  Restated from the mathematics:

  * With M = U U^+ (U: N_mu x Nchol), L^n_ik = sum_mu X*_{i mu} U_{mu n} X_{k mu}, i.e.
    L^n = X^* diag(U_{:,n}) X^T, reproduces Eq. (5) through Eq. (3)'s sum_n L^n_ik conj(L^n_lj):
    THC is a Cholesky factorisation with structured vectors, and the phaseless step applies
    unchanged to these L^n.  For real U the L^n are Hermitian (real symmetric for real X).
  * The mixed local energy follows from Wick's theorem without forming any L^n.  With the
    mixed densities G^s_ik = <c+_is c_ks>,
        g_mu = sum_s sum_ik X*_{i mu} G^s_ik X_{k mu},   T^s_{mu nu} = sum_il X*_{i mu} G^s_il X_{l nu},
        E_L = E0 + sum_s Tr(htilde_s Theta_s) + 1/2 sum_{mu nu} M_{mu nu} (g_mu g_nu - sum_s T^s_{mu nu} T^s_{nu mu}),
    and the force bias of the factorised fields is <Lhat_n> = sum_mu U_{mu n} g_mu.
  * The HS potential is sum_n c_n L^n = X^* diag(U c) X^T: O(N_mu M^2) instead of O(Nchol M^2).

Readings: U is the modified (diagonally pivoted) Cholesky factor of M -- the factorisation Sec. V
applies to the two-electron integrals themselves, here applied to the kernel: step r takes the
largest remaining diagonal entry p (lowest index on ties), sets column r of U to
(M[:, p] - U[:, :r] U[p, :r]^T) / sqrt(d_p) and subtracts its square from the remaining diagonal,
and it stops once the largest remaining diagonal is at most 1e-12 of the largest initial one.
So U U^+ = M up to that threshold, Nchol <= N_mu, and U is unique for a given pivot order (no
sign or ordering freedom), which lets independent implementations draw the same fields.

Pins (tests/test_oracle_thc.py): the four-index tensor of Eq. (5) against the one rebuilt from
the L^n; the direct local energy against the Cholesky-form local energy and Fock-space matrix
elements; the force bias, HS potential and h' against their Cholesky forms.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from . import afqmc as O

__all__ = ["thc_factor", "cholesky_from_thc", "four_index_thc", "local_energy_thc", "force_bias_traces_thc",
           "hs_potential_thc"]


def thc_factor(Mmat: np.ndarray, rtol: float = 1e-12) -> np.ndarray:
    """U with M = U U^+ (N_mu x Nchol): diagonally pivoted Cholesky, stopping once the largest
    remaining diagonal entry is at most rtol of the largest initial one."""
    n = Mmat.shape[0]
    d = np.real(np.diag(Mmat)).astype(np.float64).copy()
    stop = rtol * np.max(d)
    cols = []
    for r in range(n):
        p = int(np.argmax(d))                       # first index of the maximum
        if d[p] <= stop:
            break
        Ur = np.array(cols).T if cols else np.zeros((n, 0), dtype=Mmat.dtype)
        col = (Mmat[:, p] - Ur @ np.conj(Ur[p, :])) / np.sqrt(d[p])
        cols.append(col)
        d = d - np.abs(col) ** 2
        d[p] = 0.0
    return np.array(cols).T if cols else np.zeros((n, 0), dtype=Mmat.dtype)


def cholesky_from_thc(X: np.ndarray, Mmat: np.ndarray) -> np.ndarray:
    """L^n = X^* diag(U_{:,n}) X^T for every column n of U: [Nchol, M, M]."""
    U = thc_factor(Mmat)
    L = np.einsum("im,mn,km->nik", np.conj(X), U, X)
    return L.real if np.isrealobj(X) and np.isrealobj(U) else L


def four_index_thc(X: np.ndarray, Mmat: np.ndarray) -> np.ndarray:
    """v_ijkl of Eq. (5), by explicit loops."""
    M, Nmu = X.shape
    v = np.zeros((M, M, M, M), dtype=np.complex128)
    for i in range(M):
        for j in range(M):
            for k in range(M):
                for l in range(M):
                    acc = 0.0
                    for mu in range(Nmu):
                        for nu in range(Nmu):
                            acc += np.conj(X[i, mu]) * X[k, mu] * Mmat[mu, nu] * np.conj(X[j, nu]) * X[l, nu]
                    v[i, j, k, l] = acc
    return v


def _densities(Psi: Sequence[np.ndarray], Phi: Sequence[np.ndarray]):
    """Per spin: Theta [W, M, N] and the mixed densities G[w, i, k] = <c+_i c_k> = (Theta Psi^+)_ki."""
    out = []
    for s in range(2):
        Th = O.half_rotated_green(Psi[s], Phi[s])
        G = np.swapaxes(Th @ Psi[s].conj().T, 1, 2)
        out.append((Th, G))
    return out


def local_energy_thc(h: np.ndarray, X: np.ndarray, Mmat: np.ndarray, E0: float,
                     Psi: Sequence[np.ndarray], Phi: Sequence[np.ndarray]) -> np.ndarray:
    """E_L [W] from the THC contraction, with no Cholesky vectors formed."""
    dens = _densities(Psi, Phi)
    E1 = sum(np.einsum("ak,wka->w", Psi[s].conj().T @ h, dens[s][0]) for s in range(2))
    g = sum(np.einsum("im,wik,km->wm", np.conj(X), G, X) for _, G in dens)           # [W, Nmu]
    coul = np.einsum("wm,mn,wn->w", g, Mmat, g)
    exch = 0.0
    for _, G in dens:
        T = np.einsum("im,wil,ln->wmn", np.conj(X), G, X)                           # [W, Nmu, Nmu]
        exch = exch + np.einsum("mn,wmn,wnm->w", Mmat, T, T)
    return E0 + E1 + 0.5 * (coul - exch)


def force_bias_traces_thc(X: np.ndarray, Mmat: np.ndarray, Psi: Sequence[np.ndarray],
                          Phi: Sequence[np.ndarray]) -> np.ndarray:
    """<Lhat_n> = sum_mu U_{mu n} g_mu for the fields of the factor U of M: [W, Nchol]."""
    U = thc_factor(Mmat)
    g = sum(np.einsum("im,wik,km->wm", np.conj(X), G, X) for _, G in _densities(Psi, Phi))
    return g @ U


def hs_potential_thc(c: np.ndarray, X: np.ndarray, Mmat: np.ndarray) -> np.ndarray:
    """sum_n c[w, n] L^n = X^* diag(U c_w) X^T: [W, M, M]."""
    U = thc_factor(Mmat)
    d = c @ U.T                                                                     # [W, Nmu]
    return np.einsum("im,wm,km->wik", np.conj(X), d, X)
