"""Adjoint of the local energy and log-overlap (test infrastructure only).

Gradients of the mixed local energy E_L and the log-overlap
logS = sum_s log det(Psi_s^dagger Phi_s) with respect to the trial orbitals
Psi_s and the Cholesky tensor L, walkers Phi held fixed.  Derived here from
the energy expression of Sec. V, Eqs. (1), (3) (see ``afqmc.local_energy``):

With Q_s = Psi_s^dagger (both quantities are holomorphic in Q), S = Q Phi,
Theta = Phi S^-1, T_n = Q L_n Theta, c_n = sum_s Tr T_ns:
  d logS / dQ^T        = Theta
  d E_L  / dQ_s^T      = (I - Theta_s Q_s) [h Theta_s + sum_n L_n Theta_s (c_n I - T_ns)]
  d E_L  / dL_n (F_n)  : F_n^T = sum_s (c_n Theta_s Q_s - Theta_s T_ns Q_s)

For a real loss  ell = sum_w Re(conj(dE_w) E_w + conj(dlogS_w) logS_w):
  grad Psi_s = d ell/d Re Psi + i d ell/d Im Psi = sum_w conj(g_w) F_w^T, where
  F^T is the corresponding dQ^T derivative and g the upstream factor;
  grad L (real tensor) = sum_w Re(conj(dE_w) F_n,w)  (full unsymmetrised tensor).

Pinned against central finite differences in tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

from .afqmc import Hamiltonian, half_rotated_green, rotated_cholesky

__all__ = ["energy_logdet_backward"]


def energy_logdet_backward(ham: Hamiltonian, Psi: Sequence[np.ndarray], Phi: Sequence[np.ndarray],
                           dE: np.ndarray, dlogS: np.ndarray):
    """Return (dPsi_up [M, Nup], dPsi_dn [M, Ndn], dL [Nchol, M, M] real)."""
    M = ham.M
    W = Phi[0].shape[0]
    thetas = [half_rotated_green(Psi[s], Phi[s]) for s in range(2)]
    Lts = [rotated_cholesky(Psi[s], ham.L) for s in range(2)]
    dPsi = [np.zeros_like(Psi[s], dtype=np.complex128) for s in range(2)]
    dL = np.zeros(ham.L.shape, dtype=np.float64)
    I = np.eye(M)
    for w in range(W):
        Ts = [np.matmul(Lts[s], thetas[s][w]) for s in range(2)]          # [Nchol, N, N]
        c = sum(np.trace(Ts[s], axis1=1, axis2=2) for s in range(2))      # [Nchol]
        gE = np.conj(dE[w])
        gS = np.conj(dlogS[w])
        for s in range(2):
            Th = thetas[s][w]                                               # [M, N]
            Q = Psi[s].conj().T                                             # [N, M]
            N = Th.shape[1]
            inner = ham.h @ Th
            U = Th[None, :, :] * c[:, None, None] - np.matmul(Th[None], Ts[s])   # Theta (c_n I - T_n)
            inner = inner + np.einsum("nik,nka->ia", ham.L, U, optimize=True)
            FT = (I - Th @ Q) @ inner                                       # dE/dQ^T  [M, N]
            dPsi[s] += gE * FT + gS * Th
            # dE/dL_n: F_n^T = c_n Theta Q - Theta T_n Q
            ThQ = Th @ Q                                                    # [M, M]
            FnT = c[:, None, None] * ThQ[None] - np.matmul(np.matmul(Th[None], Ts[s]), Q[None])
            dL += np.real(gE * np.transpose(FnT, (0, 2, 1)))
    return dPsi[0], dPsi[1], dL
