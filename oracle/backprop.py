"""Back-propagated one-body density matrix, complex128 CPU oracle (test infrastructure only).

Only the test suite may import this module.  It shares no code with the CUDA path.

Sec. V names the back-propagation estimator for observables that do not commute with H (the
one-particle reduced density matrix among them) and cites it (Zhang, Carlson & Gubernatis
1997; Purwanto & Zhang 2004; Motta & Zhang 2017) without writing it out.  Restated from
the mathematics:

  A walker that starts at Phi_w(0) and takes n steps carries the product B_w(n) ... B_w(1) of
  the one-body propagators the steps applied.  The mixed expectation of an operator O taken
  n steps before the end, with the trial carried backwards through the same propagators,

      <Psi_T| B_w(n) ... B_w(1) O |Phi_w(0)> / <Psi_T| B_w(n) ... B_w(1) |Phi_w(0)>,

  is a determinant ratio with the back-propagated trial Psi_bp,w = B_w(1)^+ ... B_w(n)^+ Psi_T
  (Thouless: the adjoint of a one-body exponential maps a determinant to a determinant).  For
  O = c+_i c_j of one spin it is [Phi (Psi_bp^+ Phi)^-1 Psi_bp^+]_ji, the same form as the mixed
  one-body density with Psi_bp in place of Psi_T.  The estimate averages it over the walkers
  with the weights they carry at the end of the window.

Readings of what the paper leaves open (each one is also listed in the design notes):
  * B_w(k) = B T_K(i sqrt(tau) A_w(k)) B with A_w(k) = sum_n c_wn(k) L_n and c = x - xbar, the
    shifted fields the forward step used (the same truncated Taylor series of order K).
  * The weights are the end-of-window weights the forward run produced (phaseless factors
    included); walkers of weight 0 do not contribute.
  * Population control inside the window: a new walker carries its source walker's Phi(0)
    and shifted-field history (its ancestry).
  * The back-propagated trial may be re-orthonormalised: the estimate does not change under
    Psi_bp -> Psi_bp R for any invertible R.

Pins (tests/test_oracle_backprop.py): the back-propagated trial against the forward
propagators applied to an arbitrary matrix (adjoint and order), the zero-length window against
Fock-space mixed one-body densities, a one-step window averaged over the fields against the
Fock-space <Psi_T| exp(-tau (H - E0)) c+_i c_j |Phi> to O(tau^2), and invariance under walker
relabelling, re-orthonormalisation and an identity comb.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import afqmc as O

__all__ = ["back_propagated_trial", "rdm1", "Window"]


def back_propagated_trial(L: np.ndarray, Psi: np.ndarray, B: np.ndarray, coefs: Sequence[np.ndarray],
                          tau: float, K: int) -> np.ndarray:
    """Psi_bp,w = B_w(1)^+ ... B_w(n)^+ Psi for every walker: [W, M, N].

    coefs[k] [W, Nchol] are the shifted fields of step k+1 (coefs[0] drove the first step);
    B_w(k)^+ = B^+ T_K(X^+) B^+ with X = i sqrt(tau) A_w(k), the adjoint written out."""
    W = coefs[0].shape[0]
    Q = np.repeat(np.asarray(Psi, dtype=np.complex128)[None], W, axis=0)
    Bd = B.conj().T
    for c in reversed(coefs):
        X = 1j * np.sqrt(tau) * O.hs_potential(c, L)
        Xd = np.conj(np.swapaxes(X, 1, 2))
        Q = np.matmul(Bd, O.taylor_exp_apply(Xd, np.matmul(Bd, Q), K))
    return Q


def rdm1(Psi_bp: np.ndarray, Phi0: np.ndarray, w: np.ndarray) -> np.ndarray:
    """G[i, j] = sum_w w_w <Psi_bp,w| c+_i c_j |Phi0_w> / <Psi_bp,w|Phi0_w> / sum_w w_w, one spin.

    Per walker the ratio is [Phi0 (Psi_bp^+ Phi0)^-1 Psi_bp^+]_ji."""
    M = Phi0.shape[1]
    G = np.zeros((M, M), dtype=np.complex128)
    for k in range(Phi0.shape[0]):
        if w[k] == 0:
            continue
        Th = O.half_rotated_green(Psi_bp[k], Phi0[k][None])[0]      # Phi0 (Psi_bp^+ Phi0)^-1
        G += w[k] * (Th @ Psi_bp[k].conj().T).T
    return G / np.sum(w)


class Window:
    """A back-propagation window opened at the walkers `Phi` (per spin [W, M, N])."""

    def __init__(self, Phi: Sequence[np.ndarray]):
        self.Phi0: List[np.ndarray] = [np.array(p, dtype=np.complex128) for p in Phi]
        self.coefs: List[np.ndarray] = []

    def record(self, c: np.ndarray):
        self.coefs.append(np.array(c, dtype=np.complex128))

    def comb(self, idx: np.ndarray):
        """Population control inside the window: new walker j descends from walker idx[j]."""
        self.Phi0 = [p[idx].copy() for p in self.Phi0]
        self.coefs = [c[idx].copy() for c in self.coefs]

    def estimate(self, L: np.ndarray, Psi: Sequence[np.ndarray], B: np.ndarray, w: np.ndarray,
                 tau: float, K: int):
        """(G_up, G_dn) with the end-of-window weights w."""
        out = []
        for s in range(2):
            if self.coefs:
                Q = back_propagated_trial(L, Psi[s], B, self.coefs, tau, K)
            else:
                Q = np.repeat(np.asarray(Psi[s], dtype=np.complex128)[None], w.size, axis=0)
            out.append(rdm1(Q, self.Phi0[s], w))
        return out
