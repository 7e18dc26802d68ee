"""Multi-determinant trial wave functions, complex128 CPU oracle (test infrastructure only).

Only the test suite may import this module.  It shares no code with the CUDA path.

Sec. V allows trials |psi_T> = sum_I c_I |D_I> over N_D Slater determinants D_I (one orbital
matrix per spin), orthogonal configuration-interaction expansions or non-orthogonal ones
(NOMSD) with <D_I|D_J> = S_IJ.  It gives no formulas beyond the expansion; restated from the
mathematics:

  <psi_T|Phi> = sum_I conj(c_I) <D_I|Phi>,  <D_I|Phi> = det(D_I,up^+ Phi_up) det(D_I,dn^+ Phi_dn),

  and every mixed estimate of an operator O is the overlap-weighted average of the
  single-determinant ones,

  <psi_T|O|Phi> / <psi_T|Phi> = sum_I u_I <D_I|O|Phi>/<D_I|Phi>,  u_I = conj(c_I) <D_I|Phi> / <psi_T|Phi>,

  so the local energy and the force-bias traces <L_n> are the u-weighted sums of those of the
  single determinants (the oracle's single-determinant functions evaluate each one).

Readings of what the paper leaves open (also listed in the design notes):
  * E_T is the trial's energy shift sum'_IJ conj(c_I) c_J S_IJ E_I(D_J) / sum'_IJ conj(c_I) c_J S_IJ
    (primed sums: pairs with a non-singular overlap S_IJ), with E_I(D_J) the mixed local energy
    of trial D_I at walker D_J; this is where the overlaps S_IJ of a non-orthogonal expansion
    enter.  Without exactly orthogonal pairs -- one determinant (its own local energy), or a
    NOMSD expansion -- it is the variational energy <psi_T|H|psi_T> / <psi_T|psi_T>.  A pair with
    S_IJ = 0 (the determinants of an orthogonal CI expansion) would need the Slater-Condon
    rules for <D_I|H|D_J>, which are not restated, so for such expansions E_T is a shift, not
    the variational energy.  With phaseless (hybrid) weights it is a common factor of all
    weights, so E_mix does not depend on it; with local-energy weights it also centres the
    clip window E_T +- 2/sqrt(tau) of the energy bound.
  * Walkers start, unless given, at the determinant with the largest |c_I| (lowest index on
    ties).
  * Log-overlaps are summed over determinants as a complex log-sum-exp shifted by the
    largest real part, so no overlap under- or overflows.
  * Each determinant's term is evaluated as <D_I|Phi> times its own mixed estimate, which needs
    <D_I|Phi> away from zero: this is the non-orthogonal (NOMSD) evaluation, without fast
    updates.  An orthogonal CI expansion whose walkers sit exactly on the reference makes the
    excited determinants' terms ill-conditioned; their Sherman-Morrison evaluation relative to
    the reference is not restated here.

The variational energy itself, orthogonal pairs included, is variational_energy(): the matrix
elements <D_I|H|D_J> between any two determinants by Loewdin's rules for biorthogonalised
orbitals (below), which need no inverse of the overlap, so exactly orthogonal pairs (determinants
that differ in one, two or more orbitals) are covered.  The walker step uses energy_shift() as
E_T, which is what the GPU path forms; the two agree unless two determinants are exactly
orthogonal.

Pins (tests/test_oracle_msd.py): overlap, local energy, force bias and energy shift (the variational energy of a NOMSD expansion)
against Fock-space vectors sum_I c_I |D_I>; one determinant, a repeated determinant and a
re-gauged expansion (D_I -> D_I R_I, c_I -> c_I / det R_I, the same state) against the single-determinant
results; a short phaseless run; <D_I|H|D_J> against Fock-space matrix elements for pairs whose
overlap matrix has rank deficiency 0 to 3, and the variational energy of the exact two-electron
ground state written as M^2 orthogonal determinants against the FCI energy.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import afqmc as O

__all__ = ["MSDTrial", "determinant_matrix_elements"]


def _spin_orbitals(D: Tuple[np.ndarray, np.ndarray]) -> np.ndarray:
    """The determinant as one [2M, Nup + Ndn] spin-orbital matrix: spin-up orbitals in rows
    0..M-1 and columns 0..Nup-1, spin-down ones in rows M..2M-1 (the Fock-space ordering)."""
    up, dn = D
    M = up.shape[0]
    out = np.zeros((2 * M, up.shape[1] + dn.shape[1]), dtype=np.complex128)
    out[:M, :up.shape[1]] = up
    out[M:, up.shape[1]:] = dn
    return out


def determinant_matrix_elements(ham: O.Hamiltonian, A: Tuple[np.ndarray, np.ndarray],
                                B: Tuple[np.ndarray, np.ndarray]) -> Tuple[complex, complex]:
    """(<A|B>, <A|H|B>) for two Slater determinants (Loewdin's rules).

    Per spin, the singular value decomposition A_s^+ B_s = U_s diag(sigma) V_s^+ gives orbitals
    a = A U and b = B V with a_k^+ b_l = sigma_k delta_kl; the rotated determinants are
    |a> = det(U)|A> and |b> = det(V)|B>.  Between such biorthogonal determinants, with
    P_k = prod_{m != k} sigma_m and P_kl = prod_{m != k, l} sigma_m (k != l),

      <a|b>   = prod_k sigma_k,
      <a|h|b> = sum_k P_k a_k^+ h b_k,
      <a|V|b> = 1/2 sum_{k != l} P_kl sum_n [X_n[k,k] Y_n[l,l] - X_n[k,l] Y_n[l,k]],

    with X_n[k,r] = a_k^+ L_n b_r and Y_n[l,s] = a_l^+ L_n^+ b_s (spin-conserving, so an up
    orbital meets a down one with zero), since v_ijkl = sum_n L^n_ik conj(L^n_lj) (Eq. (3)) makes
    the two-electron integral <a_k a_l|v|b_r b_s> = sum_n X_n[k,r] Y_n[l,s].  No sigma is inverted,
    so a singular overlap (orthogonal determinants) needs no special case."""
    a_list, b_list, sig = [], [], []
    phase = 1.0 + 0j
    for s in range(2):
        S = A[s].conj().T @ B[s]
        U, sv, Vh = np.linalg.svd(S)
        V = Vh.conj().T
        a_list.append(A[s] @ U)
        b_list.append(B[s] @ V)
        sig.append(sv)
        phase *= np.conj(np.linalg.det(U)) * np.linalg.det(V)
    a = _spin_orbitals((a_list[0], a_list[1]))
    b = _spin_orbitals((b_list[0], b_list[1]))
    sigma = np.concatenate(sig).astype(np.complex128)
    n = sigma.size
    M = ham.M

    def so(Op):   # spin-conserving one-body operator on spin orbitals
        out = np.zeros((2 * M, 2 * M), dtype=np.complex128)
        out[:M, :M] = Op
        out[M:, M:] = Op
        return out

    def prod_except(skip):
        p = 1.0 + 0j
        for m in range(n):
            if m not in skip:
                p *= sigma[m]
        return p

    ovl = prod_except(())
    h1 = so(ham.h)
    e1 = sum(prod_except((k,)) * (a[:, k].conj() @ h1 @ b[:, k]) for k in range(n))
    e2 = 0.0 + 0j
    for nv in range(ham.Nchol):
        Ln = so(ham.L[nv])
        X = a.conj().T @ Ln @ b
        Y = a.conj().T @ Ln.conj().T @ b
        for k in range(n):
            for l in range(n):
                if k != l:
                    e2 += 0.5 * prod_except((k, l)) * (X[k, k] * Y[l, l] - X[k, l] * Y[l, k])
    H_ab = ham.E0 * ovl + e1 + e2
    return ovl / phase, H_ab / phase


def _logsumexp(l: np.ndarray, axis: int) -> np.ndarray:
    m = np.max(l.real, axis=axis, keepdims=True)
    return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(l - m), axis=axis))


class MSDTrial:
    """|psi_T> = sum_I c_I |D_I>; dets[I] = (D_up [M, Nup], D_dn [M, Ndn])."""

    def __init__(self, dets: Sequence[Tuple[np.ndarray, np.ndarray]], c: Sequence[complex]):
        self.dets: List[Tuple[np.ndarray, np.ndarray]] = [
            (np.asarray(u, dtype=np.complex128), np.asarray(d, dtype=np.complex128)) for u, d in dets]
        self.c = np.asarray(c, dtype=np.complex128)
        if self.c.shape != (len(self.dets),) or not np.all(np.isfinite(self.c)) or not np.any(self.c != 0):
            raise ValueError("one finite coefficient per determinant, not all zero")

    @property
    def ND(self) -> int:
        return len(self.dets)

    def reference(self) -> Tuple[np.ndarray, np.ndarray]:
        """The determinant with the largest |c_I| (lowest index on ties)."""
        return self.dets[int(np.argmax(np.abs(self.c)))]

    def _log_terms(self, Phi: Sequence[np.ndarray]) -> np.ndarray:
        """log(conj(c_I) <D_I|Phi_w>): [W, ND]."""
        cols = []
        for I, D in enumerate(self.dets):
            ld = sum(O.log_det(O.overlap_matrix(D[s], Phi[s])) for s in range(2))
            cols.append(np.log(np.conj(self.c[I])) + ld if self.c[I] != 0 else np.full(ld.shape, -np.inf + 0j))
        return np.stack(cols, axis=1)

    def log_overlap(self, Phi: Sequence[np.ndarray]) -> np.ndarray:
        """log <psi_T|Phi_w> for every walker: [W]."""
        return _logsumexp(self._log_terms(Phi), axis=1)

    def weights(self, Phi: Sequence[np.ndarray]) -> np.ndarray:
        """u_I = conj(c_I) <D_I|Phi> / <psi_T|Phi>: [W, ND]."""
        lt = self._log_terms(Phi)
        return np.exp(lt - _logsumexp(lt, axis=1)[:, None])

    def local_energy(self, ham: O.Hamiltonian, Phi: Sequence[np.ndarray]):
        """(E_L [W], t_sum [W, Nchol]): u-weighted sums of the single-determinant values."""
        u = self.weights(Phi)
        E = 0.0
        t = 0.0
        for I, D in enumerate(self.dets):
            if self.c[I] == 0:
                continue
            E_I, t_I, _ = O.local_energy(ham, D, Phi)
            E = E + u[:, I] * E_I
            t = t + u[:, I][:, None] * t_I
        return E, t

    def variational_energy(self, ham: O.Hamiltonian) -> complex:
        """<psi_T|H|psi_T> / <psi_T|psi_T> from the matrix elements between every pair of
        determinants (determinant_matrix_elements), orthogonal pairs included."""
        num = 0.0
        den = 0.0
        for I, DI in enumerate(self.dets):
            for J, DJ in enumerate(self.dets):
                w = np.conj(self.c[I]) * self.c[J]
                if w == 0:
                    continue
                S_IJ, H_IJ = determinant_matrix_elements(ham, DI, DJ)
                num += w * H_IJ
                den += w * S_IJ
        return num / den

    def energy_shift(self, ham: O.Hamiltonian) -> complex:
        """E_T through the overlaps S_IJ = <D_I|D_J> over the pairs with S_IJ != 0: the
        variational energy <psi_T|H|psi_T> / <psi_T|psi_T> when no pair is orthogonal."""
        num = 0.0
        den = 0.0
        for I, DI in enumerate(self.dets):
            for J, DJ in enumerate(self.dets):
                w = np.conj(self.c[I]) * self.c[J]
                if w == 0:
                    continue
                logS = sum(O.log_det(O.overlap_matrix(DI[s], DJ[s][None]))[0] for s in range(2))
                if not np.isfinite(logS.real):
                    continue               # exactly orthogonal pair
                S = np.exp(logS)
                E_IJ = O.local_energy(ham, DI, [DJ[0][None], DJ[1][None]])[0][0]
                num += w * S * E_IJ
                den += w * S
        return num / den
