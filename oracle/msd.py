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

Pins (tests/test_oracle_msd.py): overlap, local energy, force bias and energy shift (the variational energy of a NOMSD expansion)
against Fock-space vectors sum_I c_I |D_I>; one determinant, a repeated determinant and a
re-gauged expansion (D_I -> D_I R_I, c_I -> c_I / det R_I, the same state) against the single-determinant
results; a short phaseless run.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import afqmc as O

__all__ = ["MSDTrial"]


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
