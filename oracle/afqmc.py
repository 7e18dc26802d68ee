"""Phaseless AFQMC walker step, complex128 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA path.

What the paper fixes (Sec. V):
  * Eq. (1): H = sum_ij h_ij c+_i c_j + 1/2 sum_ijkl v_ijkl c+_i c+_j c_l c_k + E_II
    (spin summed; E_II is called E0 here).
  * Eq. (3): v_ijkl = V_(ik),(lj) ~= sum_n L^n_ik L^n*_lj with Nchol Cholesky
    vectors.  The step works with Hermitian L_n (real symmetric ones in the production
    workloads), for which v_ijkl = sum_n L^n_ik L^n_jl.  General complex L_n are reduced to
    2 Nchol Hermitian ones by ``hermitian_split``: with A_n = (L_n + L_n^+)/2 and
    B_n = (L_n - L_n^+)/(2i), sum_n L^n_ik L^n*_lj and sum_n (A_ik A*_lj + B_ik B*_lj) differ
    only by the exchange of the two electrons, so they are the same two-body operator.
  * The Hubbard-Stratonovich transformation enabled by that factorisation and
    the phaseless AFQMC algorithm are cited, not written out (Zhang & Krakauer
    2003; Motta & Zhang 2018).  The step below restates that textbook algorithm
    from the mathematics.

Rewriting Eq. (1) with c+_i c+_j c_l c_k = E_ik E_jl - delta_jk E_il
(E_ik = sum_sigma c+_{i sigma} c_{k sigma}) gives

    H = sum_il h'_il E_il + 1/2 sum_n Lhat_n^2 + E0,   h' = h - 1/2 sum_n L_n L_n^dagger,

with Lhat_n = sum_ik L^n_ik E_ik.  The HS identity
exp(-tau/2 Lhat^2) = int dx N(x; 0, 1) exp(i sqrt(tau) x Lhat) turns the
two-body factor into one-body operators, and by Thouless' theorem a one-body
exponential maps a Slater determinant Phi (an M x N orbital matrix) to the
determinant exp(X) Phi.

Readings of what the paper leaves open (each one is also listed in the design
notes of the repository):
  * HS operator convention: exponent +i sqrt(tau) sum_n (x_n - xbar_n) L_n.
  * propagate with h', measure the energy with h.
  * force bias xbar_n = -i sqrt(tau) <L_n>, capped per component at |xbar_n| <= fb_cap.
  * truncated Taylor series of order K for the field exponential; the one-body
    halves B = exp(-tau h'/2) come from a symmetric eigendecomposition.
  * weight: w <- w |I| max(0, cos dtheta), I = r exp(x.xbar - xbar.xbar/2)
    exp(tau (E_T - E0)), r = <Psi|Phi'>/<Psi|Phi>, dtheta = arg r (non-conjugated
    bilinear forms in the exponent).
  * E_T is the trial's own local energy, fixed.
  * local-energy weights (mode "local"): w <- w exp(-tau (E_b - E_T)) max(0, cos dtheta)
    with E_b = Re E_L(Phi) of the pre-propagation walker, bounded to E_T +- 2/sqrt(tau).
    This is the first-order form of the hybrid weight: averaged over the fields, the
    hybrid importance factor is exp(-tau (E_L - E_T)) + O(tau^2).
  * population control (comb, outside the step): W slots at (k + xi) W_tot / W against
    the running sum of the weights; slot k takes the walker whose interval holds it; every
    new walker gets weight W_tot / W.
  * walkers with w == 0 are frozen; the energy is measured at the
    pre-propagation Phi with the weights before the update.
  * QR every k_qr steps with diag(R) > 0; logS <- logS - sum log det R.

Pins (tests/test_oracle_pins.py, tests/test_oracle_fock.py): projector
idempotence and trace, HF energy against the 4-index tensor rebuilt by loops,
mixed local energy and force bias against the Fock-space matrix elements,
gauge invariance, Leibniz determinants, Taylor vs eigendecomposition vs
scipy expm, the zero-field one-body limit exp(-tau h), the HS convention by
Gauss-Hermite quadrature against exact Fock-space propagation, QR
properties, and long runs against FCI.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Hamiltonian", "Params", "Walkers",
    "hprime", "half_one_body_propagator", "overlap_matrix", "log_det",
    "half_rotated_green", "rotated_cholesky", "trace_terms", "local_energy",
    "force_bias", "hs_potential", "taylor_exp_apply", "propagate",
    "qr_reorthonormalise", "init_walkers", "step", "run", "mixed_energy",
]


@dataclass
class Hamiltonian:
    """h [M, M] real symmetric, L [Nchol, M, M] real symmetric, E0 scalar (Sec. V, Eqs. (1), (3))."""

    h: np.ndarray
    L: np.ndarray
    E0: float = 0.0

    @property
    def M(self) -> int:
        return self.h.shape[0]

    @property
    def Nchol(self) -> int:
        return self.L.shape[0]


@dataclass
class Params:
    tau: float
    k_taylor: int = 6
    k_qr: int = 0            # 0: never re-orthonormalise
    fb_cap: float = 1.0      # <= 0 disables the cap
    mode: str = "phaseless"  # "free" (free projection: complex weights, no cap, no cos) or
                             # "local" (local-energy weights with the energy bound)


@dataclass
class Walkers:
    Phi: List[np.ndarray]      # per spin: [W, M, N_sigma] complex128
    w: np.ndarray              # [W] float64 (phaseless) or complex128 (free)
    logS: np.ndarray           # [W] complex128, sum_sigma log det(Psi_sigma^dagger Phi_sigma)
    E_T: float
    nstep: int = 0

    @property
    def W(self) -> int:
        return self.w.shape[0]


# --------------------------------------------------------------------------------------------
# One-body pieces
# --------------------------------------------------------------------------------------------

def hprime(ham: Hamiltonian) -> np.ndarray:
    """h' = h - 1/2 sum_n L_n L_n^dagger (from Eq. (1) with Eq. (3) after normal ordering);
    real for real inputs, Hermitian for complex ones."""
    hp = ham.h - 0.5 * np.tensordot(ham.L, ham.L.conj(), axes=([0, 2], [0, 2]))   # sum_nk L_nik L*_njk
    return hp.real if np.isrealobj(ham.L) and np.isrealobj(ham.h) else hp


def half_one_body_propagator(ham: Hamiltonian, tau: float) -> np.ndarray:
    """B = exp(-tau h'/2) from the eigendecomposition of the Hermitian h'."""
    e, v = np.linalg.eigh(hprime(ham))
    return (v * np.exp(-0.5 * tau * e)) @ v.conj().T


def hermitian_split(L: np.ndarray) -> np.ndarray:
    """2 Nchol Hermitian operators [A_0, B_0, A_1, B_1, ...] from complex L [Nchol, M, M]:
    A_n = (L_n + L_n^+)/2, B_n = (L_n - L_n^+)/(2i).  They give the same two-body operator as
    L (the four-index tensors differ only by the exchange of the two electrons).  Written as
    1/2 sum (A^2 + B^2) the interaction needs h' = h - 1/4 sum (L L^+ + L^+ L), which is what
    hprime returns for the split vectors; 1/2 sum L L^+ differs from it by the one-body
    commutator term 1/4 sum [L, L^+]."""
    Ld = np.conj(np.swapaxes(L, 1, 2))
    A = 0.5 * (L + Ld)
    B = (L - Ld) / 2j
    out = np.empty((2 * L.shape[0],) + L.shape[1:], dtype=np.complex128)
    out[0::2] = A
    out[1::2] = B
    return out


# --------------------------------------------------------------------------------------------
# Overlap, Green's function, energy
# --------------------------------------------------------------------------------------------

def overlap_matrix(Psi: np.ndarray, Phi: np.ndarray) -> np.ndarray:
    """S = Psi^dagger Phi for every walker: [W, N, N]."""
    return np.einsum("ka,wkb->wab", Psi.conj(), Phi)


def log_det(S: np.ndarray) -> np.ndarray:
    """Complex log det of each matrix: log|det| + i arg(det)."""
    sign, logabs = np.linalg.slogdet(S)
    return logabs + 1j * np.angle(sign)


def half_rotated_green(Psi: np.ndarray, Phi: np.ndarray) -> np.ndarray:
    """Theta = Phi (Psi^dagger Phi)^-1: [W, M, N].  The mixed one-body density
    <c+_i c_k> equals (Theta Psi^dagger)_{ki}."""
    S = overlap_matrix(Psi, Phi)
    return np.einsum("wkj,wjb->wkb", Phi, np.linalg.inv(S))


def rotated_cholesky(Psi: np.ndarray, L: np.ndarray) -> np.ndarray:
    """Ltilde_n = Psi^dagger L_n: [Nchol, N, M] (one library matrix product per vector)."""
    return np.matmul(Psi.conj().T, L)


def trace_terms(Lt: np.ndarray, Theta: np.ndarray):
    """For T_{w,n} = Ltilde_n Theta_w (N x N): t[w, n] = Tr T and X[w, n] = Tr(T T).

    T is formed explicitly, one walker at a time (memory Nchol * N * N)."""
    W = Theta.shape[0]
    nch = Lt.shape[0]
    t = np.empty((W, nch), dtype=np.complex128)
    X = np.empty((W, nch), dtype=np.complex128)
    for w in range(W):
        T = np.matmul(Lt, Theta[w])                        # [Nchol, N, N]
        t[w] = np.trace(T, axis1=1, axis2=2)
        X[w] = np.einsum("nab,nba->n", T, T)
    return t, X


def local_energy(ham: Hamiltonian, Psi: Sequence[np.ndarray], Phi: Sequence[np.ndarray]):
    """Mixed-estimator local energy <Psi|H|Phi>/<Psi|Phi> per walker.

    E_L = E0 + sum_s Tr(htilde_s Theta_s) + 1/2 sum_n [(sum_s t_ns)^2 - sum_s X_ns]
    with htilde_s = Psi_s^dagger h.  Returns (E_L [W], t_sum [W, Nchol], Theta list)."""
    E1 = 0.0
    t_sum = 0.0
    X_sum = 0.0
    thetas = []
    for s in range(2):
        Th = half_rotated_green(Psi[s], Phi[s])
        thetas.append(Th)
        ht = Psi[s].conj().T @ ham.h                       # [N, M]
        E1 = E1 + np.einsum("ak,wka->w", ht, Th)
        t, X = trace_terms(rotated_cholesky(Psi[s], ham.L), Th)
        t_sum = t_sum + t
        X_sum = X_sum + X
    E2 = 0.5 * np.sum(t_sum * t_sum - X_sum, axis=1)
    return ham.E0 + E1 + E2, t_sum, thetas


def trial_local_energy(ham: Hamiltonian, Psi, Phi: Sequence[np.ndarray]):
    """(E_L [W], t_sum [W, Nchol]) for a single-determinant trial (the pair of orbital
    matrices Psi) or a multi-determinant one (an object with its own ``local_energy``,
    ``oracle.msd.MSDTrial``)."""
    if hasattr(Psi, "local_energy"):
        return Psi.local_energy(ham, Phi)
    E_L, t_sum, _ = local_energy(ham, Psi, Phi)
    return E_L, t_sum


def trial_log_overlap(Psi, Phi: Sequence[np.ndarray]) -> np.ndarray:
    """log <Psi_T|Phi_w>: [W] (single determinant: sum over spins of log det(Psi^+ Phi))."""
    if hasattr(Psi, "log_overlap"):
        return Psi.log_overlap(Phi)
    return sum(log_det(overlap_matrix(Psi[s], Phi[s])) for s in range(2))


def force_bias(t_sum: np.ndarray, tau: float, fb_cap: float) -> np.ndarray:
    """xbar_n = -i sqrt(tau) <L_n>, each component capped at |xbar_n| <= fb_cap."""
    xbar = -1j * np.sqrt(tau) * t_sum
    if fb_cap > 0:
        mag = np.abs(xbar)
        over = mag > fb_cap
        xbar = np.where(over, fb_cap * xbar / np.where(over, mag, 1.0), xbar)
    return xbar


# --------------------------------------------------------------------------------------------
# Propagation
# --------------------------------------------------------------------------------------------

def hs_potential(c: np.ndarray, L: np.ndarray) -> np.ndarray:
    """A_w = sum_n c[w, n] L_n: [W, M, M] complex."""
    return np.einsum("wn,nij->wij", c, L)


def taylor_exp_apply(X: np.ndarray, Phi: np.ndarray, K: int) -> np.ndarray:
    """sum_{k=0}^{K} X^k Phi / k! for every walker, by the recursion P_k = X P_{k-1} / k."""
    acc = Phi.copy()
    P = Phi
    for k in range(1, K + 1):
        P = np.matmul(X, P) / k
        acc = acc + P
    return acc


def propagate(Phi: np.ndarray, A: np.ndarray, B: np.ndarray, tau: float, K: int) -> np.ndarray:
    """Phi' = B T_K(i sqrt(tau) A) B Phi for one spin: [W, M, N]."""
    P = np.matmul(B, Phi)
    P = taylor_exp_apply(1j * np.sqrt(tau) * A, P, K)
    return np.matmul(B, P)


def qr_reorthonormalise(Phi: np.ndarray):
    """Phi = Q R with diag(R) > 0; returns (Q, sum log diag R) per walker."""
    Q, R = np.linalg.qr(Phi)
    d = np.diagonal(R, axis1=1, axis2=2)
    ph = d / np.abs(d)
    Q = Q * ph[:, None, :]
    logdetR = np.sum(np.log(np.abs(d)), axis=1)
    return Q, logdetR


# --------------------------------------------------------------------------------------------
# Walker set and step
# --------------------------------------------------------------------------------------------

def init_walkers(ham: Hamiltonian, Psi: Sequence[np.ndarray], W: int,
                 Phi0: Optional[Sequence[np.ndarray]] = None, complex_weights: bool = False) -> Walkers:
    """Walkers start at Phi0 (or the trial; a multi-determinant trial's largest-weight
    determinant), w = 1, E_T = the trial's variational energy (for one determinant its own
    local energy)."""
    multi = hasattr(Psi, "energy_shift")
    if Phi0 is None:
        ref = Psi.reference() if multi else Psi
        Phi = [np.repeat(np.asarray(p, dtype=np.complex128)[None], W, axis=0) for p in ref]
    else:
        Phi = [np.array(p, dtype=np.complex128) for p in Phi0]
    logS = trial_log_overlap(Psi, Phi)
    E_T = Psi.energy_shift(ham).real if multi else local_energy(ham, Psi, [p[None] for p in Psi])[0][0].real
    w = np.ones(W, dtype=np.complex128 if complex_weights else np.float64)
    return Walkers(Phi=Phi, w=w, logS=logS, E_T=E_T)


def mixed_energy(w: np.ndarray, E_L: np.ndarray) -> complex:
    """E_mix = sum_w w E_L / sum_w w."""
    return np.sum(w * E_L) / np.sum(w)


def step(ham: Hamiltonian, Psi: Sequence[np.ndarray], B: np.ndarray, wk: Walkers,
         x: np.ndarray, p: Params, record: Optional[list] = None):
    """One phaseless step for every walker with fields x [W, Nchol].

    Returns (E_L [W] at the pre-step walkers, E_mix with the pre-step weights).
    Updates wk in place.  Psi is the trial: the pair of orbital matrices of a single
    determinant, or an ``oracle.msd.MSDTrial``.  If `record` is a list, the shifted fields c = x - xbar that drove
    each walker's propagator are appended to it ([W, Nchol]; zero rows for frozen walkers)."""
    E_L, t_sum = trial_local_energy(ham, Psi, wk.Phi)
    E_mix = mixed_energy(wk.w, E_L)
    free = p.mode == "free"
    xbar = force_bias(t_sum, p.tau, 0.0 if free else p.fb_cap)
    alive = wk.w != 0
    c = x - xbar
    if record is not None:
        record.append(np.where(alive[:, None], c, 0.0))
    A = hs_potential(c, ham.L)
    newPhi = [propagate(wk.Phi[s], A, B, p.tau, p.k_taylor) for s in range(2)]
    newlogS = trial_log_overlap(Psi, newPhi)
    dl = newlogS - wk.logS
    expo = dl + np.sum(x * xbar, axis=1) - 0.5 * np.sum(xbar * xbar, axis=1) \
        + p.tau * (wk.E_T - ham.E0)
    ok = alive & np.isfinite(newlogS)
    if free:
        neww = wk.w * np.exp(expo)
    elif p.mode == "local":
        neww = wk.w * local_energy_factor(E_L, wk.E_T, p.tau) * np.maximum(0.0, np.cos(dl.imag))
    else:
        neww = wk.w * np.exp(expo.real) * np.maximum(0.0, np.cos(dl.imag))
    wk.w = np.where(ok, neww, np.where(alive, 0.0, wk.w))
    for s in range(2):
        wk.Phi[s] = np.where(ok[:, None, None], newPhi[s], wk.Phi[s])
    wk.logS = np.where(ok, newlogS, wk.logS)
    wk.nstep += 1
    if p.k_qr > 0 and wk.nstep % p.k_qr == 0:
        live = wk.w != 0
        for s in range(2):
            Q, ldr = qr_reorthonormalise(wk.Phi[s])
            wk.Phi[s] = np.where(live[:, None, None], Q, wk.Phi[s])
            wk.logS = np.where(live, wk.logS - ldr, wk.logS)
    return E_L, E_mix


def energy_bound(E_L: np.ndarray, E_T: float, tau: float) -> np.ndarray:
    """Re E_L clipped to E_T +- 2/sqrt(tau)."""
    b = 2.0 / np.sqrt(tau)
    return np.clip(np.real(E_L), E_T - b, E_T + b)


def local_energy_factor(E_L: np.ndarray, E_T: float, tau: float) -> np.ndarray:
    """exp(-tau (E_b - E_T)) with the bounded local energy E_b."""
    return np.exp(-tau * (energy_bound(E_L, E_T, tau) - E_T))


def comb(w: np.ndarray, xi: float) -> np.ndarray:
    """Comb population control: indices of the W walkers that fill the W new slots.

    Slot k (k = 0..W-1) sits at u_k = (k + xi) W_tot / W on the running sum of the weights
    c_j = w_0 + ... + w_j (accumulated left to right in float64); it takes the first walker
    j with c_j > u_k (the last live walker if rounding leaves none).  A walker of weight w_j is copied floor or ceil of W w_j / W_tot times;
    walkers of weight 0 are never taken.  xi in [0, 1) is the one random number of the comb."""
    w = np.asarray(w, dtype=np.float64)
    W = w.size
    c = np.empty(W)
    acc = 0.0
    for j in range(W):
        acc += w[j]
        c[j] = acc
    total = acc
    live = np.nonzero(w > 0)[0]
    last = int(live[-1]) if live.size else W - 1   # a slot rounded onto the total takes it
    idx = np.empty(W, dtype=np.int64)
    j = 0
    for k in range(W):
        u = (k + xi) * total / W
        while j < last and not (c[j] > u):
            j += 1
        idx[k] = j
    return idx


def population_control(wk: Walkers, xi: float) -> np.ndarray:
    """Apply the comb to walkers in place (phaseless weights only); returns the indices."""
    if np.iscomplexobj(wk.w):
        raise ValueError("population control needs real weights")
    idx = comb(wk.w, xi)
    total = float(np.sum(wk.w))
    for s in range(2):
        wk.Phi[s] = wk.Phi[s][idx].copy()
    wk.logS = wk.logS[idx].copy()
    wk.w = np.full(wk.w.size, total / wk.w.size)
    return idx


def run(ham: Hamiltonian, Psi: Sequence[np.ndarray], W: int, fields: np.ndarray, p: Params,
        Phi0=None, record_walkers: bool = False):
    """Trajectory driver: fields [nsteps, W, Nchol].  Returns a dict of traces."""
    B = half_one_body_propagator(ham, p.tau)
    wk = init_walkers(ham, Psi, W, Phi0, complex_weights=(p.mode == "free"))
    out = {"E_L": [], "E_mix": [], "w": [], "logS": [], "E_T": wk.E_T}
    for s in range(fields.shape[0]):
        E_L, E_mix = step(ham, Psi, B, wk, fields[s], p)
        out["E_L"].append(E_L)
        out["E_mix"].append(E_mix)
        if record_walkers:
            out["w"].append(wk.w.copy())
            out["logS"].append(wk.logS.copy())
    out["walkers"] = wk
    return out
