"""Brute-force Fock-space quantum chemistry for tiny systems (test infrastructure only).

Used solely to pin the oracle in ``afqmc.py``; the product path never calls it.

The Hamiltonian of Sec. V, Eq. (1) is built term by term from fermionic
creation/annihilation operators acting on occupation bitstrings, with the
4-index tensor v_ijkl rebuilt from the Cholesky vectors of Eq. (3) by
explicit loops.  Nothing here uses the h' rewriting, the half-rotated Green's
function or the Hubbard-Stratonovich transformation, so agreement with the
oracle's local energy, force bias and propagator checks those independently.

Conventions: spin orbitals 0..M-1 are spin up, M..2M-1 spin down; a basis
state with occupied spin orbitals p_1 < ... < p_k is c+_{p_1} ... c+_{p_k}|0>,
so c+_p and c_p carry the sign (-1)^(number of occupied orbitals below p).
"""
from __future__ import annotations

from itertools import combinations
from typing import Dict, List, Tuple

import numpy as np

__all__ = ["four_index_from_cholesky", "FockSpace", "slater_vector"]


def four_index_from_cholesky(L: np.ndarray) -> np.ndarray:
    """v_ijkl = sum_n L^n_ik conj(L^n_lj), by explicit loops (Eq. (3))."""
    nch, M, _ = L.shape
    v = np.zeros((M, M, M, M), dtype=np.result_type(L, np.float64))
    for i in range(M):
        for j in range(M):
            for k in range(M):
                for l in range(M):
                    acc = 0.0
                    for n in range(nch):
                        acc += L[n, i, k] * np.conj(L[n, l, j])
                    v[i, j, k, l] = acc
    return v


def _annihilate(state: int, p: int):
    if not (state >> p) & 1:
        return 0, state
    sign = -1 if bin(state & ((1 << p) - 1)).count("1") % 2 else 1
    return sign, state ^ (1 << p)


def _create(state: int, p: int):
    if (state >> p) & 1:
        return 0, state
    sign = -1 if bin(state & ((1 << p) - 1)).count("1") % 2 else 1
    return sign, state | (1 << p)


class FockSpace:
    """Fixed (N_up, N_dn) sector of M spatial orbitals."""

    def __init__(self, M: int, Nup: int, Ndn: int):
        self.M, self.Nup, self.Ndn = M, Nup, Ndn
        states = []
        for up in combinations(range(M), Nup):
            for dn in combinations(range(M), Ndn):
                s = 0
                for p in up:
                    s |= 1 << p
                for p in dn:
                    s |= 1 << (M + p)
                states.append(s)
        self.states = states
        self.index: Dict[int, int] = {s: i for i, s in enumerate(states)}
        self.dim = len(states)

    def hamiltonian(self, h: np.ndarray, v: np.ndarray, E0: float = 0.0) -> np.ndarray:
        """Dense matrix of Eq. (1): sum h_ij c+_i c_j + 1/2 sum v_ijkl c+_i c+_j c_l c_k + E0,
        with both spins summed in every one-body and two-body term."""
        M = self.M
        H = np.zeros((self.dim, self.dim), dtype=np.result_type(h, v, np.float64))
        for col, s0 in enumerate(self.states):
            H[col, col] += E0
            occ = [p for p in range(2 * M) if (s0 >> p) & 1]
            # one-body
            for q in occ:
                sg1, s1 = _annihilate(s0, q)
                spin_off = M if q >= M else 0
                for i in range(M):
                    sg2, s2 = _create(s1, i + spin_off)
                    if sg2:
                        H[self.index[s2], col] += sg1 * sg2 * h[i, q - spin_off]
            # two-body: c+_{i s} c+_{j s'} c_{l s'} c_{k s}, k acts first
            for kk in occ:
                sg1, s1 = _annihilate(s0, kk)
                for ll in occ:
                    if ll == kk:
                        continue
                    sg2, s2 = _annihilate(s1, ll)
                    if not sg2:
                        continue
                    off_k = M if kk >= M else 0
                    off_l = M if ll >= M else 0
                    k, l = kk - off_k, ll - off_l
                    for j in range(M):
                        sg3, s3 = _create(s2, j + off_l)
                        if not sg3:
                            continue
                        for i in range(M):
                            sg4, s4 = _create(s3, i + off_k)
                            if not sg4:
                                continue
                            H[self.index[s4], col] += 0.5 * sg1 * sg2 * sg3 * sg4 * v[i, j, k, l]
        return H

    def one_body_operator(self, O: np.ndarray) -> np.ndarray:
        """Dense matrix of sum_{ik, sigma} O_ik c+_{i sigma} c_{k sigma}."""
        M = self.M
        out = np.zeros((self.dim, self.dim), dtype=np.result_type(O, np.float64))
        for col, s0 in enumerate(self.states):
            for q in range(2 * M):
                sg1, s1 = _annihilate(s0, q)
                if not sg1:
                    continue
                off = M if q >= M else 0
                for i in range(M):
                    sg2, s2 = _create(s1, i + off)
                    if sg2:
                        out[self.index[s2], col] += sg1 * sg2 * O[i, q - off]
        return out

    def slater_vector(self, Phi_up: np.ndarray, Phi_dn: np.ndarray) -> np.ndarray:
        """Fock-space coefficients of prod_j (sum_i Phi_up[i,j] c+_i) prod_j (...) |0>.

        The coefficient of the state with occupied up rows U and down rows D
        (both ascending) is det(Phi_up[U]) det(Phi_dn[D])."""
        M = self.M
        vec = np.zeros(self.dim, dtype=np.complex128)
        for idx, s in enumerate(self.states):
            up = [p for p in range(M) if (s >> p) & 1]
            dn = [p - M for p in range(M, 2 * M) if (s >> p) & 1]
            vec[idx] = np.linalg.det(Phi_up[up, :]) * np.linalg.det(Phi_dn[dn, :])
        return vec


def slater_vector(fs: FockSpace, Phi_up, Phi_dn):
    return fs.slater_vector(Phi_up, Phi_dn)
