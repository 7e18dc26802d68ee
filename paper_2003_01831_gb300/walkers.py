"""Convenience wrapper over the C ABI: one Hamiltonian plus one walker set.

Argument marshalling only -- every step of the method runs in the CUDA
library (``include/afqmc.h``).  Inputs are numpy arrays on the host; outputs
come back as numpy arrays.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import api


class AFQMC:
    """Owns an ``afqmc_ham_t`` and an ``afqmc_wk_t``; release with ``close()``.

    With ``coeffs`` (complex [ND]) the trial is the expansion sum_I c_I |D_I>, and Psi_up /
    Psi_dn hold the determinants ([ND, M, Nup] / [ND, M, Ndn]).  With ``thc=(X, Mk)`` the
    Hamiltonian is in tensor-hypercontraction form (L is then ignored and may be None)."""

    def __init__(self, h, L, E0, Psi_up, Psi_dn, W, tau, Phi0=None, precision=api.PREC_FP64,
                 k_taylor=6, k_qr=5, fb_cap=1.0, weight_mode=api.WEIGHT_PHASELESS, walker_offset=0, energy_terms=0,
                 stream=None, coeffs=None, thc=None):
        h = np.ascontiguousarray(h, dtype=np.float64)
        if thc is not None:
            L = np.zeros((1, 1, 1))
        # complex L: general complex Cholesky vectors, run as their 2 Nchol Hermitian-split
        # vectors (A_0, B_0, A_1, B_1, ...), which is what fields and Nchol refer to
        self.complex_L = np.iscomplexobj(L)
        L = np.ascontiguousarray(L, dtype=np.complex128 if self.complex_L else np.float64)
        self.M = h.shape[0]
        self.Nchol = L.shape[0] * (2 if self.complex_L else 1)
        self.Psi = [np.ascontiguousarray(Psi_up, dtype=np.complex128),
                    np.ascontiguousarray(Psi_dn, dtype=np.complex128)]
        self.N = [self.Psi[0].shape[-1], self.Psi[1].shape[-1]]
        self.W = int(W)
        self.weight_mode = weight_mode
        self.stream = stream
        if thc is not None:
            X = np.ascontiguousarray(thc[0], dtype=np.float64)
            Mk = np.ascontiguousarray(thc[1], dtype=np.float64)
            self.ham = api.afqmc_create_hamiltonian_thc(h, X, Mk, E0, self.M, X.shape[1], stream)
            self.Nchol = api.afqmc_hamiltonian_info(self.ham)[1]
        elif self.complex_L:
            self.ham = api.afqmc_create_hamiltonian_complex(h, L, E0, self.M, L.shape[0], stream)
        else:
            self.ham = api.afqmc_create_hamiltonian(h, L, E0, self.M, self.Nchol, stream)
        opts = api.afqmc_default_opts()
        opts.precision = precision
        opts.k_taylor = k_taylor
        opts.k_qr = k_qr
        opts.fb_cap = fb_cap
        opts.weight_mode = weight_mode
        opts.walker_offset = walker_offset
        opts.energy_terms = energy_terms
        phi0 = None
        if Phi0 is not None:
            phi0 = np.ascontiguousarray(np.concatenate(
                [np.asarray(Phi0[0]).reshape(self.W, -1), np.asarray(Phi0[1]).reshape(self.W, -1)], axis=1),
                dtype=np.complex128)
        try:
            if coeffs is None:
                self.wk = api.afqmc_init_walkers(self.ham, self.Psi[0], self.Psi[1], self.N[0], self.N[1], self.W,
                                                 phi0, tau, opts, stream)
            else:
                c = np.ascontiguousarray(coeffs, dtype=np.complex128)
                self.wk = api.afqmc_init_walkers_msd(self.ham, c.size, self.Psi[0], self.Psi[1], c, self.N[0],
                                                     self.N[1], self.W, phi0, tau, opts, stream)
        except Exception:
            api.afqmc_destroy_hamiltonian(self.ham)
            self.ham = None
            self.wk = None
            raise

    # ---------------------------------------------------------------- stepping
    def step(self, nsteps: int, x: Optional[np.ndarray] = None, seed: int = 0, measure_every: int = 0):
        """Run nsteps; returns the complex E_mix trace (empty if measure_every == 0)."""
        nmeas = (nsteps + measure_every - 1) // measure_every if measure_every > 0 else 0
        trace = np.zeros(max(nmeas, 1), dtype=np.complex128)
        if x is not None:
            x = np.ascontiguousarray(x, dtype=np.float64)
            assert x.size == nsteps * self.W * self.Nchol
        api.afqmc_step(self.wk, nsteps, x, seed, measure_every, trace if nmeas else None, self.stream)
        return trace[:nmeas]

    def energy(self):
        """(E_L [W] complex, w [W], logS [W] complex, E_mix complex) at the current walkers."""
        E_L = np.zeros(self.W, dtype=np.complex128)
        logS = np.zeros(self.W, dtype=np.complex128)
        w = np.zeros(self.W, dtype=np.complex128 if self.weight_mode == api.WEIGHT_FREE else np.float64)
        E = np.zeros(1, dtype=np.complex128)
        api.afqmc_energy(self.wk, E_L, w, logS, E, self.stream)
        return E_L, w, logS, E[0]

    def walkers(self):
        """(Phi_up [W, M, Nup], Phi_dn [W, M, Ndn], w [W], step)."""
        M, (Nu, Nd) = self.M, self.N
        Phi = np.zeros((self.W, M * (Nu + Nd)), dtype=np.complex128)
        w = np.zeros(self.W, dtype=np.complex128 if self.weight_mode == api.WEIGHT_FREE else np.float64)
        step = api.afqmc_get_walkers(self.wk, Phi, w, self.stream)
        return Phi[:, :M * Nu].reshape(self.W, M, Nu), Phi[:, M * Nu:].reshape(self.W, M, Nd), w, step

    def population_control(self, xi: float) -> np.ndarray:
        """Comb population control (phaseless or local-energy weights); returns the source
        walker of every new walker."""
        idx = np.zeros(self.W, dtype=np.int32)
        api.afqmc_population_control(self.wk, xi, idx, self.stream)
        return idx

    def bp_begin(self, nbp: int):
        """Open a back-propagation window of nbp steps at the current walkers."""
        api.afqmc_bp_begin(self.wk, nbp, self.stream)

    def bp_rdm1(self):
        """(G_up, G_dn): back-propagated one-body density matrices, G[i, j] = <c+_i c_j>,
        once the window's nbp steps have run."""
        G = [np.zeros((self.M, self.M), dtype=np.complex128) for _ in range(2)]
        api.afqmc_bp_rdm1(self.wk, G[0], G[1], self.stream)
        return G[0], G[1]

    def set_walkers(self, Phi_up, Phi_dn, w, step: int):
        Phi = np.ascontiguousarray(np.concatenate(
            [np.asarray(Phi_up).reshape(self.W, -1), np.asarray(Phi_dn).reshape(self.W, -1)], axis=1),
            dtype=np.complex128)
        api.afqmc_set_walkers(self.wk, Phi, np.ascontiguousarray(w), step, self.stream)

    def backward(self, dE=None, dlogS=None, want_L: bool = True):
        dE = None if dE is None else np.ascontiguousarray(dE, dtype=np.complex128)
        dlogS = None if dlogS is None else np.ascontiguousarray(dlogS, dtype=np.complex128)
        dPu = np.zeros((self.M, self.N[0]), dtype=np.complex128)
        dPd = np.zeros((self.M, self.N[1]), dtype=np.complex128)
        dL = np.zeros((self.Nchol, self.M, self.M), dtype=np.float64) if want_L and not self.complex_L else None
        api.afqmc_energy_backward(self.wk, dE, dlogS, dPu, dPd, dL, self.stream)
        return dPu, dPd, dL

    def close(self):
        if getattr(self, "wk", None):
            api.afqmc_destroy_walkers(self.wk)
            self.wk = None
        if getattr(self, "ham", None):
            api.afqmc_destroy_hamiltonian(self.ham)
            self.ham = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owns an ``afqmc_batch_t``: independent systems (h, L, E0, Psi_up, Psi_dn, W) stepped
    together, one CUDA-graph launch per step; release with ``close()``."""

    def __init__(self, systems, tau, precision=api.PREC_FP64, k_taylor=6, k_qr=5, fb_cap=1.0,
                 weight_mode=api.WEIGHT_PHASELESS, pad_mode=api.PAD_AUTO, stream=None):
        self.stream = stream
        self.weight_mode = weight_mode
        keep, structs = [], []
        self.shapes = []
        for (h, L, E0, Pu, Pd, W) in systems:
            h = np.ascontiguousarray(h, dtype=np.float64)
            L = np.ascontiguousarray(L, dtype=np.float64)
            Pu = np.ascontiguousarray(Pu, dtype=np.complex128)
            Pd = np.ascontiguousarray(Pd, dtype=np.complex128)
            keep += [h, L, Pu, Pd]
            M, nch = h.shape[0], L.shape[0]
            self.shapes.append((M, Pu.shape[1], Pd.shape[1], nch, int(W)))
            structs.append(api.System(h=h.ctypes.data, L=L.ctypes.data, E0=float(E0), M=M, Nchol=nch,
                                      Psi_up=Pu.ctypes.data, Psi_dn=Pd.ctypes.data, Nup=Pu.shape[1],
                                      Ndn=Pd.shape[1], W=int(W), Phi0=None))
        opts = api.afqmc_default_opts()
        opts.precision = precision
        opts.k_taylor = k_taylor
        opts.k_qr = k_qr
        opts.fb_cap = fb_cap
        opts.weight_mode = weight_mode
        self.n = len(structs)
        self.b = api.afqmc_create_batch(structs, tau, opts, pad_mode, stream)

    def step(self, nsteps: int, seed: int = 0, measure_every: int = 0):
        """Run nsteps; returns the complex E_mix trace [nmeas][nsys]."""
        nmeas = (nsteps + measure_every - 1) // measure_every if measure_every > 0 else 0
        trace = np.zeros((max(nmeas, 1), self.n), dtype=np.complex128)
        api.afqmc_batch_step(self.b, nsteps, seed, measure_every, trace if nmeas else None, self.stream)
        return trace[:nmeas]

    def energy(self, s: int):
        W = self.shapes[s][4]
        E_L = np.zeros(W, dtype=np.complex128)
        logS = np.zeros(W, dtype=np.complex128)
        w = np.zeros(W, dtype=np.complex128 if self.weight_mode == api.WEIGHT_FREE else np.float64)
        E = np.zeros(1, dtype=np.complex128)
        api.afqmc_batch_energy(self.b, s, E_L, w, logS, E, self.stream)
        return E_L, w, logS, E[0]

    def walkers(self, s: int):
        M, Nu, Nd, _, W = self.shapes[s]
        Phi = np.zeros((W, M * (Nu + Nd)), dtype=np.complex128)
        w = np.zeros(W, dtype=np.complex128 if self.weight_mode == api.WEIGHT_FREE else np.float64)
        step = api.afqmc_batch_get_walkers(self.b, s, Phi, w, self.stream)
        return Phi[:, :M * Nu].reshape(W, M, Nu), Phi[:, M * Nu:].reshape(W, M, Nd), w, step

    def info(self, s: int = 0):
        return api.afqmc_batch_info(self.b, s)

    def autotune(self, reps: int = 2) -> float:
        return api.afqmc_batch_autotune(self.b, reps, self.stream)

    def close(self):
        if getattr(self, "b", None):
            api.afqmc_destroy_batch(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
