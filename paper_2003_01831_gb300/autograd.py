"""torch.autograd.Function around the local-energy / log-overlap adjoint of the C ABI.

Forward builds an FP64 walker set for the given trial orbitals, Cholesky tensor and
walkers and returns the per-walker local energies and log-overlaps (complex).
Backward calls ``afqmc_energy_backward``, which recomputes the Green's function on the
GPU and returns gradients with respect to the trial orbitals and the Cholesky tensor
in PyTorch's complex convention (d loss/d Re + i d loss/d Im).  Walkers, the one-body
matrix and E0 are treated as constants.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from .walkers import AFQMC


def _np(t):
    return t.detach().cpu().numpy()


class LocalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn):
        W = Phi_up.shape[0]
        sys_ = AFQMC(_np(h), _np(L), float(E0), _np(Psi_up), _np(Psi_dn), W, 0.01,
                     Phi0=[_np(Phi_up), _np(Phi_dn)], precision=api.PREC_FP64, k_qr=0)
        E_L, _, logS, _ = sys_.energy()
        ctx.sys = sys_
        ctx.dev = Psi_up.device
        return (torch.from_numpy(E_L).to(Psi_up.device), torch.from_numpy(logS).to(Psi_up.device))

    @staticmethod
    def backward(ctx, gE, gS):
        sys_ = ctx.sys
        dE = None if gE is None else _np(gE).astype(np.complex128)
        dS = None if gS is None else _np(gS).astype(np.complex128)
        dPu, dPd, dL = sys_.backward(dE, dS, want_L=ctx.needs_input_grad[2])
        sys_.close()
        dev = ctx.dev
        out_L = torch.from_numpy(dL).to(dev) if dL is not None else None
        return (torch.from_numpy(dPu).to(dev), torch.from_numpy(dPd).to(dev), out_L, None, None, None, None)


def local_energy(Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn):
    """(E_L [W], logS [W]) with gradients w.r.t. Psi_up, Psi_dn and L."""
    return LocalEnergy.apply(Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn)
