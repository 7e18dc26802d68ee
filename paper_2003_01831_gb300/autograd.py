"""torch.autograd.Function around the local-energy / log-overlap adjoint of the C ABI.

Forward creates an FP64 walker set for the given trial orbitals and walkers on a Hamiltonian
built from the given Cholesky tensor and one-body matrix, and returns the per-walker local
energies and log-overlaps (complex).  Backward calls ``afqmc_energy_backward``, which
recomputes the Green's function on the GPU and returns gradients with respect to the trial
orbitals and the Cholesky tensor in PyTorch's complex convention (d loss/d Re + i d loss/d Im).
Walkers, the one-body matrix and E0 are treated as constants.

Tensors stay where they are: CUDA tensors go to the library as device pointers (inputs are
copied device to device, outputs written on the current stream), and host tensors as host
pointers.  The Hamiltonian (the library's copy of L and h and the derived one-body factor) is
kept across calls while L, h and E0 are unchanged -- same storage, same in-place version
counter -- so an optimisation loop over the trial orbitals uploads L once.
"""
from __future__ import annotations

import torch

from . import api


class _Hamiltonian:
    """A library Hamiltonian with a reference count of the walker sets that use it."""

    def __init__(self, key, h, L, E0, stream):
        self.key = key
        # the key is (storage address, in-place version) of h and L: holding them keeps their
        # memory from being reused by another tensor while this Hamiltonian is cached
        self.refs = (h, L)
        self.M, self.Nchol = h.shape[0], L.shape[0]
        self.handle = api.afqmc_create_hamiltonian(h, L, E0, self.M, self.Nchol, stream)
        self.users = 0
        self.retired = False

    def release(self):
        self.users -= 1
        if self.retired and self.users == 0 and self.handle:
            api.afqmc_destroy_hamiltonian(self.handle)
            self.handle = None


_cache = {"ham": None}


def _key(t):
    return (t.data_ptr(), t._version, tuple(t.shape), str(t.device), t.dtype)


def _hamiltonian(h, L, E0, stream) -> _Hamiltonian:
    key = (_key(h), _key(L), float(E0))
    cur = _cache["ham"]
    if cur is not None and cur.key == key:
        return cur
    if cur is not None:   # retire the previous one; freed once its last walker set is gone
        cur.retired = True
        if cur.users == 0 and cur.handle:
            api.afqmc_destroy_hamiltonian(cur.handle)
            cur.handle = None
    _cache["ham"] = _Hamiltonian(key, h, L, E0, stream)
    return _cache["ham"]


class _WalkerSet:
    """An FP64 walker set; destroyed by backward, or when the autograd graph is freed."""

    def __init__(self, ham, Psi_up, Psi_dn, Phi0, W, stream):
        self.ham = ham
        self.stream = stream
        opts = api.afqmc_default_opts()
        opts.precision = api.PREC_FP64
        opts.k_qr = 0
        self.handle = api.afqmc_init_walkers(ham.handle, Psi_up, Psi_dn, Psi_up.shape[1], Psi_dn.shape[1], W, Phi0,
                                             0.01, opts, stream)
        ham.users += 1

    def close(self):
        if self.handle:
            api.afqmc_destroy_walkers(self.handle)
            self.handle = None
            self.ham.release()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream(dev):
    return torch.cuda.current_stream(dev).cuda_stream if dev.type == "cuda" else None


class LocalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn):
        dev = Psi_up.device
        c128 = lambda t: t.detach().to(device=dev, dtype=torch.complex128).contiguous()
        f64 = lambda t: t.detach().to(device=dev, dtype=torch.float64).contiguous()
        st = _stream(dev)
        hL, Lc = f64(h), f64(L)
        ham = _hamiltonian(hL, Lc, E0, st)
        W = Phi_up.shape[0]
        Phi0 = torch.cat([c128(Phi_up).reshape(W, -1), c128(Phi_dn).reshape(W, -1)], dim=1).contiguous()
        ws = _WalkerSet(ham, c128(Psi_up), c128(Psi_dn), Phi0, W, st)
        E_L = torch.empty(W, dtype=torch.complex128, device=dev)
        logS = torch.empty(W, dtype=torch.complex128, device=dev)
        api.afqmc_energy(ws.handle, E_L, None, logS, None, st)
        ctx.ws = ws
        ctx.shapes = (tuple(Psi_up.shape), tuple(Psi_dn.shape), tuple(L.shape))
        ctx.dev = dev
        return E_L, logS

    @staticmethod
    def backward(ctx, gE, gS):
        ws, dev = ctx.ws, ctx.dev
        c128 = lambda t: None if t is None else t.detach().to(device=dev, dtype=torch.complex128).contiguous()
        su, sd, sL = ctx.shapes
        dPu = torch.empty(su, dtype=torch.complex128, device=dev)
        dPd = torch.empty(sd, dtype=torch.complex128, device=dev)
        dL = torch.empty(sL, dtype=torch.float64, device=dev) if ctx.needs_input_grad[2] else None
        api.afqmc_energy_backward(ws.handle, c128(gE), c128(gS), dPu, dPd, dL, ws.stream)
        ws.close()
        return dPu, dPd, dL, None, None, None, None


def local_energy(Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn):
    """(E_L [W], logS [W]) with gradients w.r.t. Psi_up, Psi_dn and L."""
    return LocalEnergy.apply(Psi_up, Psi_dn, L, h, E0, Phi_up, Phi_dn)
