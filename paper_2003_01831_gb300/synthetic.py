"""Seeded synthetic inputs shaped like the AFQMC workloads of Sec. V.

This module only draws random numbers and arranges them into the inputs of
the Hamiltonian of Sec. V, Eq. (1) with the modified-Cholesky factorisation
of Eq. (3): a one-body matrix ``h``, a real symmetric Cholesky tensor
``L[n, i, k]``, a single-determinant trial and, for timing runs, Gaussian
auxiliary fields.  It holds none of the AFQMC arithmetic (no overlaps,
energies, propagators or weights), so the CUDA path and the CPU oracle can
both consume what it produces without sharing any of the method.

Workload recipe (the paper's molecules and solids are not available, so these
stand in for them):

* ``h`` (molecule-like): symmetric, diagonal ~ U[-2, 2], off-diagonal
  ~ N(0, 0.1) (standard deviation 0.1).
* ``h`` (solid-like, ``band`` given): symmetric, entries ~ N(0, 0.2) for
  ``|i - j| <= band`` (diagonal included), zero outside the band.
* ``L_n``: upper triangle (diagonal included) i.i.d. N(0, 1), mirrored, times
  ``0.5 * exp(-n / decay)``.  Reading "R1" multiplies by a further
  ``1 / sqrt(M)`` so that the field operator ``sqrt(tau) * sum_n x_n L_n``
  keeps a spectral norm below one at every size (the literal reading "R0"
  makes the truncated Taylor propagator diverge at M = 512).
* trial: the ``N`` lowest eigenvectors of ``h`` for both spins.
* random generator: ``numpy.random.default_rng(1000 + index)``, drawing
  ``h`` first and ``L`` second.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Workload",
    "make_hamiltonian",
    "make_trial",
    "make_fields",
    "make_random_walkers",
    "make_thc",
    "WORKLOADS",
    "workload",
    "uneven_batch",
    "make_uneven_system",
]


@dataclass
class Workload:
    """One synthetic system and the run parameters used with it."""

    name: str
    index: int
    M: int
    Nup: int
    Ndn: int
    Nchol: int
    W: int
    tau: float
    nsteps: int
    k_qr: int
    decay: float = 20.0
    band: Optional[int] = None
    reading: str = "R1"
    notes: str = ""

    def rng(self) -> np.random.Generator:
        return np.random.default_rng(1000 + self.index)


WORKLOADS = {
    # molecule-like, plain FP64 parity case
    "m24": Workload("m24", 1, M=24, Nup=5, Ndn=5, Nchol=120, W=16, tau=0.005,
                    nsteps=50, k_qr=5),
    # single system, FP64 vs mixed precision
    "m128": Workload("m128", 2, M=128, Nup=32, Ndn=32, Nchol=640, W=512, tau=0.005,
                     nsteps=200, k_qr=10),
    # differentiation workload
    "m256": Workload("m256", 4, M=256, Nup=64, Ndn=64, Nchol=1280, W=256, tau=0.005,
                     nsteps=1, k_qr=5),
    # large solid-like system, the throughput workload
    "m512": Workload("m512", 5, M=512, Nup=128, Ndn=128, Nchol=2560, W=1024, tau=0.005,
                     nsteps=100, k_qr=5, decay=200.0, band=64),
}


def workload(name: str, **overrides) -> Workload:
    base = WORKLOADS[name]
    d = dict(base.__dict__)
    d.update(overrides)
    return Workload(**d)


def make_hamiltonian(M: int, Nchol: int, rng: np.random.Generator, *, decay: float = 20.0,
                     band: Optional[int] = None, reading: str = "R1"):
    """Return ``(h, L, E0)``: h [M, M] float64, L [Nchol, M, M] float64, E0 = 0."""
    if band is None:
        h = rng.normal(0.0, 0.1, size=(M, M))
        h = np.triu(h, 1)
        h = h + h.T
        h[np.diag_indices(M)] = rng.uniform(-2.0, 2.0, size=M)
    else:
        h = rng.normal(0.0, 0.2, size=(M, M))
        i, j = np.indices((M, M))
        h = np.where(np.abs(i - j) <= band, h, 0.0)
        h = np.triu(h)
        h = h + np.triu(h, 1).T
    iu = np.triu_indices(M)
    L = np.empty((Nchol, M, M))
    scale_r = 1.0 / np.sqrt(M) if reading == "R1" else 1.0
    for n in range(Nchol):
        a = np.zeros((M, M))
        a[iu] = rng.normal(0.0, 1.0, size=iu[0].size)
        a = a + np.triu(a, 1).T
        L[n] = a * (0.5 * np.exp(-n / decay) * scale_r)
    return np.ascontiguousarray(h), np.ascontiguousarray(L), 0.0


def make_trial(h: np.ndarray, Nup: int, Ndn: int):
    """Lowest eigenvectors of ``h`` for each spin, as complex128 [M, N] arrays."""
    _, v = np.linalg.eigh(h)
    return (np.ascontiguousarray(v[:, :Nup].astype(np.complex128)),
            np.ascontiguousarray(v[:, :Ndn].astype(np.complex128)))


def make_fields(nsteps: int, W: int, Nchol: int, seed: int = 0) -> np.ndarray:
    """Auxiliary fields ``x[step, walker, n] ~ N(0, 1)`` (float64)."""
    return np.random.default_rng(seed).standard_normal((nsteps, W, Nchol))


def make_random_walkers(M: int, N: int, W: int, seed: int) -> np.ndarray:
    """Complex Gaussian walker orbitals [W, M, N] with orthonormal columns."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((W, M, N)) + 1j * rng.standard_normal((W, M, N))
    q, _ = np.linalg.qr(z)
    return np.ascontiguousarray(q)


def make_thc(M: int, Nmu: int, rng: np.random.Generator, complex_orbitals: bool = False):
    """THC factors of Sec. V, Eq. (5): orbital values X [M, Nmu] at Nmu interpolating points,
    entries ~ N(0, 1/M) (complex: independent real and imaginary parts), and a positive
    semidefinite kernel Mmat = B B^T [Nmu, Nmu] with B ~ N(0, 0.5 / sqrt(Nmu)); X drawn first."""
    X = rng.normal(0.0, 1.0 / np.sqrt(M), size=(M, Nmu))
    if complex_orbitals:
        X = X + 1j * rng.normal(0.0, 1.0 / np.sqrt(M), size=(M, Nmu))
    B = rng.normal(0.0, 0.5 / np.sqrt(Nmu), size=(Nmu, Nmu))
    return X, B @ B.T


@dataclass
class UnevenSystem:
    M: int
    N: int
    Nchol: int
    W: int


def uneven_batch(n_systems: int = 64, seed: int = 1003) -> List[UnevenSystem]:
    """Sizes of the uneven multi-system batch: M ~ U{32..256}, N = floor(M/4),
    Nchol = 5 M, W ~ U{32..256}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_systems):
        M = int(rng.integers(32, 257))
        W = int(rng.integers(32, 257))
        out.append(UnevenSystem(M=M, N=M // 4, Nchol=5 * M, W=W))
    return out


def make_uneven_system(sysdims: UnevenSystem, index: int, seed: int = 1003, decay: float = 20.0,
                       reading: str = "R1"):
    """Hamiltonian and trial of system ``index`` of an uneven batch: the molecule-like
    generators above with ``default_rng([seed, index])``.  Returns ``(h, L, E0, Psi)``."""
    rng = np.random.default_rng([seed, index])
    h, L, E0 = make_hamiltonian(sysdims.M, sysdims.Nchol, rng, decay=decay, reading=reading)
    return h, L, E0, make_trial(h, sysdims.N, sysdims.N)
