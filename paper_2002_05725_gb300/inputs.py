"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws random numbers and nothing else: it holds none of the
method's arithmetic (no Jordan-Wigner map, no term table, no evolution).

* Couplings J_ijkl (Eq. 1): i.i.d. real Gaussian, mean 0, variance 6 J^2 / N^3,
  one value per quadruple i<j<k<l in lexicographic order (0-based).
* Random initial states |psi~> (Supp. Sec. I.C, "Disorder averaging"): every
  complex amplitude has independent standard-normal real and imaginary parts.
  The states live in one parity sector of dimension D = 2^(N/2-1) and are
  indexed by the compact sector index (the low N/2-1 bits of the spin basis
  index).

Seeding (numpy PCG64 via ``default_rng``):
* realization r of base seed b draws J from ``default_rng(b + 1000 r)``;
* state s of realization r draws its amplitudes from
  ``default_rng(b + 1000 r + 1 + s)`` as interleaved (re, im) pairs.
"""
from __future__ import annotations

import math

import numpy as np


def n_terms(N: int) -> int:
    """Number of couplings C(N, 4)."""
    return math.comb(N, 4)


def sector_dim(N: int) -> int:
    """Dimension 2^(N/2-1) of one fermion-parity sector."""
    return 1 << (N // 2 - 1)


def couplings(N: int, seed: int = 0, realization: int = 0, J: float = 1.0) -> np.ndarray:
    """C(N,4) float64 couplings with variance 6 J^2 / N^3 (Eq. 1)."""
    if N < 4 or N % 2:
        raise ValueError("N must be even and >= 4")
    rng = np.random.default_rng(seed + 1000 * realization)
    sigma = math.sqrt(6.0 * J * J / float(N) ** 3)
    return rng.normal(0.0, sigma, size=n_terms(N))


def random_states(N: int, nstates: int, seed: int = 0, realization: int = 0) -> np.ndarray:
    """(nstates, D) complex128 Gaussian random states in the compact sector index."""
    D = sector_dim(N)
    out = np.empty((nstates, D), dtype=np.complex128)
    for s in range(nstates):
        rng = np.random.default_rng(seed + 1000 * realization + 1 + s)
        ri = rng.standard_normal(2 * D)
        out[s] = ri[0::2] + 1j * ri[1::2]
    return out


def random_tridiagonal(m: int, seed: int = 0, scale: float = 1.0):
    """Random real symmetric tridiagonal (alpha[m], beta[m-1]) with beta > 0.

    Used only to exercise the tridiagonal exponential in isolation.
    """
    rng = np.random.default_rng(seed)
    alpha = rng.normal(0.0, scale, size=m)
    beta = np.abs(rng.normal(0.0, scale, size=max(m - 1, 0))) + 0.05 * scale
    return alpha, beta


def random_states_device(N: int, nstates: int, seed: int, device, dtype):
    """(D, nstates) Gaussian random states drawn directly in device memory.

    For sizes where a host draw is too slow (N >= 48).  Seeded by a torch
    generator on ``device``; real and imaginary parts are standard normal.
    """
    import torch
    D = sector_dim(N)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    real = torch.float32 if dtype == torch.complex64 else torch.float64
    out = torch.empty((D, nstates), dtype=dtype, device=device)
    v = torch.view_as_real(out)
    v.copy_(torch.randn(v.shape, generator=g, device=device, dtype=real))
    return out
