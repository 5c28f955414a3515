"""Majorana operators from the Jordan-Wigner map (Supp. Sec. I.A).

chi_i = (1/sqrt 2) (prod_{j<k} sigma^z_j) sigma^x_k   for even i,
chi_i = (1/sqrt 2) (prod_{j<k} sigma^z_j) sigma^y_k   for odd i,
with k = floor(i/2), 0 <= i < N, on n = N/2 spins.

The 1/sqrt 2 is not written in the map itself; it is what the normalisation
{chi_i, chi_j} = delta_ij of Eq. 1 requires (checked by the pins).
Spin k is bit k of the basis index (least significant bit = spin 0); a set
bit means sigma^z = -1.
"""
from __future__ import annotations

import numpy as np

SQRT_HALF = 1.0 / np.sqrt(2.0)

I2 = np.eye(2, dtype=np.complex128)
SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def popcount(a):
    """Bit count of a non-negative integer array."""
    a = np.asarray(a, dtype=np.uint64)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    out = np.zeros(a.shape, dtype=np.int64)
    b = a.copy()
    while np.any(b):
        out += (b & np.uint64(1)).astype(np.int64)
        b >>= np.uint64(1)
    return out


def chi_dense(N: int, i: int) -> np.ndarray:
    """Dense 2^n x 2^n matrix of chi_i (small N only)."""
    n = N // 2
    k = i // 2
    ops = [I2] * n
    for j in range(k):
        ops[j] = SZ
    ops[k] = SX if i % 2 == 0 else SY
    # numpy's kron puts the last factor on the fastest index, i.e. bit 0
    M = np.ones((1, 1), dtype=np.complex128)
    for j in reversed(range(n)):
        M = np.kron(M, ops[j])
    return SQRT_HALF * M


def chi_basis(i, x):
    """Action of chi_i on basis states: chi_i |x> = amp |x_out>.

    ``i`` and ``x`` broadcast against each other (integer arrays).  Returns
    (amp complex128, x_out int64).
    """
    i = np.asarray(i, dtype=np.int64)
    x = np.asarray(x, dtype=np.int64)
    k = i // 2
    bit = (x >> k) & 1
    below = x & ((np.int64(1) << k) - 1)
    sign = 1.0 - 2.0 * (popcount(below) & 1)            # Z string on spins j < k
    odd = (i & 1).astype(bool)
    # sigma^y |0> = i |1>,  sigma^y |1> = -i |0>;  sigma^x has amplitude 1
    yfac = np.where(bit == 0, 1j, -1j)
    amp = sign * np.where(odd, yfac, 1.0 + 0j) * SQRT_HALF
    x_out = x ^ (np.int64(1) << k)
    return amp.astype(np.complex128), x_out
