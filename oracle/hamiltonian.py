"""The SYK Hamiltonian of Eq. 1 on the CPU, from the operator definitions.

H = sum_{i<j<k<l} J_ijkl chi_i chi_j chi_k chi_l   (Eq. 1)

Terms are indexed by quadruples i<j<k<l in lexicographic order (0-based).
Everything here applies the Majorana operators of ``jw`` one at a time to
basis states; no grouping, no sign tables.

Parity sector (Supp. Sec. I.A): H conserves the parity of the number of set
bits of the basis index.  Sector s holds the states with popcount(x) = s
(mod 2).  Its compact index c is the low n-1 bits of x; the top bit is
restored as x = c | ((popcount(c) + s) mod 2) << (n-1).  Compact order is
used for every sector vector.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

from .jw import chi_basis, chi_dense, popcount


def quadruples(N: int) -> np.ndarray:
    """(C(N,4), 4) int64 array of i<j<k<l in lexicographic order."""
    q = np.fromiter(itertools.chain.from_iterable(itertools.combinations(range(N), 4)),
                    dtype=np.int64, count=4 * math.comb(N, 4))
    return q.reshape(-1, 4)


def term_action(quads: np.ndarray, x):
    """chi_i chi_j chi_k chi_l |x> = amp |x_out> for every row (i,j,k,l) of ``quads``.

    The rightmost operator acts first.  ``x`` broadcasts against the rows.
    """
    amp = np.ones(np.broadcast(quads[:, 0], x).shape, dtype=np.complex128)
    cur = np.broadcast_to(np.asarray(x, dtype=np.int64), amp.shape)
    for col in (3, 2, 1, 0):
        a, cur = chi_basis(quads[:, col], cur)
        amp = amp * a
    return amp, cur


def flip_mask(quads: np.ndarray) -> np.ndarray:
    """Spins flipped by each term: chi_a flips spin floor(a/2)."""
    m = np.zeros(len(quads), dtype=np.int64)
    for col in range(4):
        m ^= np.int64(1) << (quads[:, col] // 2)
    return m


def term_table(N: int):
    """Pauli-string form of every term: 4 chi_i chi_j chi_k chi_l = i^p X^m Z^z.

    X^m Z^z |x> = (-1)^{popcount(z & x)} |x xor m>.  m, z and p are read off
    the action of the term on |0> and on each single-spin state |e_k>.
    Returns (m uint64, z uint64, p uint8) arrays in lexicographic term order.
    """
    n = N // 2
    q = quadruples(N)
    amp0, x0 = term_action(q, 0)
    ph = 4.0 * amp0                                   # = i^p exactly
    p = np.rint(np.angle(ph) / (np.pi / 2)).astype(np.int64) % 4
    if not np.allclose(ph, 1j ** p, atol=1e-12):
        raise AssertionError("term phase is not a power of i")
    ip = 1j ** p
    z = np.zeros(len(q), dtype=np.int64)
    for k in range(n):
        ak, xk = term_action(q, np.int64(1) << k)
        if not np.array_equal(xk, (np.int64(1) << k) ^ x0):
            raise AssertionError("flip mask differs between basis states")
        sgn = np.real(4.0 * ak / ip)
        if not np.allclose(np.abs(sgn), 1.0, atol=1e-12):
            raise AssertionError("term amplitude is not a signed phase")
        z |= (sgn < 0).astype(np.int64) << k
    return x0.astype(np.uint64), z.astype(np.uint64), p.astype(np.uint8)


# ----------------------------------------------------------------------------- sectors

def full_index(N: int, sector: int, c):
    """Spin basis index of compact index ``c`` in parity sector ``sector``."""
    n = N // 2
    c = np.asarray(c, dtype=np.int64)
    top = (popcount(c) + sector) & 1
    return c | (top << (n - 1))


def sector_of(x) -> np.ndarray:
    return popcount(x) & 1


# ----------------------------------------------------------------------------- H

def H_dense(N: int, J: np.ndarray) -> np.ndarray:
    """Full 2^n x 2^n matrix of Eq. 1 from dense Majorana matrices (N <= 14)."""
    chis = [chi_dense(N, i) for i in range(N)]
    H = np.zeros_like(chis[0])
    for t, (i, j, k, l) in enumerate(quadruples(N)):
        H += J[t] * (chis[i] @ chis[j] @ chis[k] @ chis[l])
    return H


def H_sector_sparse(N: int, J: np.ndarray, sector: int) -> sp.csr_matrix:
    """CSR matrix of H restricted to one parity sector, compact order.

    Column c is H applied to |full(c)>, summed term by term.
    """
    D = 1 << (N // 2 - 1)
    q = quadruples(N)
    cols = np.arange(D, dtype=np.int64)
    x = full_index(N, sector, cols)
    H = sp.csr_matrix((D, D), dtype=np.complex128)
    chunk = max(1, (1 << 22) // D)
    for t0 in range(0, len(q), chunk):
        qq = q[t0:t0 + chunk]
        amp, xo = _term_action_grid(qq, x)
        vals = (J[t0:t0 + chunk, None] * amp).ravel()
        rows = (xo & (D - 1)).ravel()
        cc = np.broadcast_to(cols[None, :], xo.shape).ravel()
        if np.any(sector_of(xo) != sector):
            raise AssertionError("a term left the parity sector")
        H = H + sp.csr_matrix((vals, (rows, cc)), shape=(D, D))
    H.sum_duplicates()
    return H


def _term_action_grid(qq: np.ndarray, x: np.ndarray):
    """term_action for every (term, state) pair: arrays of shape (len(qq), len(x))."""
    amp = np.ones((len(qq), len(x)), dtype=np.complex128)
    cur = np.broadcast_to(x[None, :], amp.shape).copy()
    for col in (3, 2, 1, 0):
        a, cur = chi_basis(qq[:, col][:, None], cur)
        amp = amp * a
    return amp, cur


def H_sector_dense(N: int, J: np.ndarray, sector: int) -> np.ndarray:
    return H_sector_sparse(N, J, sector).toarray()


def apply_rows(N: int, J: np.ndarray, sector: int, psi: np.ndarray, rows) -> np.ndarray:
    """Brute force (H psi)[c] for compact rows c: all C(N,4) terms, one row at a time.

    (H psi)[x] = sum_T J_T <x| P_T |x xor m_T> psi[x xor m_T], where P_T|x xor m_T>
    is evaluated by applying the four Majoranas to the basis state.  Works for
    any N (cost C(N,4) per row); ``psi`` has shape (D,) or (D, B).
    """
    D = 1 << (N // 2 - 1)
    q = quadruples(N)
    m = flip_mask(q)
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows),) + psi.shape[1:], dtype=np.complex128)
    for r, c in enumerate(rows):
        x = int(full_index(N, sector, c))
        src = np.int64(x) ^ m
        amp, xo = term_action(q, src)
        if not np.all(xo == x):
            raise AssertionError("flip mask mismatch")
        coef = J * amp
        vals = psi[src & (D - 1)]
        out[r] = np.tensordot(coef, vals, axes=(0, 0))
    return out


def chi_sector_sparse(N: int, i: int, sector_in: int) -> sp.csr_matrix:
    """chi_i as a D x D matrix from sector ``sector_in`` to the other sector."""
    D = 1 << (N // 2 - 1)
    c = np.arange(D, dtype=np.int64)
    x = full_index(N, sector_in, c)
    amp, xo = chi_basis(np.full(D, i, dtype=np.int64), x)
    if np.any(sector_of(xo) == sector_in):
        raise AssertionError("chi_i must flip the parity sector")
    return sp.csr_matrix((amp, (xo & (D - 1), c)), shape=(D, D))


def apply_chi(N: int, i: int, sector_in: int, psi: np.ndarray) -> np.ndarray:
    return chi_sector_sparse(N, i, sector_in) @ psi
