"""Exact sector evolution e^{zH} psi and the tridiagonal exponential.

The paper's Krylov method (Supp. Sec. I.B) approximates e^{-iHt}|psi>; the
oracle computes the exact quantity instead:

* D <= DENSE_MAX: eigendecomposition H_s = V diag(w) V^dagger, then
  e^{zH} psi = V e^{z w} V^dagger psi (z complex: -i t for real time,
  -tau for imaginary time).
* larger sectors: scipy.sparse.linalg.expm_multiply (Al-Mohy & Higham) on the
  CSR matrix of the sector.

``tridiag_expm_e1`` is the m x m step the Krylov method needs: for the
real symmetric tridiagonal T (alpha on the diagonal, beta off it) it returns
beta0 * e^{zT} e_1 by scipy.linalg.expm.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .hamiltonian import H_sector_sparse, chi_sector_sparse

DENSE_MAX = 4096


class SectorSystem:
    """H of one coupling draw, restricted to both parity sectors, plus chi_i."""

    def __init__(self, N: int, J: np.ndarray, dense_max: int = DENSE_MAX):
        self.N = N
        self.J = np.asarray(J, dtype=np.float64)
        self.D = 1 << (N // 2 - 1)
        self.dense = self.D <= dense_max
        self._H = {}
        self._eig = {}
        self._chi = {}

    def H(self, sector: int):
        if sector not in self._H:
            self._H[sector] = H_sector_sparse(self.N, self.J, sector)
        return self._H[sector]

    def eig(self, sector: int):
        if sector not in self._eig:
            self._eig[sector] = np.linalg.eigh(self.H(sector).toarray())
        return self._eig[sector]

    def chi(self, i: int, sector_in: int, psi: np.ndarray) -> np.ndarray:
        key = (i, sector_in)
        if key not in self._chi:
            self._chi[key] = chi_sector_sparse(self.N, i, sector_in)
        return self._chi[key] @ psi

    def apply_H(self, sector: int, psi: np.ndarray) -> np.ndarray:
        return self.H(sector) @ psi

    def expmv(self, z: complex, psi: np.ndarray, sector: int) -> np.ndarray:
        """e^{z H_s} psi, psi of shape (D,) or (D, B)."""
        if z == 0:
            return np.array(psi, dtype=np.complex128, copy=True)
        if self.dense:
            w, V = self.eig(sector)
            c = V.conj().T @ psi
            f = np.exp(z * w)
            c = c * (f[:, None] if c.ndim == 2 else f)
            return V @ c
        A = self.H(sector) * z
        return spla.expm_multiply(A, psi)


def tridiag_expm_e1(alpha: np.ndarray, beta: np.ndarray, z: complex, beta0: float = 1.0):
    """beta0 * e^{zT} e_1 for T = tridiag(beta, alpha, beta) (real symmetric)."""
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64)).astype(np.complex128)
    if m > 1:
        T += np.diag(beta[: m - 1], 1) + np.diag(beta[: m - 1], -1)
    E = sla.expm(z * T)
    return beta0 * E[:, 0]
