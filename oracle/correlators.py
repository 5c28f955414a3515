"""G(t) and the regularized OTOC F(t) from one random state (exact evolution).

Thermal averages are replaced by a random state |psi~> in the even parity
sector (Eq. q_typicality):

  Tr[O e^{-beta H}] ~ <psi~| e^{-beta H/2} O e^{-beta H/2} |psi~>.

G (Eq. G, real-time form):
  phi = e^{-beta H/2} psi~,
  G(t) = <phi| U(t)^dag chi_i U(t) chi_i |phi> / <phi|phi>,  U(t) = e^{-iHt};
  G_R(t) = 2 Re G(t).

F (Eq. F_reg, rho = e^{-beta H} split into four quarters), rearranged by
cyclicity of the trace to
  <psi~| rho^{1/8} chi_i(t) rho^{1/4} chi_j rho^{1/4} chi_i(t) rho^{1/4} chi_j rho^{1/8} |psi~>
and evaluated as a chain of states:
  phi = rho^{1/8} psi~,           a0 = rho^{1/4} chi_j phi,
  p   = chi_i U(t) phi,            q  = chi_i U(t) a0,
  r   = rho^{1/4} U(t)^dag p,      s  = rho^{1/4} U(t)^dag q,
  F(t) = <r| chi_j |s>,            F~(t) = F(t) / F(0).

chi flips the parity sector, so the chain alternates between the sectors.
Every evolution is computed from scratch by ``SectorSystem.expmv`` (exact),
never incrementally.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .evolve import SectorSystem
from .hamiltonian import H_dense, full_index
from .jw import chi_dense


def _dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """<a|b> per column (conjugating a)."""
    return np.sum(np.conj(a) * b, axis=0)


def G_state(sys: SectorSystem, beta: float, i: int, times, psi: np.ndarray):
    """Returns (G[nt(, B)], Z[(B)]) with Z = <phi|phi>, psi~ in the even sector."""
    phi = sys.expmv(-beta / 2.0, psi, 0)
    Z = np.real(_dot(phi, phi))
    b0 = sys.chi(i, 0, phi)
    out = []
    for t in times:
        a = sys.expmv(-1j * t, phi, 0)
        b = sys.expmv(-1j * t, b0, 1)
        out.append(_dot(a, sys.chi(i, 1, b)) / Z)
    return np.array(out), Z


def F_state(sys: SectorSystem, beta: float, i: int, j: int, times, psi: np.ndarray):
    """Unnormalised regularized OTOC F(t) for psi~ in the even sector."""
    phi = sys.expmv(-beta / 8.0, psi, 0)
    a0 = sys.expmv(-beta / 4.0, sys.chi(j, 0, phi), 1)
    out = []
    for t in times:
        p = sys.chi(i, 0, sys.expmv(-1j * t, phi, 0))        # odd sector
        q = sys.chi(i, 1, sys.expmv(-1j * t, a0, 1))         # even sector
        r = sys.expmv(-beta / 4.0, sys.expmv(1j * t, p, 1), 1)
        s = sys.expmv(-beta / 4.0, sys.expmv(1j * t, q, 0), 0)
        out.append(_dot(r, sys.chi(j, 0, s)))
    return np.array(out)


def F_state_split(sys: SectorSystem, beta: float, x, i: int, j: int, times, psi: np.ndarray):
    """OTOC with a general split of rho = e^{-beta H} between the operators:

      F(t) = Tr[W(t) rho^{x1} V rho^{x2} W(t) rho^{x3} V rho^{x4}],  x1+x2+x3+x4 = 1,

    W = chi_i, V = chi_j (x = 1/4 each: Eq. F_reg; x = (0, 0, 0, 1): the unregularized
    OTOC of Supp. Sec. unreg).  By cyclicity the one-state estimate (Eq. q_typicality) is
    <psi~| rho^{x4/2} W rho^{x1} V rho^{x2} W rho^{x3} V rho^{x4/2} |psi~> = <r|chi_j|s> with
      phi = rho^{x4/2} psi~,  a0 = rho^{x3} chi_j phi,
      r = rho^{x1} U^dag chi_i U phi,  s = rho^{x2} U^dag chi_i U a0.
    """
    x1, x2, x3, x4 = x
    phi = sys.expmv(-beta * x4 / 2.0, psi, 0)
    a0 = sys.expmv(-beta * x3, sys.chi(j, 0, phi), 1)
    out = []
    for t in times:
        p = sys.chi(i, 0, sys.expmv(-1j * t, phi, 0))
        q = sys.chi(i, 1, sys.expmv(-1j * t, a0, 1))
        r = sys.expmv(-beta * x1, sys.expmv(1j * t, p, 1), 1)
        s = sys.expmv(-beta * x2, sys.expmv(1j * t, q, 0), 0)
        out.append(_dot(r, sys.chi(j, 0, s)))
    return np.array(out)


def G_imag_state(sys: SectorSystem, beta: float, i: int, taus, psi: np.ndarray):
    """Imaginary-time G(tau) = <chi_i(tau) chi_i(0)>_beta (Eq. G), chi(tau) = e^{tau H} chi e^{-tau H},
    estimated as <psi~|e^{-beta H/2} chi_i(tau) chi_i e^{-beta H/2}|psi~> / <psi~|e^{-beta H}|psi~>
    (Eq. q_typicality).  Returns (G[ntau(, B)], Z)."""
    x = sys.expmv(-beta / 2.0, psi, 0)
    Z = np.real(_dot(x, x))
    out = []
    for tau in taus:
        w = sys.expmv(tau, x, 0)                                  # e^{(tau - beta/2) H} psi~
        y = sys.expmv(-tau, sys.chi(i, 0, x), 1)                  # e^{-tau H} chi_i x
        out.append(_dot(w, sys.chi(i, 1, y)) / Z)
    return np.array(out), Z


def G_imag_trace_even(N: int, J: np.ndarray, beta: float, i: int, taus):
    """Tr[P_e e^{-beta H} chi_i(tau) chi_i] / Tr[P_e e^{-beta H}] from full dense matrices."""
    H = H_dense(N, J)
    Pe = _even_projector_full(N)
    c = chi_dense(N, i)
    R = sla.expm(-beta * H)
    Z = np.trace(Pe @ R).real
    out = []
    for tau in taus:
        ct = sla.expm(tau * H) @ c @ sla.expm(-tau * H)
        out.append(np.trace(Pe @ sla.expm(-beta / 2 * H) @ ct @ c @ sla.expm(-beta / 2 * H)) / Z)
    return np.array(out)


def F_trace_split(N: int, J: np.ndarray, beta: float, x, i: int, j: int, times, sector=0):
    """Tr[P rho^{x4/2} W(t) rho^{x1} V rho^{x2} W(t) rho^{x3} V rho^{x4/2}] (dense; P: sector projector)."""
    H = H_dense(N, J)
    P = _even_projector_full(N, sector)
    W0 = chi_dense(N, i)
    V = chi_dense(N, j)
    rr = [sla.expm(-beta * xk * H) for xk in x]
    rh = sla.expm(-beta * x[3] / 2 * H)
    out = []
    for t in times:
        U = sla.expm(-1j * t * H)
        W = U.conj().T @ W0 @ U
        out.append(np.trace(P @ rh @ W @ rr[0] @ V @ rr[1] @ W @ rr[2] @ V @ rh))
    return np.array(out)


# ----------------------------------------------------------------------------- traces

def _even_projector_full(N: int, sector=0) -> np.ndarray:
    """Projector on one parity sector of the full space (identity if sector is None)."""
    n = N // 2
    if sector is None:
        return np.eye(1 << n, dtype=np.complex128)
    x = np.arange(1 << n)
    par = np.array([bin(v).count("1") & 1 for v in x])
    return np.diag((par == sector).astype(np.complex128))


def G_trace_even(N: int, J: np.ndarray, beta: float, i: int, times):
    """Tr[P_e e^{-bH/2} chi_i(t) chi_i e^{-bH/2}] / Tr[P_e e^{-bH}] from full dense matrices.

    P_e projects on the even sector; this is what the state estimate averages
    to over a basis of that sector.
    """
    H = H_dense(N, J)
    Pe = _even_projector_full(N)
    c = chi_dense(N, i)
    R = sla.expm(-beta / 2.0 * H)
    Z = np.trace(Pe @ R @ R).real
    out = []
    for t in times:
        U = sla.expm(-1j * t * H)
        W = U.conj().T @ c @ U
        out.append(np.trace(Pe @ R @ W @ c @ R) / Z)
    return np.array(out)


def F_trace_even(N: int, J: np.ndarray, beta: float, i: int, j: int, times, sector=0):
    """Tr[P_e rho^{1/8} W(t) rho^{1/4} V rho^{1/4} W(t) rho^{1/4} V rho^{1/8}] (unnormalised).

    ``sector=None`` drops the projector (full trace of Eq. F_reg).
    """
    H = H_dense(N, J)
    Pe = _even_projector_full(N, sector)
    W0 = chi_dense(N, i)
    V = chi_dense(N, j)
    r8 = sla.expm(-beta / 8.0 * H)
    r4 = sla.expm(-beta / 4.0 * H)
    out = []
    for t in times:
        U = sla.expm(-1j * t * H)
        W = U.conj().T @ W0 @ U
        out.append(np.trace(Pe @ r8 @ W @ r4 @ V @ r4 @ W @ r4 @ V @ r8))
    return np.array(out)


def basis_states_even(N: int) -> np.ndarray:
    """Identity matrix of the even sector (columns = compact basis states)."""
    D = 1 << (N // 2 - 1)
    return np.eye(D, dtype=np.complex128)


def compact_to_full(N: int, sector: int) -> np.ndarray:
    D = 1 << (N // 2 - 1)
    return full_index(N, sector, np.arange(D))
