"""Exact derivatives of the one-state correlators with respect to the couplings and beta.

TEST INFRASTRUCTURE (CPU oracle, small N: dense sector matrices).

Both correlators are sesquilinear forms F = <a|b> of two chains of operators
applied to the random state psi~ (Eq. F_reg, Eq. G with Eq. q_typicality):

  F (regularized OTOC): a = R U^dag chi_i U R8 psi~,
                        b = chi_j R U^dag chi_i U R chi_j R8 psi~,
  G numerator:          a = U R2 psi~,    b = chi_i U chi_i R2 psi~,
  Z = <R2 psi~|R2 psi~>,

with U = e^{-iHt}, R8 = e^{-beta H/8}, R = e^{-beta H/4}, R2 = e^{-beta H/2}.
The derivative of every exponential e^{zH} in the direction E = dH/dJ_T =
chi_i chi_j chi_k chi_l (Eq. 1) is the Daleckii-Krein formula in the
eigenbasis H = V diag(w) V^dag:

  D e^{zH}[E] = V (L o (V^dag E V)) V^dag,
  L_ab = (e^{z w_a} - e^{z w_b}) / (w_a - w_b)   (z e^{z w_a} if w_a = w_b),

and dF = <da|b> + <a|db> with d(M_K ... M_1) = sum_k M_K .. dM_k .. M_1.
For beta: d e^{-c beta H}/d beta = -c H e^{-c beta H}.
``*_fd`` are central finite differences of the exact correlators (pins).
"""
from __future__ import annotations

import numpy as np

from .evolve import SectorSystem
from .hamiltonian import _term_action_grid, full_index, quadruples


def term_sector_matrix(N: int, q: np.ndarray, sector: int) -> np.ndarray:
    """Dense D x D matrix of chi_i chi_j chi_k chi_l (rows of q) on one parity sector."""
    D = 1 << (N // 2 - 1)
    x = full_index(N, sector, np.arange(D, dtype=np.int64))
    amp, xo = _term_action_grid(q[None, :], x)
    P = np.zeros((D, D), dtype=np.complex128)
    P[xo[0] & (D - 1), np.arange(D)] = amp[0]
    return P


class ChainGrad:
    """Dense evaluation of <a|b> and its gradient for chains of exp / chi operators.

    An op is ("exp", c_beta, c_time) meaning e^{z H} with z = -c_beta*beta - 1j*c_time*t,
    or ("chi", i).  The sector of the input of every op is tracked from sector 0.
    """

    def __init__(self, N: int, J: np.ndarray, beta: float, t: float):
        self.N, self.J, self.beta, self.t = N, np.asarray(J, float), beta, t
        self.sys = SectorSystem(N, self.J)
        self.q = quadruples(N)
        self.eig = {s: self.sys.eig(s) for s in (0, 1)}
        self.Hd = {s: self.sys.H(s).toarray() for s in (0, 1)}
        self._P = {}

    def P(self, T: int, s: int) -> np.ndarray:
        key = (T, s)
        if key not in self._P:
            self._P[key] = term_sector_matrix(self.N, self.q[T], s)
        return self._P[key]

    def z(self, op):
        return -op[1] * self.beta - 1j * op[2] * self.t

    def apply(self, op, s, v):
        if op[0] == "chi":
            return self.sys.chi(op[1], s, v), 1 - s
        w, V = self.eig[s]
        z = self.z(op)
        return V @ (np.exp(z * w)[:, None] * (V.conj().T @ v)), s

    def forward(self, ops, psi):
        xs, ss = [psi], [0]
        for op in ops:
            v, s = self.apply(op, ss[-1], xs[-1])
            xs.append(v)
            ss.append(s)
        return xs, ss

    def adjoint(self, op, s_in, v):
        """M^dag v for op M acting on sector s_in (v lives in the output sector)."""
        if op[0] == "chi":
            return self.sys.chi(op[1], 1 - s_in, v)
        w, V = self.eig[s_in]
        z = np.conj(self.z(op))
        return V @ (np.exp(z * w)[:, None] * (V.conj().T @ v))

    def _dexp(self, op, s, E):
        w, V = self.eig[s]
        z = self.z(op)
        f = np.exp(z * w)
        dw = w[:, None] - w[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            L = (f[:, None] - f[None, :]) / dw
        same = np.abs(dw) < 1e-13 * max(1.0, np.abs(w).max())
        L[same] = (z * np.broadcast_to(f[:, None], L.shape))[same]
        return V @ (L * (V.conj().T @ E @ V)) @ V.conj().T

    def grad_side(self, ops, psi, left, terms):
        """sum over exp factors of <lam_k| dM_k x_{k-1}> for every term and d/dbeta."""
        xs, ss = self.forward(ops, psi)
        lam = left
        gJ = np.zeros((len(terms),) + psi.shape[1:], dtype=np.complex128)
        gb = np.zeros(psi.shape[1:], dtype=np.complex128)
        for k in range(len(ops) - 1, -1, -1):
            op, s = ops[k], ss[k]
            if op[0] == "exp":
                for n, T in enumerate(terms):
                    dM = self._dexp(op, s, self.P(T, s))
                    gJ[n] += np.sum(np.conj(lam) * (dM @ xs[k]), axis=0)
                if op[1] != 0:
                    gb += np.sum(np.conj(lam) * (-op[1]) * (self.Hd[s] @ xs[k + 1]), axis=0)
            lam = self.adjoint(op, s, lam)
        return gJ, gb

    def value_grad(self, opsA, opsB, psi, terms):
        """(<a|b>, d<a|b>/dJ_T for T in terms, d<a|b>/dbeta) per column of psi."""
        a = self.forward(opsA, psi)[0][-1]
        b = self.forward(opsB, psi)[0][-1]
        val = np.sum(np.conj(a) * b, axis=0)
        gJ_b, gb_b = self.grad_side(opsB, psi, a, terms)      # <a|db>
        gJ_a, gb_a = self.grad_side(opsA, psi, b, terms)      # <b|da> = conj(<da|b>)
        return val, gJ_b + np.conj(gJ_a), gb_b + np.conj(gb_a)


def otoc_ops(i: int, j: int):
    """Chains of the regularized OTOC F(t) = <a|b> (evaluated at time t)."""
    A = [("exp", 1 / 8, 0.0), ("exp", 0.0, 1.0), ("chi", i), ("exp", 0.0, -1.0), ("exp", 1 / 4, 0.0)]
    B = [("exp", 1 / 8, 0.0), ("chi", j), ("exp", 1 / 4, 0.0), ("exp", 0.0, 1.0), ("chi", i), ("exp", 0.0, -1.0),
         ("exp", 1 / 4, 0.0), ("chi", j)]
    return A, B


def g_ops(i: int):
    """Chains of the G numerator <a|b> and of Z = <phi|phi>."""
    A = [("exp", 1 / 2, 0.0), ("exp", 0.0, 1.0)]
    B = [("exp", 1 / 2, 0.0), ("chi", i), ("exp", 0.0, 1.0), ("chi", i)]
    Z = [("exp", 1 / 2, 0.0)]
    return A, B, Z


def otoc_tilde_grad(N, J, beta, i, j, t, psi, terms=None):
    """F~(t) = F(t)/F(0) per state and its gradient (dJ for `terms`, dbeta)."""
    terms = np.arange(len(quadruples(N))) if terms is None else np.asarray(terms)
    A, B = otoc_ops(i, j)
    Ft, dFt, bFt = ChainGrad(N, J, beta, t).value_grad(A, B, psi, terms)
    F0, dF0, bF0 = ChainGrad(N, J, beta, 0.0).value_grad(A, B, psi, terms)
    Ftil = Ft / F0
    return Ftil, (dFt - Ftil * dF0) / F0, (bFt - Ftil * bF0) / F0


def g_grad(N, J, beta, i, t, psi, terms=None):
    """G(t) = <a|b>/Z per state and its gradient (dJ for `terms`, dbeta)."""
    terms = np.arange(len(quadruples(N))) if terms is None else np.asarray(terms)
    A, B, Zc = g_ops(i)
    cg = ChainGrad(N, J, beta, t)
    num, dnum, bnum = cg.value_grad(A, B, psi, terms)
    Z, dZ, bZ = cg.value_grad(Zc, Zc, psi, terms)
    G = num / Z
    return G, (dnum - G * dZ) / Z, (bnum - G * bZ) / Z


def fd_grad(fun, J, beta, terms, h=1e-6):
    """Central differences of fun(J, beta) w.r.t. J_T (T in terms) and beta."""
    J = np.asarray(J, float)
    out = []
    for T in terms:
        Jp, Jm = J.copy(), J.copy()
        Jp[T] += h
        Jm[T] -= h
        out.append((fun(Jp, beta) - fun(Jm, beta)) / (2 * h))
    db = (fun(J, beta + h) - fun(J, beta - h)) / (2 * h)
    return np.array(out), db
