"""Large-N imaginary-time Green's function of the SYK model from the Schwinger-Dyson equations
(Supp. Sec. "Schwinger-Dyson equations", Eq. SD), as a physics cross-check of the finite-N
G(tau) that `syk.syk_correlator_G_imag` computes on the GPU.

Equations, with G(tau) = <chi(tau) chi(0)>_beta (G(0+) = 1/2 for {chi_i, chi_j} = delta_ij),
couplings of variance 6 J^2 / N^3 and fermionic frequencies omega_n = pi (2n + 1) / beta:

    G(i omega_n) = 1 / (-i omega_n - Sigma(i omega_n)),    Sigma(tau) = J^2 G(tau)^3,
    F(i omega_n) = int_0^beta d tau e^{i omega_n tau} F(tau).

Reading: the paper writes 1/G = i omega + Sigma. That is the same system under the opposite
Fourier sign, or for G of opposite sign. The convention here is the one whose free limit is
G(tau) = 1/2 on (0, beta).

Numerics: L midpoints tau_j = (j + 1/2) beta / L and L frequencies, so the transforms are FFTs.
The jumps at tau = 0 are taken out analytically, because the antiperiodic step s(tau) = 1/2 on
(0, beta) has the transform -1/(i omega_n):
* G = s + g: only g, whose transform decays like omega^-3, goes through the FFT.
* Sigma = 2 Sigma(0+) s + r, with r(0+) = r(beta-) = 0: only r goes through the FFT.
The fixed point is reached by the damped iteration G <- (1 - x) G + x G_new. The damping x is
halved whenever the change grows, as commonly done for these equations.

Running the module (`python -m paper_2002_05725_gb300.schwinger_dyson`) solves the equations at
one beta J. It computes the finite-N G(tau) of several N on the GPU and prints one JSON line with
the deviation of each N from the large-N solution.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np


class SDSolution:
    """Converged solution on an L-point grid: G_iw (L Matsubara values, n = -L/2 .. L/2-1)."""

    def __init__(self, beta, J, L, G_iw, iterations, residual):
        self.beta, self.J, self.L = float(beta), float(J), int(L)
        self.G_iw = G_iw
        self.iterations, self.residual = iterations, residual
        n = np.arange(-L // 2, L // 2)
        self.omega = math.pi * (2 * n + 1) / self.beta

    def G(self, tau) -> np.ndarray:
        """G(tau) for 0 < tau < beta: 1/2 + (1/beta) sum_n [G(i w_n) + 1/(i w_n)] e^{-i w_n tau}."""
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        rem = self.G_iw + 1.0 / (1j * self.omega)
        ph = np.exp(-1j * np.outer(tau, self.omega))
        return 0.5 + np.real(ph @ rem) / self.beta


def _grid(beta, L):
    j = np.arange(L)
    n = np.arange(-L // 2, L // 2)
    w = math.pi * (2 * n + 1) / beta
    return j, n, w


def _to_freq(f_tau, beta, L):
    """F(i w_n) = (beta/L) sum_j f(tau_j) e^{i w_n tau_j} for n = -L/2 .. L/2-1 (midpoint rule)."""
    j, n, _ = _grid(beta, L)
    a = np.fft.ifft(f_tau * np.exp(1j * math.pi * j / L)) * L  # sum_j (.) e^{+2 pi i n j / L}
    return (beta / L) * np.exp(1j * math.pi * (2 * n + 1) / (2 * L)) * a[n % L]


def _to_time(F_iw, beta, L):
    """f(tau_j) = (1/beta) sum_n F(i w_n) e^{-i w_n tau_j} over the L frequencies."""
    j, n, _ = _grid(beta, L)
    b = np.zeros(L, dtype=complex)
    b[n % L] = F_iw * np.exp(-1j * math.pi * (2 * n + 1) / (2 * L))
    return np.exp(-1j * math.pi * j / L) * np.fft.fft(b) / beta


def solve(beta: float, J: float = 1.0, L: int = 1 << 14, tol: float = 1e-13, max_iter: int = 10000,
          mix: float = 0.5) -> SDSolution:
    """Solves the Schwinger-Dyson equations at inverse temperature beta and coupling J."""
    if not (beta > 0.0) or J < 0.0 or L < 8 or L % 2:
        raise ValueError("need beta > 0, J >= 0 and an even L >= 8")
    _, _, w = _grid(beta, L)
    G0_iw = -1.0 / (1j * w)
    G_tau = np.full(L, 0.5)
    prev = math.inf
    x = mix
    for it in range(1, max_iter + 1):
        sig = J * J * G_tau ** 3
        s0 = J * J / 8.0  # Sigma(0+) = J^2 G(0+)^3, G(0+) = 1/2
        Sig_iw = -2.0 * s0 / (1j * w) + _to_freq(sig - s0, beta, L)
        G_iw = 1.0 / (-1j * w - Sig_iw)
        G_new = 0.5 + np.real(_to_time(G_iw - G0_iw, beta, L))
        diff = float(np.max(np.abs(G_new - G_tau)))
        if diff > prev:
            x *= 0.5
        prev = diff
        G_tau = (1.0 - x) * G_tau + x * G_new
        if diff < tol:
            return SDSolution(beta, J, L, G_iw, it, diff)
    raise RuntimeError(f"Schwinger-Dyson iteration did not converge in {max_iter} steps (last change {diff:.3e})")


def conformal(tau, beta, J=1.0):
    """Conformal limit (Eq. conformal): b [pi / (beta J sin(pi tau / beta))]^{1/2},
    b = 1/(sqrt(2) pi^{1/4}), J restored by dimensional analysis."""
    tau = np.asarray(tau, dtype=np.float64)
    b = 1.0 / (math.sqrt(2.0) * math.pi ** 0.25)
    return b * np.sqrt(math.pi / (beta * J * np.sin(math.pi * tau / beta)))


def main():
    import argparse

    import torch

    from . import inputs, syk
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--beta", type=float, default=5.0)
    ap.add_argument("--N", default="20,24,28,32,36,40")
    ap.add_argument("--states", type=int, default=16)
    ap.add_argument("--draws", type=int, default=2)
    ap.add_argument("--ntau", type=int, default=11)
    ap.add_argument("--L", type=int, default=1 << 14)
    a = ap.parse_args()
    t0 = time.perf_counter()
    sd = solve(a.beta, 1.0, a.L)
    sd_s = time.perf_counter() - t0
    taus = np.linspace(0.0, a.beta / 2, a.ntau)
    g_sd = sd.G(np.where(taus == 0.0, 1e-12, taus))
    g_sd[taus == 0.0] = 0.5
    syk.load()
    out = {"beta_J": a.beta, "tau": taus.tolist(), "G_sd": g_sd.tolist(), "sd_iterations": sd.iterations,
           "sd_seconds": sd_s, "L": a.L, "finite_N": {}}
    for N in [int(v) for v in a.N.split(",")]:
        num = np.zeros(len(taus))
        den = 0.0
        t1 = time.perf_counter()
        for r in range(a.draws):
            terms = syk.syk_build_terms(N, inputs.couplings(N, seed=0, realization=r))
            psi = torch.from_numpy(np.ascontiguousarray(inputs.random_states(N, a.states, 0, r).T)).to(
                torch.complex64).cuda()
            G, Z = syk.syk_correlator_G_imag(terms, a.beta, 0, taus, psi, krylov_dim=40, tol=1e-8)
            # typicality over states and draws: ratio of summed numerators and partition sums
            num += np.real((G * Z[None, :]).sum(axis=1))
            den += float(np.sum(Z))
        gN = num / den
        out["finite_N"][str(N)] = {"G": gN.tolist(), "max_dev": float(np.max(np.abs(gN - g_sd))),
                                   "dev_half_beta": float(gN[-1] - g_sd[-1]), "seconds": time.perf_counter() - t1}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
