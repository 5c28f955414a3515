"""Finite-N G(tau) on the GPU against the large-N Schwinger-Dyson solution (a physics check)."""
import numpy as np
import pytest

from helpers import to_dev, torch_or_skip
from paper_2002_05725_gb300 import inputs, schwinger_dyson as sd, syk

pytestmark = pytest.mark.gpu


def test_G_tau_N32_close_to_large_N():
    """N = 32, beta J = 1, 2 draws x 16 states: the typicality estimate of G(tau) lies within
    6e-3 of the large-N solution (the 1/N correction is about 2.5e-3 here, the sampling error
    about 1e-3), and above it at beta/2, as the finite-N correction is at high temperature."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    N, beta = 32, 1.0
    taus = np.linspace(0.0, beta / 2, 6)
    num, den = np.zeros(len(taus)), 0.0
    for r in range(2):
        terms = syk.syk_build_terms(N, inputs.couplings(N, seed=1, realization=r))
        psi = to_dev(torch, inputs.random_states(N, 16, 1, r), "c64")
        G, Z = syk.syk_correlator_G_imag(terms, beta, 0, taus, psi, krylov_dim=40, tol=1e-8)
        num += np.real((G * Z[None, :]).sum(axis=1))
        den += float(np.sum(Z))
    gN = num / den
    ref = sd.solve(beta, 1.0, L=1 << 13).G(np.maximum(taus, 1e-12))
    assert np.abs(gN - ref).max() < 6e-3
    assert gN[-1] > ref[-1]
