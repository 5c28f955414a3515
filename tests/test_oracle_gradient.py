"""Pins of the oracle gradient (Daleckii-Krein) to closed forms and finite differences."""
import numpy as np
import pytest

from oracle import correlators as co, evolve, gradient as gr
from paper_2002_05725_gb300 import inputs


@pytest.mark.parametrize("beta", [0.0, 2.5])
def test_N4_closed_forms(beta):
    """N=4, even sector: F~(t) = e^{-iJt} and G(t) = e^{-iJt/2}/2 for every beta, so
    dF~/dJ = -it e^{-iJt}, dG/dJ = -(it/4) e^{-iJt/2} and both beta derivatives vanish."""
    Jv, t = 0.8, 1.7
    psi = inputs.random_states(4, 2, 3).T
    Ft, dF, bF = gr.otoc_tilde_grad(4, np.array([Jv]), beta, 0, 1, t, psi)
    assert np.allclose(Ft, np.exp(-1j * Jv * t), atol=1e-14)
    assert np.allclose(dF[0], -1j * t * np.exp(-1j * Jv * t), atol=1e-12)
    assert np.allclose(bF, 0, atol=1e-12)
    G, dG, bG = gr.g_grad(4, np.array([Jv]), beta, 0, t, psi)
    assert np.allclose(G, 0.5 * np.exp(-0.5j * Jv * t), atol=1e-14)
    assert np.allclose(dG[0], -0.25j * t * np.exp(-0.5j * Jv * t), atol=1e-12)
    assert np.allclose(bG, 0, atol=1e-12)


def test_value_matches_correlator_oracle():
    N = 8
    J = inputs.couplings(N, 4) * 2.0
    psi = inputs.random_states(N, 2, 1).T
    sysm = evolve.SectorSystem(N, J)
    Ft, _, _ = gr.otoc_tilde_grad(N, J, 3.0, 1, 5, 2.0, psi, terms=[0])
    F = co.F_state(sysm, 3.0, 1, 5, [0.0, 2.0], psi)
    assert np.abs(Ft - F[1] / F[0]).max() < 1e-13
    G, _, _ = gr.g_grad(N, J, 3.0, 2, 1.5, psi, terms=[0])
    Gref, _ = co.G_state(sysm, 3.0, 2, [1.5], psi)
    assert np.abs(G - Gref[0]).max() < 1e-13


def test_daleckii_krein_vs_finite_differences():
    N = 8
    J = inputs.couplings(N, 9) * 2.0
    psi = inputs.random_states(N, 1, 6).T
    beta, t, i, j = 2.0, 1.3, 0, 3
    terms = list(range(0, 70, 3))
    _, dF, bF = gr.otoc_tilde_grad(N, J, beta, i, j, t, psi, terms=terms)

    def Ftil(Jx, b):
        return gr.otoc_tilde_grad(N, Jx, b, i, j, t, psi, terms=[0])[0]

    fdJ, fdb = gr.fd_grad(Ftil, J, beta, terms)
    scale = np.abs(dF).max()
    assert np.abs(dF - fdJ).max() < 1e-7 * scale
    assert np.abs(bF - fdb).max() < 1e-7 * max(scale, np.abs(bF).max())
    _, dG, bG = gr.g_grad(N, J, beta, i, t, psi, terms=terms)

    def Gf(Jx, b):
        return gr.g_grad(N, Jx, b, i, t, psi, terms=[0])[0]

    fdJ, fdb = gr.fd_grad(Gf, J, beta, terms)
    assert np.abs(dG - fdJ).max() < 1e-7 * np.abs(dG).max()
    assert np.abs(bG - fdb).max() < 1e-7 * max(np.abs(dG).max(), np.abs(bG).max())
