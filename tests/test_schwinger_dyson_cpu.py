"""Large-N Schwinger-Dyson solver (host code) against limits it must reproduce."""
import numpy as np
import pytest

from paper_2002_05725_gb300 import schwinger_dyson as sd


def test_free_limit():
    """J = 0: a free Majorana, G(tau) = 1/2 on (0, beta)."""
    s = sd.solve(2.0, 0.0, L=1 << 10)
    assert np.abs(s.G(np.linspace(0.05, 1.95, 7)) - 0.5).max() < 1e-15


def test_second_order_in_J():
    """To order J^2, Sigma = J^2/8 on (0, beta); d G1/d tau = (Sigma * G0)(tau) = (J^2/16)(2 tau - beta)
    with G1(0+) + G1(beta-) = 0 gives G = 1/2 - (J^2/16) tau (beta - tau); the next order is J^4."""
    beta, J = 1.0, 0.1
    s = sd.solve(beta, J, L=1 << 12)
    tau = np.linspace(0.05, 0.95, 10)
    assert np.abs(s.G(tau) - (0.5 - J * J / 16 * tau * (beta - tau))).max() < 1e-6


def test_grid_convergence_and_symmetry():
    a, b = sd.solve(5.0, 1.0, L=1 << 12), sd.solve(5.0, 1.0, L=1 << 14)
    tau = np.linspace(0.1, 4.9, 9)
    assert np.abs(a.G(tau) - b.G(tau)).max() < 1e-9
    assert np.abs(b.G(tau) - b.G(5.0 - tau)).max() < 1e-14  # G(beta - tau) = G(tau)
    assert np.all(np.diff(b.G(np.linspace(0.1, 2.5, 9))) < 0)  # decreasing towards beta/2


def test_conformal_limit_approach():
    """At beta J >> 1 the solution approaches the conformal form (Eq. conformal) with a relative
    gap at tau = beta/2 that falls like 1/(beta J)."""
    gaps = []
    for bJ in (25.0, 50.0, 100.0):
        s = sd.solve(bJ, 1.0, L=1 << 14)
        gaps.append(1.0 - s.G(bJ / 2)[0] / float(sd.conformal(bJ / 2, bJ)))
    gaps = np.array(gaps)
    assert np.all(gaps > 0) and gaps[-1] < 0.01
    assert np.allclose(gaps[:-1] / gaps[1:], 2.0, rtol=0.1)


def test_invalid():
    with pytest.raises(ValueError):
        sd.solve(-1.0)
    with pytest.raises(ValueError):
        sd.solve(1.0, 1.0, L=7)
