"""Correlator chains run with the Krylov step control on the device (syk_use_graphs(2): each
evolution one CUDA graph launch with conditional WHILE/IF nodes, no host synchronisation
until the chain ends) against the same chains driven from the host (graphs off, and the
default segment graphs): the kernels, convergence checks
and accepted steps are the same, so the results are bit-identical and the work counters
agree.  The benchmark's shapes: N = 24 with 16 and 8 states (complex64, coset matvec) and 2
states (complex128, double-float matvec); plus the exact oracle for the device-driven curves.
"""
import numpy as np
import pytest

from helpers import TOL, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu

N = 24
T_GRID = np.round(np.linspace(0.0, 12.0, 5), 12)


@pytest.fixture(scope="module")
def setup():
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    J = inputs.couplings(N, 9)
    psi = inputs.random_states(N, 16, 9)
    return torch, syk.syk_build_terms(N, J), J, psi


def _run(fn, mode):
    syk.syk_use_graphs(mode)
    try:
        syk.syk_counters(reset=True)
        syk.syk_matvec_launches(reset=True)
        out = fn()
        return out, syk.syk_counters(reset=True), syk.syk_matvec_launches(reset=True)
    finally:
        syk.syk_use_graphs(syk.GRAPHS_SEGMENTS)


@pytest.mark.parametrize("dt,B", [("c64", 16), ("c64", 8), ("c128", 2)])
def test_device_driven_chains_match_host_driven(setup, dt, B):
    torch, terms, J, psi = setup
    x = to_dev(torch, psi[:B], dt)
    tol = 1e-7 if dt == "c64" else 1e-12
    calls = {
        "otoc": lambda: syk.syk_otoc(terms, 10.0, 0, 1, T_GRID, x, krylov_dim=40, tol=tol),
        "G": lambda: syk.syk_correlator_G(terms, 5.0, 2, T_GRID, x, krylov_dim=40, tol=tol)[0],
        "G_imag": lambda: syk.syk_correlator_G_imag(terms, 4.0, 3, np.linspace(0, 2.0, 5), x, krylov_dim=40,
                                                    tol=tol)[0],
    }
    for name, fn in calls.items():
        host, ch, mh = _run(fn, syk.GRAPHS_OFF)
        dev1, c1, m1 = _run(fn, syk.GRAPHS_DEVICE)   # builds the evolution graphs
        dev2, c2, m2 = _run(fn, syk.GRAPHS_DEVICE)   # replays them
        seg, cs, ms = _run(fn, syk.GRAPHS_SEGMENTS)  # the default: host-driven segment graphs
        assert np.array_equal(seg, host) and cs == ch and ms == mh, name
        assert np.array_equal(dev1, host) and np.array_equal(dev2, host), name
        assert c1["h_applies"] == ch["h_applies"] == c2["h_applies"], (name, ch, c1, c2)
        assert c1["krylov_bases"] == ch["krylov_bases"] == c2["krylov_bases"], (name, ch, c1, c2)
        assert m1 == mh == m2, (name, mh, m1, m2)
        assert m1["rows"] == 0


def test_device_driven_otoc_vs_oracle(setup):
    torch, terms, J, psi = setup
    F, _, _ = _run(lambda: syk.syk_otoc(terms, 10.0, 0, 1, T_GRID, to_dev(torch, psi, "c64"), krylov_dim=40,
                                        tol=1e-7), syk.GRAPHS_DEVICE)
    Fr = co.F_state(evolve.SectorSystem(N, J), 10.0, 0, 1, T_GRID, psi.T)
    a, b = F / F[0], Fr / Fr[0]
    assert float(np.max(np.max(np.abs(a - b), axis=0) / np.max(np.abs(b), axis=0))) < TOL["c64"]
