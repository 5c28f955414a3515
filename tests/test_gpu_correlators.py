"""G(t) and the regularized OTOC on the GPU against the exact oracle (same random states)."""
import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    return t


@pytest.mark.parametrize("beta", [0.0, 5.0])
def test_G_N12_workload(torch, beta):
    """N=12, one seed, one state, c128, t in [0, 20] step 0.1, Krylov dimension 30."""
    N = 12
    J = inputs.couplings(N, 0)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 1, 0)
    ts = np.round(np.arange(201) * 0.1, 10)
    G, Z = syk.syk_correlator_G(terms, beta, 0, ts, to_dev(torch, psi, "c128"), krylov_dim=30, tol=1e-12)
    Gref, Zref = co.G_state(evolve.SectorSystem(N, J), beta, 0, ts, psi.T)
    assert rel(G, Gref) < TOL["c128"]
    assert rel(Z, Zref) < 1e-12
    if beta == 0.0:
        assert abs(G[0, 0] - 0.5) < 1e-14


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_G_host_input_and_batch(torch, dt):
    N = 16
    J = inputs.couplings(N, 3)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 4, 3)
    ts = [0.0, 0.5, 3.0, 3.0, 7.25]
    host = np.ascontiguousarray(psi.T.astype(np.complex64 if dt == "c64" else np.complex128))
    G, Z = syk.syk_correlator_G(terms, 2.0, 5, ts, host, krylov_dim=30, tol=1e-12 if dt == "c128" else 1e-7)
    Gref, _ = co.G_state(evolve.SectorSystem(N, J), 2.0, 5, ts, psi.T)
    assert rel(G, Gref) < TOL[dt]


@pytest.mark.parametrize("N", [4, 12, 16])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_otoc_vs_exact(torch, N, dt):
    J = inputs.couplings(N, 1)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 4, 11)
    ts = np.linspace(0.0, 15.0, 11)
    F = syk.syk_otoc(terms, 10.0, 0, 1, ts, to_dev(torch, psi, dt), krylov_dim=40,
                     tol=1e-12 if dt == "c128" else 1e-7)
    Fref = co.F_state(evolve.SectorSystem(N, J), 10.0, 0, 1, ts, psi.T)
    # error of the normalised curve F~ = F/F(0) of every state
    assert rel(F / F[0], Fref / Fref[0]) < TOL[dt]
    assert rel(F, Fref) < TOL[dt]
    assert np.allclose(F[0] / F[0], 1.0)


def test_otoc_beta0_t0_identity(torch):
    """beta = 0, t = 0: F(0) = <psi|chi_i chi_j chi_i chi_j|psi> = -|psi|^2 / 4 at any N."""
    N = 28
    J = inputs.couplings(N, 2)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 2, 5)
    F = syk.syk_otoc(terms, 0.0, 3, 8, [0.0], to_dev(torch, psi, "c128"))
    assert rel(F[0], -0.25 * np.sum(np.abs(psi) ** 2, axis=1)) < 1e-13


def test_otoc_N32_c64_vs_c128(torch):
    """Full size of the N=32 OTOC workload (dimension 2^15, beta J = 10), a few points, 4 states."""
    N = 32
    J = inputs.couplings(N, 0)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 4, 0)
    ts = [0.0, 2.5, 6.0]
    a = syk.syk_otoc(terms, 10.0, 0, 1, ts, to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
    b = syk.syk_otoc(terms, 10.0, 0, 1, ts, to_dev(torch, psi, "c64"), krylov_dim=40, tol=1e-7)
    assert rel(b / b[0], a / a[0]) < TOL["c64"]


def test_otoc_invalid(torch):
    terms = syk.syk_build_terms(8, inputs.couplings(8, 0))
    psi = to_dev(torch, inputs.random_states(8, 1, 0), "c128")
    with pytest.raises(syk.SykError):
        syk.syk_otoc(terms, 1.0, 2, 2, [0.0], psi)
    with pytest.raises(syk.SykError):
        syk.syk_otoc(terms, 1.0, 0, 1, [1.0, 0.5], psi)
    with pytest.raises(syk.SykError):
        syk.syk_correlator_G(terms, -1.0, 0, [0.0], psi)


@pytest.mark.parametrize("x", [(0.0, 0.0, 0.0, 1.0), (0.1, 0.4, 0.2, 0.3)])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_otoc_split_vs_exact(torch, x, dt):
    """Unregularized OTOC and a general rho split against the exact chain."""
    N = 12
    J = inputs.couplings(N, 4)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 3, 2)
    ts = np.linspace(0.0, 8.0, 9)
    F = syk.syk_otoc_split(terms, 6.0, x, 0, 1, ts, to_dev(torch, psi, dt), krylov_dim=30,
                           tol=1e-12 if dt == "c128" else 1e-7)
    Fr = co.F_state_split(evolve.SectorSystem(N, J), 6.0, x, 0, 1, ts, psi.T)
    assert rel(F, Fr) < TOL[dt]
    reg = syk.syk_otoc_split(terms, 6.0, (0.25,) * 4, 0, 1, ts[:3], to_dev(torch, psi, "c128"), krylov_dim=30)
    assert rel(reg, syk.syk_otoc(terms, 6.0, 0, 1, ts[:3], to_dev(torch, psi, "c128"), krylov_dim=30)) < 1e-13


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_G_imag_vs_exact(torch, dt):
    """c128 on 0 <= tau <= beta within 1e-10 of the oracle; c64 on tau <= beta/2.

    G(tau) = <w|chi_i y>/Z with w = e^{tau H} x, y = e^{-tau H} chi_i x, x = e^{-beta H/2} psi~.
    Rounding the stored vectors to FP32 perturbs this dot by about eps * |w| |y| / Z, and that
    factor amp(tau) = |w| |y| / Z is computed here from the oracle's exact vectors (it grows
    from 1/sqrt(2) at tau = 0 to about 1.2-1.5 at tau = beta/2 for these states); the c64
    error is bounded per tau by 1e-5 * amp(tau).  At tau = 0 the chain is <x|chi chi x>/<x|x>
    on one stored vector, so |G(0) - 1/2| is FP32 rounding only (bound 1e-6).  For
    tau > beta/2 the factor e^{(tau - beta/2) H} grows without bound; G(beta - tau) = G(tau)
    gives those values."""
    N = 16
    J = inputs.couplings(N, 5)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 2, 6)
    beta, i = 10.0, 3
    taus = np.linspace(0.0, beta if dt == "c128" else beta / 2, 11)
    G, Z = syk.syk_correlator_G_imag(terms, beta, i, taus, to_dev(torch, psi, dt), krylov_dim=30,
                                     tol=1e-12 if dt == "c128" else 1e-8)
    sysm = evolve.SectorSystem(N, J)
    Gr, Zr = co.G_imag_state(sysm, beta, i, taus, psi.T)
    assert np.abs(G[0] - 0.5).max() < (1e-13 if dt == "c128" else 1e-6)
    if dt == "c128":
        assert rel(G, Gr) < TOL["c128"] and rel(Z, Zr) < 1e-11
        return
    x = sysm.expmv(-beta / 2, psi.T, 0)
    amp = np.array([np.linalg.norm(sysm.expmv(tau, x, 0), axis=0) *
                    np.linalg.norm(sysm.expmv(-tau, sysm.chi(i, 0, x), 1), axis=0) / Zr for tau in taus])
    assert float(np.max(np.abs(G - Gr) / amp)) < 1e-5, np.abs(G - Gr) / amp
    assert rel(Z, Zr) < 1e-5


def test_G_N40_c64_vs_c128(torch):
    """G(t) at full size (N = 40, sector 2^19, beta J = 5), two states: complex64 vectors with
    FP64 scalars against the complex128 path; G(0) = 1/2 for every state."""
    N = 40
    J = inputs.couplings(N, 3)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 2, 3)
    ts = [0.0, 1.0, 2.5]
    a, Za = syk.syk_correlator_G(terms, 5.0, 2, ts, to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
    b, Zb = syk.syk_correlator_G(terms, 5.0, 2, ts, to_dev(torch, psi, "c64"), krylov_dim=40, tol=1e-7)
    assert rel(b, a) < TOL["c64"]
    assert rel(Zb, Za) < TOL["c64"]
    assert np.abs(a[0] - 0.5).max() < 1e-12


def test_otoc_unregularized_N40_c64_vs_c128(torch):
    """The unregularized OTOC (rho split (0, 0, 0, 1)) at full size (N = 40, beta J = 10), two
    states, t = 0 and 1.2: complex64 against complex128."""
    N = 40
    J = inputs.couplings(N, 4)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 2, 4)
    x = (0.0, 0.0, 0.0, 1.0)
    a = syk.syk_otoc_split(terms, 10.0, x, 0, 1, [0.0, 1.2], to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
    b = syk.syk_otoc_split(terms, 10.0, x, 0, 1, [0.0, 1.2], to_dev(torch, psi, "c64"), krylov_dim=40, tol=1e-7)
    assert rel(b / b[0], a / a[0]) < TOL["c64"]
