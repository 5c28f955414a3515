"""K3 (tridiagonal exponential) and the Lanczos expmv (K2-K4) against the oracle."""
import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from oracle import evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    return t


@pytest.mark.parametrize("m", [1, 2, 5, 30, 40, 64])
def test_tridiag_expm_vs_oracle(torch, m):
    B = 3
    al = np.zeros((m, B))
    be = np.zeros((max(m - 1, 0), B))
    for b in range(B):
        a, e = inputs.random_tridiagonal(m, 10 * m + b, scale=0.7)
        al[:, b], be[:, b] = a, e
    b0 = np.array([1.0, 2.5, 0.3])
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), device="cuda")
    for z in (-2.3j, -0.7, 0.3 - 1.5j, -9.0j):
        out = syk.syk_tridiag_expm(dev(al), dev(be), dev(b0), z).cpu().numpy()
        for b in range(B):
            ref = evolve.tridiag_expm_e1(al[:, b], be[:, b], z, beta0=b0[b])
            assert rel(out[:, b], ref) < 1e-12, (m, z, b)


@pytest.mark.parametrize("N", [8, 12, 16, 20])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_expmv_vs_exact(torch, N, dt):
    J = inputs.couplings(N, 31)
    terms = syk.syk_build_terms(N, J)
    sysm = evolve.SectorSystem(N, J)
    tol = 1e-12 if dt == "c128" else 1e-7
    for sector in (0, 1):
        for B in (1, 5):
            psi = inputs.random_states(N, B, 40 + B)
            for z in (-5.0j, -2.5, -1.1 - 0.7j, 3.0j):
                ref = sysm.expmv(z, psi.T, sector)
                out, nsteps = syk.syk_expmv(terms, sector, z, to_dev(torch, psi, dt), krylov_dim=30, tol=tol)
                assert nsteps >= 1
                assert rel(out.cpu().numpy(), ref) < TOL[dt], (N, sector, B, z)


def test_expmv_substeps_and_inplace(torch):
    N = 16
    J = inputs.couplings(N, 2)
    terms = syk.syk_build_terms(N, J)
    sysm = evolve.SectorSystem(N, J)
    psi = inputs.random_states(N, 2, 8)
    x = to_dev(torch, psi, "c128")
    out, nsteps = syk.syk_expmv(terms, 0, -40.0j, x, krylov_dim=12, tol=1e-12, out=x)
    assert nsteps > 1
    assert out.data_ptr() == x.data_ptr()
    ref = sysm.expmv(-40.0j, psi.T, 0)
    assert rel(out.cpu().numpy(), ref) < TOL["c128"]
    assert np.allclose(np.linalg.norm(out.cpu().numpy(), axis=0), np.linalg.norm(psi, axis=1), rtol=1e-11)


def test_expmv_breakdown_small_space(torch):
    """N=8: sector dimension 8 < Krylov dimension 30, so Lanczos breaks down (exact)."""
    N = 8
    J = inputs.couplings(N, 4)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 3, 1)
    out, nsteps = syk.syk_expmv(terms, 1, -25.0j, to_dev(torch, psi, "c128"), krylov_dim=30, tol=1e-12)
    assert nsteps == 1
    ref = evolve.SectorSystem(N, J).expmv(-25.0j, psi.T, 1)
    assert rel(out.cpu().numpy(), ref) < 1e-11


def test_expmv_zero_column_and_workspace(torch):
    N = 12
    J = inputs.couplings(N, 6)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 3, 5)
    psi[1] = 0
    nb = syk.syk_workspace_bytes(N, syk.SYK_C128, 20, 3)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out, _ = syk.syk_expmv(terms, 0, -3.0j, to_dev(torch, psi, "c128"), krylov_dim=20, workspace=ws)
    ref = evolve.SectorSystem(N, J).expmv(-3.0j, psi.T, 0)
    assert np.all(out.cpu().numpy()[:, 1] == 0)
    assert rel(out.cpu().numpy(), ref) < TOL["c128"]
    small = torch.empty(nb // 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(syk.SykError):
        syk.syk_expmv(terms, 0, -3.0j, to_dev(torch, psi, "c128"), krylov_dim=20, workspace=small)


def test_expmv_c64_matches_c128_N32(torch):
    """Full size of the N=32 workload (dimension 2^15), 16 states: c64 against c128."""
    N = 32
    J = inputs.couplings(N, 0)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 16, 0)
    a, _ = syk.syk_expmv(terms, 0, -4.0j, to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
    b, _ = syk.syk_expmv(terms, 0, -4.0j, to_dev(torch, psi, "c64"), krylov_dim=40, tol=1e-7)
    assert rel(b.cpu().numpy(), a.cpu().numpy()) < TOL["c64"]
    n0 = np.linalg.norm(psi, axis=1)
    assert np.allclose(np.linalg.norm(a.cpu().numpy(), axis=0), n0, rtol=1e-11)
