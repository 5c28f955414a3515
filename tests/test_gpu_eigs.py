"""syk_lowest_eigenvalues (GPU Lanczos) against the oracle's exact sector spectra."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from helpers import torch_or_skip
from oracle import hamiltonian as hm
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    return t


def _distinct(ev, gap=1e-9):
    ev = np.sort(ev)
    return ev[np.concatenate([[True], np.diff(ev) > gap])]


@pytest.mark.parametrize("N", [12, 14, 16, 18, 20])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_lowest_eigenvalues_vs_dense(torch, N, dt):
    """Both sectors, k = 8 lowest distinct levels (N = 12, 20: Kramers pairs within a sector,
    one copy each from a single start vector) against dense diagonalisation."""
    J = inputs.couplings(N, 6)
    terms = syk.syk_build_terms(N, J)
    start = inputs.random_states(N, 1, 9)[0].astype(np.complex64 if dt == "c64" else np.complex128)
    tol = 1e-10 if dt == "c128" else 1e-5
    for sector in (0, 1):
        spec = np.linalg.eigvalsh(hm.H_sector_sparse(N, J, sector).toarray())
        ref = _distinct(spec)[:8]
        scale = max(1.0, np.abs(spec).max())
        ev, res, n = syk.syk_lowest_eigenvalues(terms, 8, start, parity=sector, tol=tol)
        assert np.abs(ev - ref).max() < (1e-9 if dt == "c128" else 2e-5) * scale, (sector, ev, ref)
        assert np.all(res <= tol * scale * (1 + 1e-12))
        assert 8 <= n <= 1 << (N // 2 - 1)


def test_lowest_eigenvalues_N28_vs_eigsh(torch):
    """N = 28 (sector 2^13; N = 4 mod 8, so levels come in pairs): the 3 lowest distinct levels
    against scipy's ARPACK (8 lowest with multiplicity) on the oracle's sparse sector matrix."""
    N = 28
    J = inputs.couplings(N, 1)
    terms = syk.syk_build_terms(N, J)
    ref = _distinct(spla.eigsh(hm.H_sector_sparse(N, J, 0), k=8, which="SA", tol=1e-12)[0], gap=1e-8)[:3]
    ev, res, n = syk.syk_lowest_eigenvalues(terms, 3, inputs.random_states(N, 1, 4)[0], tol=1e-10)
    assert np.abs(ev - ref).max() < 1e-8


def test_lowest_eigenvalues_invalid(torch):
    J = inputs.couplings(8, 0)
    terms = syk.syk_build_terms(8, J)
    start = inputs.random_states(8, 1, 0)[0]
    with pytest.raises(syk.SykError):
        syk.syk_lowest_eigenvalues(terms, 9, start)          # k above the sector dimension 8
    with pytest.raises(syk.SykError):
        syk.syk_lowest_eigenvalues(terms, 2, start, max_steps=5000)
    with pytest.raises(syk.SykError):
        syk.syk_lowest_eigenvalues(terms, 2, np.zeros(8, dtype=np.complex128))  # zero start: no Krylov space
    ev, res, n = syk.syk_lowest_eigenvalues(terms, 8, start)  # the whole sector: all 8 levels exact
    assert np.allclose(ev, np.linalg.eigvalsh(hm.H_sector_sparse(8, J, 0).toarray()), atol=1e-12)


def test_lowest_eigenvalues_unconverged_bounds(torch):
    """A run cut short raises by default; with check=False it returns Ritz values, each an upper
    bound on the corresponding true level (Cauchy interlacing), with residual bounds above tol."""
    N = 20
    J = inputs.couplings(N, 6)
    terms = syk.syk_build_terms(N, J)
    start = inputs.random_states(N, 1, 9)[0]
    with pytest.raises(syk.SykError):
        syk.syk_lowest_eigenvalues(terms, 6, start, max_steps=16, tol=1e-12)
    ev, res, n = syk.syk_lowest_eigenvalues(terms, 6, start, max_steps=16, tol=1e-12, check=False)
    ref = _distinct(np.linalg.eigvalsh(hm.H_sector_sparse(N, J, 0).toarray()))[:6]
    assert n == 16 and np.all(ev >= ref - 1e-12) and res.max() > 1e-12
