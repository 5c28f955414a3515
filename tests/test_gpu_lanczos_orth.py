"""expmv with the Lanczos basis orthogonalised by the three-term recurrence alone
(syk_lanczos_orth mode 1) against the exact oracle, next to full Gram-Schmidt (mode 0).

The Krylov approximation of e^{zH}psi from a Lanczos basis that has lost global orthogonality
in finite precision stays accurate to about the rounding level of the vectors (Druskin,
Greenbaum & Knizhnerman 1998); these tests hold it to the same per-curve tolerances as the
fully orthogonalised basis, on the benchmark's matvec kernels (N = 24, 16 states) and at
beta J = 10 to t = 12.
"""
import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu

T_GRID = np.round(np.linspace(0.0, 12.0, 7), 12)


def curve_err(F, Fref):
    a, b = F / F[0], Fref / Fref[0]
    return float(np.max(np.max(np.abs(a - b), axis=0) / np.max(np.abs(b), axis=0)))


@pytest.fixture(scope="module")
def n24():
    torch_or_skip()
    syk.load(build_if_missing=True)
    N = 24
    J = inputs.couplings(N, 2)
    psi = inputs.random_states(N, 16, 2)
    F = co.F_state(evolve.SectorSystem(N, J), 10.0, 0, 1, T_GRID, psi.T)
    return {"terms": syk.syk_build_terms(N, J), "psi": psi, "F": F}


def _with_orth(dtype, mode, fn):
    prev = syk.syk_lanczos_orth(dtype, mode)
    try:
        return fn()
    finally:
        syk.syk_lanczos_orth(dtype, prev)


@pytest.mark.parametrize("dt,B", [("c64", 16), ("c64", 8), ("c128", 2), ("c128", 16)])
@pytest.mark.parametrize("mode", [syk.ORTH_FULL, syk.ORTH_LOCAL])
def test_otoc_N24_by_orthogonalisation(n24, dt, B, mode):
    torch = torch_or_skip()
    code = syk.SYK_C64 if dt == "c64" else syk.SYK_C128
    x = to_dev(torch, n24["psi"][:B], dt)
    tol = 1e-7 if dt == "c64" else 1e-12
    F = _with_orth(code, mode, lambda: syk.syk_otoc(n24["terms"], 10.0, 0, 1, T_GRID, x, krylov_dim=40, tol=tol))
    assert curve_err(F, n24["F"][:, :B]) < TOL[dt]


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expmv_N20_local_orthogonalisation_vs_exact(dt):
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    N = 20
    J = inputs.couplings(N, 6)
    psi = inputs.random_states(N, 4, 6)
    code = syk.SYK_C64 if dt == "c64" else syk.SYK_C128
    z = complex(-2.5, -12.0)
    out, _ = _with_orth(code, syk.ORTH_LOCAL, lambda: syk.syk_expmv(
        syk.syk_build_terms(N, J), 0, z, to_dev(torch, psi, dt), krylov_dim=40,
        tol=1e-7 if dt == "c64" else 1e-12))
    ref = evolve.SectorSystem(N, J).expmv(z, psi.T, 0)
    assert rel(out.cpu().numpy(), ref) < TOL[dt]


def test_orth_mode_api():
    torch_or_skip()
    syk.load(build_if_missing=True)
    with pytest.raises(syk.SykError):
        syk.syk_lanczos_orth(syk.SYK_C64, 5)
    with pytest.raises(syk.SykError):
        syk.syk_lanczos_orth(9, 0)
    prev = syk.syk_lanczos_orth(syk.SYK_C64, syk.ORTH_LOCAL)
    assert syk.syk_lanczos_orth(syk.SYK_C64) == syk.ORTH_LOCAL
    syk.syk_lanczos_orth(syk.SYK_C64, prev)
