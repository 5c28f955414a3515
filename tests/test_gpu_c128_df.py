"""The complex128 matvec in double-float arithmetic (the default; syk_c128_arith(0)) against
the FP64 oracle and against the native FP64 kernel (syk_c128_arith(1)).

Double-float keeps 48 significand bits: a sum of M(N) terms per row carries a relative error
of order 2^-48 sqrt(M) typically and M 2^-48 at worst (M = 5036 at N = 40: 2.5e-13 and
1.8e-11), against the FP64 kernel's 2^-53 scale; the bound used here is 1e-12 relative to
the largest element of each result, two orders below the 1e-10 curve tolerance.
"""
import numpy as np
import pytest

from helpers import rel, to_dev, torch_or_skip
from oracle import hamiltonian as hm
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu

DF_TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    assert syk.syk_c128_arith() == syk.C128_DOUBLE_FLOAT  # the default
    return t


def _apply(terms, sector, x, mode):
    prev = syk.syk_c128_arith(mode)
    try:
        syk.syk_matvec_launches(reset=True)
        y = syk.syk_apply_H(terms, sector, x)
        return y.cpu().numpy(), syk.syk_matvec_launches(reset=True)
    finally:
        syk.syk_c128_arith(prev)


@pytest.mark.parametrize("N", [20, 24])
@pytest.mark.parametrize("B", [1, 2, 4, 8, 16])
def test_df_apply_full_vs_oracle_and_fp64(torch, N, B):
    J = inputs.couplings(N, 31)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, B, 200 + B)
    x = to_dev(torch, psi, "c128")
    for sector in (0, 1):
        ref = hm.H_sector_sparse(N, J, sector) @ psi.T
        ydf, mv = _apply(terms, sector, x, syk.C128_DOUBLE_FLOAT)
        y64, _ = _apply(terms, sector, x, syk.C128_FP64)
        assert mv["tiled"] == 1 and mv["rows"] == 0, mv
        assert rel(ydf, ref) < DF_TOL, (sector, rel(ydf, ref))
        assert rel(ydf, y64) < DF_TOL
        assert rel(y64, ref) < 1e-14


def test_df_one_state_every_launch_shape(torch):
    """One complex128 state: the double-float tiled kernel at every CTA width and cluster size,
    full H at N = 24 (sector 2^11: 8, 4 or 2 tiles of 4 rows per thread), both sectors, against
    the FP64 oracle."""
    N = 24
    J = inputs.couplings(N, 32)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 1, 301)
    x = to_dev(torch, psi, "c128")
    try:
        for sector in (0, 1):
            ref = hm.H_sector_sparse(N, J, sector) @ psi.T
            for ntb in (6, 7, 8):
                for cs in (1, 2, 4, 8):
                    syk.syk_autotune_import('{"apply_tiles": [{"N": %d, "dtype": %d, "batch": 1, "ntb": %d, '
                                            '"cluster": %d}]}' % (N, syk.SYK_C128, ntb, cs))
                    y, mv = _apply(terms, sector, x, syk.C128_DOUBLE_FLOAT)
                    assert mv["tiled"] == 1 and mv["rows"] == 0, (ntb, cs, mv)
                    assert rel(y, ref) < DF_TOL, (sector, ntb, cs, rel(y, ref))
    finally:
        syk.syk_autotune_reset()


@pytest.mark.parametrize("B", [1, 16])
def test_df_apply_sampled_rows_N40(torch, B):
    """N = 40 (sector 2^19, 5036 X-masks per row): sampled rows against the oracle's
    term-by-term FP64 row sums."""
    N = 40
    J = inputs.couplings(N, 8)
    terms = syk.syk_build_terms(N, J)
    D = 1 << (N // 2 - 1)
    psi = inputs.random_states(N, B, 9)
    rng = np.random.default_rng(40)
    rows = np.unique(np.concatenate([[0, 1, D - 1], rng.integers(0, D, 13)]))
    x = to_dev(torch, psi, "c128")
    for sector in (0, 1):
        ydf, mv = _apply(terms, sector, x, syk.C128_DOUBLE_FLOAT)
        assert mv["tiled"] == 1, mv
        ref = hm.apply_rows(N, J, sector, psi.T, rows)
        assert rel(ydf[rows], ref) < DF_TOL, (sector, rel(ydf[rows], ref))


def test_df_expmv_matches_fp64_kernel(torch):
    """A Krylov evolution e^{(-1 - 6i) H} psi at N = 24 with either arithmetic agrees to 1e-12."""
    N = 24
    terms = syk.syk_build_terms(N, inputs.couplings(N, 4))
    x = to_dev(torch, inputs.random_states(N, 4, 5), "c128")
    out = {}
    for mode in (syk.C128_DOUBLE_FLOAT, syk.C128_FP64):
        prev = syk.syk_c128_arith(mode)
        try:
            out[mode], _ = syk.syk_expmv(terms, 0, complex(-1.0, -6.0), x, krylov_dim=40, tol=1e-13)
        finally:
            syk.syk_c128_arith(prev)
    assert rel(out[0].cpu().numpy(), out[1].cpu().numpy()) < 1e-12


def test_c128_arith_rejects_bad_mode(torch):
    with pytest.raises(syk.SykError):
        syk.syk_c128_arith(7)
    assert syk.syk_c128_arith() == syk.C128_DOUBLE_FLOAT
