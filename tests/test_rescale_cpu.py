"""Finite-size rescaling analysis (host code) against closed forms and an independent library."""
import math

import numpy as np
import pytest

from paper_2002_05725_gb300 import rescale


def test_crossing_time_linear_and_exponential():
    t = np.linspace(0.0, 4.0, 41)
    # piecewise linear data: interpolation is exact
    assert abs(rescale.crossing_time(t, 1.0 - 0.1 * t, 0.75) - 2.5) < 1e-12
    # 1 - a e^{lam t}: analytic crossing log(F0/a)/lam, interpolation error O(dt^2)
    a, lam, F0 = 0.02, 1.3, 0.25
    tf = np.linspace(0.0, 4.0, 4001)
    assert abs(rescale.crossing_time(tf, 1.0 - a * np.exp(lam * tf), 1.0 - F0) - math.log(F0 / a) / lam) < 1e-5
    # never reached, starts below, bad grids
    assert math.isnan(rescale.crossing_time(t, np.ones_like(t), 0.75))
    assert math.isnan(rescale.crossing_time(t, np.full_like(t, 0.5), 0.75))
    with pytest.raises(ValueError):
        rescale.crossing_time(t[::-1], 1.0 - 0.1 * t, 0.75)


def test_rescaling_symmetric_family_recovers_lambda():
    """F~_N(t) = 1 - (c/N) e^{lam t} obeys N -> rN, t -> t + log(r)/lam exactly: t*_N =
    log(F0 N / c)/lam, so lambda_fit(N) = lam at every N and the extrapolation returns lam."""
    lam, c, F0 = 0.83, 0.4, 0.25
    Ns = list(range(20, 42, 2))
    t = np.linspace(0.0, 12.0, 24001)
    Ft = {N: 1.0 - (c / N) * np.exp(lam * t) for N in Ns}
    for beta, deg in ((1.8, 1), (5.6, 2)):
        res = rescale.lyapunov(Ns, t, Ft, beta, F0=F0)
        assert res["degree"] == deg
        assert np.allclose(res["t_star"], [math.log(F0 * N / c) / lam for N in Ns], atol=2e-6)
        assert np.allclose(res["lambda_fit"], lam, rtol=1e-4)
        assert abs(res["lambda"] - lam) < 1e-4 * lam


def test_extrapolation_exact_polynomial_and_stderr():
    Ns = np.arange(20.0, 48.0, 2.0)
    lam = 1.1 - 3.0 / Ns + 20.0 / Ns ** 2
    l0, se, coef = rescale.extrapolate(Ns, lam, 2)
    assert np.allclose(coef, [1.1, -3.0, 20.0], rtol=1e-8)
    assert se < 1e-10
    l0, se, coef = rescale.extrapolate(Ns[:2], lam[:2], 1)  # no residual degrees of freedom
    assert math.isnan(se)
    with pytest.raises(ValueError):
        rescale.extrapolate(Ns[:2], lam[:2], 2)


def test_extrapolation_stderr_matches_linregress():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    Ns = np.arange(20.0, 42.0, 2.0)
    lam = 0.9 - 4.0 / Ns + 0.01 * rng.standard_normal(len(Ns))
    l0, se, coef = rescale.extrapolate(Ns, lam, 1)
    ref = scipy_stats.linregress(1.0 / Ns, lam)
    assert abs(l0 - ref.intercept) < 1e-12
    assert abs(se - ref.intercept_stderr) < 1e-12 * max(1.0, ref.intercept_stderr)


def test_lambda_fit_successive_sizes():
    Nk, lam = rescale.lambda_fit([20, 24, 30], [1.0, 1.5, 1.9])
    assert np.array_equal(Nk, [24.0, 30.0])
    assert np.allclose(lam, [math.log(24 / 20) / 0.5, math.log(30 / 24) / 0.4])
    with pytest.raises(ValueError):
        rescale.lambda_fit([20, 20], [1.0, 2.0])


def test_disorder_average_normalizes_per_draw():
    F1 = np.array([[2.0, 2.0], [1.0, 1.0]], dtype=complex)      # draw 1: sum 4 -> 2
    F2 = np.array([[-1.0, -3.0], [-3.0, -1.0]], dtype=complex)  # draw 2: sum -4 -> -4
    Ft = rescale.disorder_average([F1, F2])
    assert np.allclose(Ft, [1.0, (0.5 + 1.0) / 2])


def test_admissible_window():
    ev = {20: np.linspace(0.0, 3.0, 25), 30: np.linspace(0.0, 0.5, 25), 40: np.linspace(0.0, 0.1, 25),
          50: np.linspace(0.0, 0.1, 10)}
    # 20th eigenvalue: 3.0 * 19/24, 0.5 * 19/24, 0.1 * 19/24; N=50 has fewer than 20 eigenvalues
    assert rescale.admissible(ev, beta=2.0) == [30, 40]
    assert rescale.admissible(ev, beta=2.0, window=0.1) == [40]


@pytest.mark.parametrize("N", [12, 14, 16, 18])
def test_full_space_levels_match_dense_spectrum(N):
    """The N mod 8 degeneracy rules (12: doubling within a sector; 14, 18: sectors are copies;
    16: none) rebuild the lowest full-space levels from distinct sector levels: checked against
    the oracle's dense full-space spectrum."""
    from oracle import hamiltonian as hm
    from paper_2002_05725_gb300 import inputs
    J = inputs.couplings(N, 2)
    full = np.linalg.eigvalsh(hm.H_dense(N, J))
    distinct = {}
    for sec in (0, 1):
        ev = np.linalg.eigvalsh(hm.H_sector_sparse(N, J, sec).toarray())
        keep = np.concatenate([[True], np.diff(ev) > 1e-9])
        distinct[sec] = ev[keep]
    secs, kk = rescale.sector_levels_needed(N, 20)
    got = rescale.full_space_levels(N, {s: distinct[s][:kk] for s in secs}, 20)
    assert np.allclose(got, full[:20], atol=1e-10)
    if N % 8 in (2, 6):  # either sector alone suffices
        assert np.allclose(rescale.full_space_levels(N, {1: distinct[1]}, 20), full[:20], atol=1e-10)


def test_lyapunov_restricted_to_admissible_sizes():
    """use_Ns restricts the extrapolation to the listed sizes: an outlier at a non-admissible
    size then has no influence on the extrapolated lambda."""
    lam, c = 0.7, 0.3
    Ns = [20, 24, 28, 32, 36]
    t = np.linspace(0.0, 15.0, 30001)
    Ft = {N: 1.0 - (c / N) * np.exp(lam * t) for N in Ns}
    Ft[24] = 1.0 - (2 * c / 24) * np.exp(lam * t)  # size 24 off the scaling family
    bad = rescale.lyapunov(Ns, t, Ft, 1.8)
    good = rescale.lyapunov(Ns, t, Ft, 1.8, use_Ns=[28, 32, 36])
    assert abs(bad["lambda"] - lam) > 1e-2
    assert good["fit_N"] == [32.0, 36.0] and abs(good["lambda"] - lam) < 1e-4


def test_lyapunov_pairs_only_admissible_sizes():
    """An admissible size whose lower neighbour is not admissible is paired with the next
    admissible size below it, never with the outlier: with the outlier at 28 and sizes 20, 32,
    36 admissible, lambda_fit(32) comes from (20, 32) and is exact for the scaling family."""
    lam, c = 0.7, 0.3
    Ns = [20, 24, 28, 32, 36]
    t = np.linspace(0.0, 15.0, 30001)
    Ft = {N: 1.0 - (c / N) * np.exp(lam * t) for N in Ns}
    Ft[28] = 1.0 - (3 * c / 28) * np.exp(lam * t)  # size 28 off the scaling family
    res = rescale.lyapunov(Ns, t, Ft, 1.8, use_Ns=[20, 32, 36])
    assert res["fit_N"] == [32.0, 36.0]
    assert np.allclose(res["lambda_fit"], lam, rtol=1e-4)
    assert abs(res["lambda"] - lam) < 1e-4
    assert len(res["t_star"]) == len(Ns)
    with pytest.raises(ValueError):
        rescale.lyapunov(Ns, t, Ft, 1.8, use_Ns=[36])


def test_sector_levels_needed_by_N_mod_8():
    assert rescale.sector_levels_needed(40) == ((0, 1), 20)   # 0 mod 8: no degeneracy
    assert rescale.sector_levels_needed(36) == ((0, 1), 10)   # 4 mod 8: pairs within sectors
    assert rescale.sector_levels_needed(34) == ((0,), 10)     # 2 mod 8: sectors are copies
    assert rescale.sector_levels_needed(38) == ((0,), 10)     # 6 mod 8
    with pytest.raises(ValueError):
        rescale.full_space_levels(40, {0: np.zeros(20)}, 20)  # both sectors needed
