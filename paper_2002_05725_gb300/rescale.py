"""Finite-size rescaling extraction of the Lyapunov exponent (Supp. Sec. "Finite-size rescaling
method", Eq. scaling) from OTOC curves computed on the GPU.

The OTOCs are assumed to obey the rescaling symmetry N -> rN, t -> t + log(r)/lambda. The
procedure has three steps:

1. For each system size N, find the time t*(N) at which the disorder-averaged normalized OTOC
   F~(t) = F(t)/F(0) reaches a fixed level. The data are interpolated between grid points.
2. Estimate lambda_fit(N) from successive sizes: 1/lambda_fit = (t*_N - t*_N') / (log N - log N').
3. Extrapolate lambda_fit(N) to N -> infinity by least squares in 1/N, with a linear function
   for beta J < 5.6 and a quadratic one for beta J >= 5.6. The error bar is the standard error
   of the constant term.

Only sizes whose lowest 20 eigenvalues lie within an energy window of the ground state enter
the extrapolation.

Readings:
* The crossing level is F~(t*) = 1 - F0, with F0 = 0.25 (main results) or 0.16, as the figure
  captions of the procedure and of the fluctuation study state it; this is the early-time
  regime where 1 - F~ grows like e^{lambda t}/N. One passage of the text writes F~(t_N) = F0;
  pass `level` to use any other level.
* The energy window is 1/beta (the text; the caption writes beta J).
* Interpolation is linear between the two grid points that bracket the first crossing.
* lambda_fit from sizes N' < N is attributed to the larger size N.
* Disorder average: each coupling draw's one-state estimates are summed over its states (the
  typicality trace estimator) and normalized by their sum at t = 0; the draws' normalized
  curves are then averaged.

Host code (numpy) working on curves returned by `syk.syk_otoc_batch`. Running the module
(`python -m paper_2002_05725_gb300.rescale`) computes the curves on the GPU and prints one JSON
line with t*(N), lambda_fit(N) and the extrapolated lambda.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np


def disorder_average(F_draws) -> np.ndarray:
    """F~(t) from a list of per-draw one-state OTOC estimates F (nt, nstates) (complex).

    Per draw: Re sum_s F[t, s] / Re sum_s F[0, s]; then the mean over draws."""
    curves = []
    for F in F_draws:
        F = np.asarray(F)
        if F.ndim == 1:
            F = F[:, None]
        tot = np.real(F.sum(axis=1))
        if tot[0] == 0.0:
            raise ValueError("F(0) sums to zero: cannot normalize")
        curves.append(tot / tot[0])
    if not curves:
        raise ValueError("no draws")
    return np.mean(curves, axis=0)


def crossing_time(t, Ft, level: float) -> float:
    """First time at which Ft reaches `level` from above (Ft[0] > level), by linear
    interpolation between the bracketing grid points; NaN if the curve never reaches it."""
    t = np.asarray(t, dtype=np.float64)
    Ft = np.asarray(Ft, dtype=np.float64)
    if t.shape != Ft.shape or t.ndim != 1 or len(t) < 2:
        raise ValueError("t and Ft must be 1-d arrays of the same length >= 2")
    if np.any(np.diff(t) <= 0):
        raise ValueError("t must be increasing")
    if Ft[0] <= level:
        return float(t[0]) if Ft[0] == level else math.nan
    below = np.nonzero(Ft <= level)[0]
    if len(below) == 0:
        return math.nan
    k = int(below[0])
    f0, f1 = Ft[k - 1], Ft[k]
    return float(t[k - 1] + (f0 - level) / (f0 - f1) * (t[k] - t[k - 1]))


def lambda_fit(Ns, tstar):
    """lambda_fit between successive sizes: (log N_k - log N_{k-1}) / (t*_k - t*_{k-1}),
    attributed to N_k. Returns (N_k, lambda_k) for k = 1..len(Ns)-1."""
    Ns = np.asarray(Ns, dtype=np.float64)
    tstar = np.asarray(tstar, dtype=np.float64)
    if Ns.shape != tstar.shape or len(Ns) < 2 or np.any(np.diff(Ns) <= 0):
        raise ValueError("need >= 2 increasing sizes with one t* each")
    lam = np.diff(np.log(Ns)) / np.diff(tstar)
    return Ns[1:], lam


def extrapolate(Ns, lam, degree: int):
    """Least-squares fit lambda(N) = sum_{p=0}^{degree} c_p N^{-p}.

    Returns (c_0, standard error of c_0, all coefficients). The standard error is
    sqrt(s^2 [(A^T A)^{-1}]_00) with s^2 = RSS / (n - degree - 1); it is NaN when the fit has no
    residual degrees of freedom."""
    Ns = np.asarray(Ns, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    n, p = len(Ns), degree + 1
    if degree < 0 or n < p:
        raise ValueError(f"{n} points cannot fix a degree-{degree} polynomial")
    A = np.vander(1.0 / Ns, p, increasing=True)
    coef, *_ = np.linalg.lstsq(A, lam, rcond=None)
    if n == p:
        return float(coef[0]), math.nan, coef
    resid = lam - A @ coef
    s2 = float(resid @ resid) / (n - p)
    cov = s2 * np.linalg.inv(A.T @ A)
    return float(coef[0]), float(math.sqrt(max(cov[0, 0], 0.0))), coef


def full_space_levels(N: int, sector_levels: dict, k: int) -> np.ndarray:
    """The k lowest eigenvalues of H on the whole 2^{N/2}-dimensional space, with multiplicity,
    from the distinct levels of the parity sectors (sector_levels[0], sector_levels[1]; what
    single-vector Lanczos returns).  The particle-hole symmetry of the SYK model fixes the
    degeneracies by N mod 8: for N = 4 mod 8 every level is doubly degenerate within its sector
    (both sectors needed); for N = 2, 6 mod 8 the two sectors carry the same levels (either one
    suffices); for N = 0 mod 8 levels are non-degenerate and both sectors are needed."""
    r = N % 8
    if r in (2, 6):
        lv = np.asarray(sector_levels[0] if 0 in sector_levels else sector_levels[1], dtype=np.float64)
        out = np.repeat(np.sort(lv), 2)
    else:
        if 0 not in sector_levels or 1 not in sector_levels:
            raise ValueError(f"N = {N}: both parity sectors are needed")
        both = np.concatenate([np.asarray(sector_levels[0], np.float64), np.asarray(sector_levels[1], np.float64)])
        out = np.sort(np.repeat(both, 2) if r == 4 else both)
    if len(out) < k:
        raise ValueError(f"N = {N}: {len(out)} levels known, {k} needed")
    return out[:k]


def sector_levels_needed(N: int, k: int = 20):
    """(sectors, distinct levels per sector) that `full_space_levels` needs for k full-space levels."""
    r = N % 8
    if r in (2, 6):
        return (0,), (k + 1) // 2
    return ((0, 1), (k + 1) // 2) if r == 4 else ((0, 1), k)


def admissible(evals_by_N: dict, beta: float, k: int = 20, window=None):
    """Sizes whose k lowest eigenvalues lie within `window` (default 1/beta) of the ground state."""
    w = (1.0 / beta) if window is None else float(window)
    out = []
    for N, ev in sorted(evals_by_N.items()):
        ev = np.sort(np.asarray(ev, dtype=np.float64))
        if len(ev) >= k and ev[k - 1] - ev[0] <= w:
            out.append(N)
    return out


def lyapunov(Ns, t, Ft_by_N: dict, beta: float, F0: float = 0.25, level=None, degree=None, use_Ns=None):
    """The whole procedure on disorder-averaged curves Ft_by_N[N] (on the common grid t).

    level defaults to 1 - F0; degree to 2 for beta >= 5.6 and 1 below; use_Ns restricts the
    procedure to those sizes (e.g. `admissible(...)`), default all: only they enter the pairs
    of lambda_fit and the extrapolation (t* is still reported for every size)."""
    lev = 1.0 - F0 if level is None else float(level)
    Ns = sorted(int(N) for N in Ns)
    tstar = [crossing_time(t, Ft_by_N[N], lev) for N in Ns]
    if any(math.isnan(x) for x in tstar):
        missing = [N for N, x in zip(Ns, tstar) if math.isnan(x)]
        raise ValueError(f"F~ never reaches {lev} for N = {missing}: extend the time grid")
    keep = Ns if use_Ns is None else [N for N in Ns if N in {int(u) for u in use_Ns}]
    if len(keep) < 2:
        raise ValueError(f"lambda_fit needs at least two sizes, got {keep}")
    Nk, lam = lambda_fit(keep, [ts for N, ts in zip(Ns, tstar) if N in keep])
    deg = (2 if beta >= 5.6 else 1) if degree is None else int(degree)
    lam0, se, coef = extrapolate(Nk, lam, deg)
    return {"beta": beta, "level": lev, "N": Ns, "t_star": tstar, "lambda_fit_N": Nk.tolist(),
            "lambda_fit": lam.tolist(), "degree": deg, "fit_N": Nk.tolist(), "lambda": lam0,
            "lambda_stderr": se, "coefficients": coef.tolist()}


def main():
    import argparse

    import torch

    from . import inputs, syk
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", default="20,22,24,26,28,30,32,34,36,38,40")
    ap.add_argument("--beta", type=float, default=1.8)
    ap.add_argument("--F0", type=float, default=0.25)
    ap.add_argument("--states", type=int, default=8)
    ap.add_argument("--draws", type=int, default=1)
    ap.add_argument("--tmax", type=float, default=8.0)
    ap.add_argument("--dt", type=float, default=0.1)
    ap.add_argument("--krylov", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--out-dir", default=None,
                    help="store each item's curves in this directory (one .npz per item) and reuse the ones "
                         "already there, so that an interrupted run resumes")
    ap.add_argument("--spectral-window", action="store_true",
                    help="extrapolate over the sizes whose lowest 20 eigenstates (GPU Lanczos on the first "
                         "coupling draw) lie within 1/beta of the ground state")
    a = ap.parse_args()
    syk.load()
    Ns = [int(v) for v in a.N.split(",")]
    t = np.round(np.arange(0.0, a.tmax + 0.5 * a.dt, a.dt), 12)
    keys = [N for N in Ns for _ in range(a.draws)]
    t0 = time.perf_counter()
    if a.out_dir:
        from . import curves
        specs = [{"N": N, "seed": 0, "realization": r, "beta": a.beta, "states": a.states}
                 for N in Ns for r in range(a.draws)]
        Fs, _ = curves.run_otoc_items(specs, t, a.out_dir, dtype=syk.SYK_C64, krylov_dim=a.krylov, tol=a.tol,
                                      nworkers=a.workers)
    else:
        items = []
        for N in Ns:
            for r in range(a.draws):
                terms = syk.syk_build_terms(N, inputs.couplings(N, seed=0, realization=r))
                psi = torch.from_numpy(np.ascontiguousarray(inputs.random_states(N, a.states, 0, r).T)).to(
                    torch.complex64).cuda()
                items.append((terms, a.beta, psi))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Fs = syk.syk_otoc_batch(items, 0, 1, t, syk.SYK_C64, a.krylov, a.tol, a.workers)
    wall = time.perf_counter() - t0
    Ft = {N: disorder_average([F for F, k in zip(Fs, keys) if k == N]) for N in Ns}
    use, low, resid, eig_s = None, {}, {}, 0.0
    if a.spectral_window:
        t1 = time.perf_counter()
        for N in Ns:
            terms = syk.syk_build_terms(N, inputs.couplings(N, seed=0, realization=0))
            start = np.ascontiguousarray(inputs.random_states(N, 1, 7)[0].astype(np.complex64))
            secs, kk = sector_levels_needed(N)
            lv = {}
            for sec in secs:
                # an unconverged run still bounds every level from above (Cauchy interlacing), so
                # its E_20 - E_0 overestimates the spread; the residuals are reported
                ev, rs, _ = syk.syk_lowest_eigenvalues(terms, kk, start, parity=sec, max_steps=2048, tol=1e-4,
                                                       check=False)
                lv[sec] = ev
                resid[N] = max(resid.get(N, 0.0), float(np.max(rs)))
            low[N] = full_space_levels(N, lv, 20)
        use = admissible(low, a.beta)
        eig_s = time.perf_counter() - t1
    res = lyapunov(Ns, t, Ft, a.beta, F0=a.F0, use_Ns=use)
    if a.spectral_window:
        res.update({"spectral_window": 1.0 / a.beta, "admissible_N": use, "eig_seconds": eig_s,
                    "E20_minus_E0": {str(N): float(low[N][19] - low[N][0]) for N in Ns},
                    "eig_max_residual": {str(N): resid[N] for N in Ns}})
    res.update({"states": a.states, "draws": a.draws, "t_grid": [float(t[0]), float(t[-1]), a.dt],
                "otoc_seconds": wall, "curves": len(keys) * a.states, "dtype": "c64"})
    print(json.dumps(res))


if __name__ == "__main__":
    main()
