"""End-to-end parity on the matvec kernels the benchmark runs: G(t) and the regularized OTOC
through the tiled and coset matvecs (not the row kernel of small sectors), with Lanczos
segments replayed from captured CUDA graphs, against the exact oracle.

N = 24 (sector 2^11) is the smallest size at which every batch shape of the benchmark's path
has whole tiles: complex64 batches of 4, 8 and 16 states take the coset kernel with
thread-block clusters, complex128 batches of 1, 2 and 16 the tiled kernel.  The grid runs to
t = 12 at beta J = 10 like the benchmark's.  Tolerance per curve (Supp. Sec. I.B accuracy
measure, max over t): max_t |F~ - F~_oracle| / max_t |F~_oracle| <= 1e-10 (complex128) and
1e-5 (complex64), for every state.
"""
import json
import os

import numpy as np
import pytest

from helpers import TOL, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
N24, BETA = 24, 10.0
T_GRID = np.round(np.linspace(0.0, 12.0, 11), 12)


def curve_err(F, Fref):
    """Largest over states of max_t |F~ - F~ref| / max_t |F~ref|, F~ = F / F(0)."""
    a = F / F[0]
    b = Fref / Fref[0]
    return float(np.max(np.max(np.abs(a - b), axis=0) / np.max(np.abs(b), axis=0)))


def curve_err_raw(G, Gref):
    """Largest over states of max_t |G - Gref| / max_t |Gref| (no normalisation)."""
    return float(np.max(np.max(np.abs(G - Gref), axis=0) / np.max(np.abs(Gref), axis=0)))


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    syk.syk_use_graphs(True)
    return t


@pytest.fixture(scope="module")
def n24():
    """Couplings, 16 states and the oracle's F and G curves at N = 24 (dense eigh)."""
    J = inputs.couplings(N24, 0)
    psi = inputs.random_states(N24, 16, 0)
    sysm = evolve.SectorSystem(N24, J)
    F = co.F_state(sysm, BETA, 0, 1, T_GRID, psi.T)
    G, Z = co.G_state(sysm, 5.0, 2, T_GRID, psi.T)
    return {"J": J, "psi": psi, "F": F, "G": G, "Z": Z, "terms": syk.syk_build_terms(N24, J)}


def _otoc_twice(torch, terms, x, tol):
    """Two identical calls: the second replays the Lanczos segments captured during the first."""
    syk.syk_matvec_launches(reset=True)
    a = syk.syk_otoc(terms, BETA, 0, 1, T_GRID, x, krylov_dim=40, tol=tol)
    b = syk.syk_otoc(terms, BETA, 0, 1, T_GRID, x, krylov_dim=40, tol=tol)
    return a, b, syk.syk_matvec_launches(reset=True)


@pytest.mark.parametrize("B", [16, 8, 4])
def test_otoc_N24_c64_coset_path(torch, n24, B):
    """complex64 with FP64 scalars on the benchmark's default kernel (coset, cluster split)."""
    syk.syk_autotune_reset()
    x = to_dev(torch, n24["psi"][:B], "c64")
    a, b, mv = _otoc_twice(torch, n24["terms"], x, 1e-7)
    assert mv["coset"] > 0 and mv["rows"] == 0, mv
    assert np.array_equal(a, b)  # graph replay is bit-identical to the eager first call
    assert curve_err(a, n24["F"][:, :B]) < TOL["c64"]


@pytest.mark.parametrize("shape", [
    {"ntb": 6, "cluster": 1, "variant": 1},
    {"ntb": 6, "cluster": 4, "variant": 1},
    {"ntb": 7, "cluster": 2, "variant": 1},
    {"ntb": 6, "cluster": 8, "variant": 2},
    {"ntb": 6, "cluster": 2, "variant": 0},
])
def test_otoc_N24_c64_16_states_every_launch_shape(torch, n24, shape):
    """The 16-state curves through each launch shape the autotuner can choose (CTA width,
    cluster size, coset rows per thread or the plain tiled kernel)."""
    entry = dict(N=N24, dtype=syk.SYK_C64, batch=16, ms=0.0, **shape)
    syk.syk_autotune_reset()
    syk.syk_autotune_import(json.dumps({"apply_tiles": [entry]}))
    try:
        x = to_dev(torch, n24["psi"], "c64")
        a, b, mv = _otoc_twice(torch, n24["terms"], x, 1e-7)
    finally:
        syk.syk_autotune_reset()
    assert mv["rows"] == 0 and mv["coset" if shape["variant"] else "tiled"] > 0, mv
    assert np.array_equal(a, b)
    assert curve_err(a, n24["F"]) < TOL["c64"]


@pytest.mark.parametrize("B", [1, 2, 16])
def test_otoc_N24_c128_tiled_path(torch, n24, B):
    """complex128 (the paper's precision) on the tiled kernel, within 1e-10 per curve."""
    syk.syk_autotune_reset()
    x = to_dev(torch, n24["psi"][:B], "c128")
    a, b, mv = _otoc_twice(torch, n24["terms"], x, 1e-12)
    assert mv["tiled"] > 0 and mv["rows"] == 0, mv
    assert np.array_equal(a, b)
    assert curve_err(a, n24["F"][:, :B]) < TOL["c128"]


@pytest.mark.parametrize("dt,B", [("c64", 16), ("c128", 2)])
def test_G_N24_tile_paths(torch, n24, dt, B):
    syk.syk_autotune_reset()
    syk.syk_matvec_launches(reset=True)
    G, Z = syk.syk_correlator_G(n24["terms"], 5.0, 2, T_GRID, to_dev(torch, n24["psi"][:B], dt), krylov_dim=40,
                                tol=1e-12 if dt == "c128" else 1e-7)
    mv = syk.syk_matvec_launches(reset=True)
    assert mv["rows"] == 0 and mv["coset" if dt == "c64" else "tiled"] > 0, mv
    assert curve_err_raw(G, n24["G"][:, :B]) < TOL[dt]
    assert float(np.max(np.abs(Z - n24["Z"][:B]) / n24["Z"][:B])) < TOL[dt]


@pytest.fixture(scope="module")
def n28():
    with open(os.path.join(HERE, "golden", "oracle_N28_curves.json")) as f:
        g = json.load(f)
    cplx = lambda v: np.array([[complex(*z) for z in col] for col in v]).T  # (nt, B)
    return {"J": inputs.couplings(g["N"], g["seed"]), "psi": inputs.random_states(g["N"], g["nstates"], g["seed"]),
            "t": np.array(g["t"]), "F": cplx(g["F"]["values"]), "G": cplx(g["G"]["values"]),
            "Z": np.array(g["G"]["Z"]), "betaF": g["F"]["beta"], "betaG": g["G"]["beta"], "iG": g["G"]["i"]}


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_otoc_and_G_N28_vs_expm_multiply_oracle(torch, n28, dt):
    """N = 28 (sector 2^13), two states, t = 0, 3, 6, 12: the oracle's curves from scipy's
    expm_multiply (stored by tests/golden/make_oracle_curves.py, which calls only the oracle)."""
    syk.syk_autotune_reset()
    terms = syk.syk_build_terms(28, n28["J"])
    x = to_dev(torch, n28["psi"], dt)
    tol = 1e-12 if dt == "c128" else 1e-7
    syk.syk_matvec_launches(reset=True)
    F = syk.syk_otoc(terms, n28["betaF"], 0, 1, n28["t"], x, krylov_dim=40, tol=tol)
    G, Z = syk.syk_correlator_G(terms, n28["betaG"], n28["iG"], n28["t"], x, krylov_dim=40, tol=tol)
    mv = syk.syk_matvec_launches(reset=True)
    assert mv["rows"] == 0, mv
    assert curve_err(F, n28["F"]) < TOL[dt]
    assert curve_err_raw(G, n28["G"]) < TOL[dt]
    assert float(np.max(np.abs(Z - n28["Z"]) / n28["Z"])) < TOL[dt]


def test_otoc_N40_bench_shape_c64_vs_c128(torch):
    """The benchmark's own shape at full size: N = 40 (sector 2^19), 16 states, beta J = 10,
    Krylov dimension 40, t = 0 and 12 (the end of the benchmark's grid): the complex64 coset
    path with FP64 scalars against the complex128 tiled path, per curve within 1e-5."""
    N = 40
    syk.syk_autotune_reset()
    terms = syk.syk_build_terms(N, inputs.couplings(N, 0))
    psi = inputs.random_states(N, 16, 0)
    ts = [0.0, 12.0]
    syk.syk_matvec_launches(reset=True)
    b = syk.syk_otoc(terms, BETA, 0, 1, ts, to_dev(torch, psi, "c64"), krylov_dim=40, tol=1e-7)
    mv = syk.syk_matvec_launches(reset=True)
    a = syk.syk_otoc(terms, BETA, 0, 1, ts, to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
    assert mv["coset"] > 0 and mv["rows"] == 0, mv
    assert curve_err(b, a) < TOL["c64"]
    assert np.allclose(b[0] / b[0], 1.0)
