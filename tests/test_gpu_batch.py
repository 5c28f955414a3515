"""The batched workload: mixed-N items on concurrent streams match single calls and the oracle
(every item, N = 12 to 24)."""
import numpy as np
import pytest

from helpers import rel, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_otoc_batch_mixed_N(dt):
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    code = syk.SYK_C128 if dt == "c128" else syk.SYK_C64
    tol = 1e-12 if dt == "c128" else 1e-7
    ts = [0.0, 0.8, 2.0, 3.5]
    items, refs = [], []
    for k, (N, beta) in enumerate([(12, 1.0), (16, 3.0), (20, 10.0), (12, 10.0), (24, 3.0), (16, 1.0)]):
        J = inputs.couplings(N, seed=3, realization=k)
        psi = inputs.random_states(N, 2 if N != 24 else 8, seed=3, realization=k)
        terms = syk.syk_build_terms(N, J)
        x = to_dev(torch, psi, dt) if k % 2 == 0 else np.ascontiguousarray(
            psi.T.astype(np.complex128 if dt == "c128" else np.complex64))   # device and host inputs
        items.append((terms, beta, x))
        single = syk.syk_otoc(terms, beta, 0, 1, ts, x, krylov_dim=30, tol=tol)
        refs.append((single, N, J, beta, psi))
    out = syk.syk_otoc_batch(items, 0, 1, ts, dtype=code, krylov_dim=30, tol=tol, nworkers=3)
    for F, (single, N, J, beta, psi) in zip(out, refs):
        # complex64 items run in the persistent launch, whose convergence checks follow their own
        # plan: the two evaluations agree to a few tol = 1e-7 Krylov steps
        assert rel(F, single) < (1e-12 if dt == "c128" else 5e-6)
        # every item against the exact oracle, the N = 20 and 24 items (tiled and coset
        # matvecs) included
        Fr = co.F_state(evolve.SectorSystem(N, J), beta, 0, 1, ts, psi.T)
        assert rel(F / F[0], Fr / Fr[0]) < (1e-10 if dt == "c128" else 1e-5), N


def test_otoc_batch_reports_item_errors():
    torch_or_skip()
    syk.load(build_if_missing=True)
    terms = syk.syk_build_terms(12, inputs.couplings(12, 0))
    psi = np.zeros((32, 1), dtype=np.complex64)
    with pytest.raises(syk.SykError):
        syk.syk_otoc_batch([(terms, -1.0, psi)], 0, 1, [0.0], dtype=syk.SYK_C64)


def test_graph_replay_matches_eager():
    """Lanczos segments replayed from captured CUDA graphs give the same numbers as eager launches."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    N = 16
    terms = syk.syk_build_terms(N, inputs.couplings(N, 8))
    x = to_dev(torch, inputs.random_states(N, 4, 8), "c128")
    ts = [0.0, 0.5, 1.5, 4.0]
    syk.syk_use_graphs(False)
    eager = syk.syk_otoc(terms, 2.0, 0, 1, ts, x, krylov_dim=30, tol=1e-12)
    syk.syk_use_graphs(True)
    syk.syk_counters(reset=True)
    g1 = syk.syk_otoc(terms, 2.0, 0, 1, ts, x, krylov_dim=30, tol=1e-12)   # captures within the call
    c1 = syk.syk_counters(reset=True)
    g2 = syk.syk_otoc(terms, 2.0, 0, 1, ts, x, krylov_dim=30, tol=1e-12)
    c2 = syk.syk_counters(reset=True)
    assert np.array_equal(g1, eager) and np.array_equal(g2, eager)
    assert c1["h_applies"] == c2["h_applies"] and c1["launches"] == c2["launches"]
