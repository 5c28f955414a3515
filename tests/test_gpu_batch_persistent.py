"""The persistent batched launch (one CTA per small-sector item, the whole OTOC chain on the
device): every item against the exact oracle (Eq. F_reg by Eq. q_typicality), against the
per-item path of the same batch, mixed with items that take the per-item path, and its
error report."""
import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


def _items(torch, spec, seed):
    items, raw = [], []
    for k, (N, B, beta) in enumerate(spec):
        J = inputs.couplings(N, seed=seed, realization=k)
        psi = inputs.random_states(N, B, seed=seed, realization=k)
        terms = syk.syk_build_terms(N, J)
        # device inputs for even items, host inputs for odd ones
        x = to_dev(torch, psi, "c64") if k % 2 == 0 else np.ascontiguousarray(psi.T.astype(np.complex64))
        items.append((terms, beta, x))
        raw.append((N, J, beta, psi))
    return items, raw


@pytest.fixture
def persistent_on():
    prev = syk.syk_batch_persistent(syk.BATCH_PERSISTENT)
    yield
    syk.syk_batch_persistent(prev)


@pytest.fixture
def persistent_split():
    """Items split over several CTAs go to the persistent launch whatever the batch size."""
    prev = syk.syk_batch_persistent(syk.BATCH_PERSISTENT_SPLIT_ALWAYS)
    yield
    syk.syk_batch_persistent(prev)


# (N, states, beta J): every batch size the kernel is built for, sectors of 2^5 to 2^11 rows
SPEC = [(24, 8, 10.0), (20, 16, 3.0), (16, 1, 1.0), (12, 2, 10.0), (20, 4, 1.0), (24, 2, 3.0), (16, 8, 5.0)]


def test_persistent_items_vs_oracle(persistent_on):
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    ts = [0.0, 0.7, 2.0, 4.5]
    items, raw = _items(torch, SPEC, seed=11)
    out = syk.syk_otoc_batch(items, 0, 1, ts, dtype=syk.SYK_C64, krylov_dim=30, tol=1e-7, nworkers=2)
    rep = syk.syk_batch_report()
    assert rep["persistent_items"] == len(SPEC) and rep["stream_items"] == 0, rep
    assert rep["h_applies"] > 0 and rep["cycles_matvec"] > 0
    for F, (N, J, beta, psi) in zip(out, raw):
        Fr = co.F_state(evolve.SectorSystem(N, J), beta, 0, 1, ts, psi.T)
        assert rel(F / F[0], Fr / Fr[0]) < TOL["c64"], (N, psi.shape[0], beta, rel(F / F[0], Fr / Fr[0]))
        assert rel(F, Fr) < TOL["c64"], (N, rel(F, Fr))


def test_persistent_matches_per_item_path_on_the_bench_grid(persistent_on):
    """N = 20 and 24 items at beta J = 10 on the benchmark's grid (t = 0 and 10 points to 12,
    Krylov 40): the persistent launch and the per-item streams agree, and both the oracle."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    ts = [0.0] + [1.2 * k for k in range(1, 11)]
    spec = [(24, 8, 10.0), (20, 8, 10.0)]
    items, raw = _items(torch, spec, seed=5)
    pers = syk.syk_otoc_batch(items, 0, 1, ts, dtype=syk.SYK_C64, krylov_dim=40, tol=1e-7)
    assert syk.syk_batch_report()["persistent_items"] == 2
    syk.syk_batch_persistent(False)
    streams = syk.syk_otoc_batch(items, 0, 1, ts, dtype=syk.SYK_C64, krylov_dim=40, tol=1e-7)
    rep = syk.syk_batch_report()
    assert rep["persistent_items"] == 0 and rep["stream_items"] == 2
    for Fp, Fs, (N, J, beta, psi) in zip(pers, streams, raw):
        # two complex64 evaluations with their own convergence-check plans, each step within
        # tol = 1e-7 of the exact exponential
        assert rel(Fp, Fs) < 5e-6, (N, rel(Fp, Fs))
        Fr = co.F_state(evolve.SectorSystem(N, J), beta, 0, 1, ts, psi.T)
        assert rel(Fp / Fp[0], Fr / Fr[0]) < TOL["c64"], (N, rel(Fp / Fp[0], Fr / Fr[0]))


def test_persistent_and_per_item_items_in_one_batch(persistent_split):
    """A batch mixing items for the persistent launch -- N = 28 at 8 states is split into four
    CTAs of 2 states, whose 2^13 x 2 sector vectors fit shared memory -- with one it cannot
    take (N = 32 at 8 states: 2^14 rows per state even one state per CTA would exceed it),
    which runs on the per-item streams concurrently."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    ts = [0.0, 1.0, 3.0]
    spec = [(32, 8, 3.0), (28, 8, 3.0), (20, 8, 3.0), (24, 4, 1.0)]
    items, raw = _items(torch, spec, seed=2)
    out = syk.syk_otoc_batch(items, 0, 1, ts, dtype=syk.SYK_C64, krylov_dim=30, tol=1e-7, nworkers=2)
    rep = syk.syk_batch_report()
    assert rep["persistent_items"] == 3 and rep["stream_items"] == 1, rep
    assert rep["persistent_subitems"] == 4 + 1 + 1, rep
    for F, (terms, beta, x), (N, J, _, psi) in zip(out, items, raw):
        single = syk.syk_otoc(terms, beta, 0, 1, ts, x, krylov_dim=30, tol=1e-7)
        assert rel(F, single) < 5e-6, (N, rel(F, single))
        if N <= 24:
            Fr = co.F_state(evolve.SectorSystem(N, J), beta, 0, 1, ts, psi.T)
            assert rel(F / F[0], Fr / Fr[0]) < TOL["c64"], N


def _golden_n28():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_N28_curves.json")) as f:
        g = json.load(f)
    F = np.array(g["F"]["values"])  # (state, t, re/im)
    return g, (F[..., 0] + 1j * F[..., 1]).T  # (t, state)


@pytest.mark.parametrize("B", [2, 8])
def test_persistent_N28_vs_stored_oracle_curves(persistent_split, B):
    """N = 28 (sector 2^13), beta J = 10, t = 0, 3, 6, 12 against the oracle's expm_multiply
    curves stored by tests/golden/make_oracle_curves.py: 2 states (one CTA) and 8 states (four
    CTAs of 2; the stored states are the first two of the seeded draw)."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    g, Fref = _golden_n28()
    J = inputs.couplings(28, g["seed"])
    psi = inputs.random_states(28, B, g["seed"])
    terms = syk.syk_build_terms(28, J)
    F = syk.syk_otoc_batch([(terms, g["F"]["beta"], to_dev(torch, psi, "c64"))], 0, 1, g["t"], dtype=syk.SYK_C64,
                           krylov_dim=40, tol=1e-7)[0]
    rep = syk.syk_batch_report()
    assert rep["persistent_items"] == 1 and rep["persistent_subitems"] == B // 2, rep
    for s in range(2):
        err = np.max(np.abs(F[:, s] - Fref[:, s])) / np.max(np.abs(Fref[:, s]))
        assert err < TOL["c64"], (B, s, err)


def test_persistent_reports_non_finite_items(persistent_on):
    """A state with a NaN amplitude makes its item's Lanczos scalars non-finite: that item's
    status is SYK_ENUMERIC, the call fails with its message, the other item is unaffected."""
    torch = torch_or_skip()
    lib = syk.load(build_if_missing=True)
    ts = [0.0, 1.0]
    N = 16
    good = inputs.random_states(N, 4, seed=1)
    bad = good.copy()
    bad[2, 5] = np.nan
    terms = syk.syk_build_terms(N, inputs.couplings(N, 1))
    items = [(terms, 1.0, to_dev(torch, good, "c64")), (terms, 1.0, to_dev(torch, bad, "c64"))]
    import ctypes
    arr = (syk._OtocItem * 2)()
    Fs = [np.zeros((len(ts), 4, 2)) for _ in range(2)]
    for k, (tm, beta, x) in enumerate(items):
        arr[k] = syk._OtocItem(tm.ptr.value, beta, x.data_ptr(), 4, Fs[k].ctypes.data)
    status = np.zeros(2, dtype=np.int32)
    t = np.asarray(ts, dtype=np.float64)
    rc = lib.syk_otoc_batch(ctypes.cast(arr, ctypes.c_void_p), 2, 0, 1, t.ctypes.data, len(t), syk.SYK_C64, 20,
                            1e-7, 1, status.ctypes.data)
    assert rc == syk.SYK_ENUMERIC and b"non-finite" in lib.syk_last_error()
    assert status[0] == syk.SYK_OK and status[1] == syk.SYK_ENUMERIC
    assert syk.syk_batch_report()["persistent_items"] == 2
    Fr = co.F_state(evolve.SectorSystem(N, inputs.couplings(N, 1)), 1.0, 0, 1, ts, good.T)
    F0 = Fs[0][..., 0] + 1j * Fs[0][..., 1]
    assert rel(F0, Fr) < TOL["c64"]


def test_split_items_stay_on_streams_in_small_batches(persistent_on):
    """In the default mode a lone N = 28 item of 8 states (four CTAs of 2 states, far fewer
    than half the SMs) takes the per-item path, while an N = 24 item of 8 states (one CTA)
    takes the persistent launch."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    items, _ = _items(torch, [(28, 8, 1.0), (24, 8, 1.0)], seed=4)
    syk.syk_otoc_batch(items, 0, 1, [0.0, 0.5], dtype=syk.SYK_C64, krylov_dim=30, tol=1e-7)
    rep = syk.syk_batch_report()
    assert rep["persistent_items"] == 1 and rep["stream_items"] == 1 and rep["persistent_subitems"] == 1, rep
