"""Resumable curve files on the GPU: items computed through syk_otoc_batch are stored; a rerun
loads them without any H application, and the stored curves equal a direct syk_otoc call."""
import numpy as np
import pytest

from helpers import to_dev, torch_or_skip
from paper_2002_05725_gb300 import curves, inputs, syk

pytestmark = pytest.mark.gpu


def test_resumable_items_on_gpu(tmp_path):
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    specs = [{"N": 16, "seed": 3, "realization": 0, "beta": 2.0, "states": 2},
             {"N": 20, "seed": 3, "realization": 1, "beta": 5.0, "states": 4}]
    t = [0.0, 0.8, 2.0]
    syk.syk_counters(reset=True)
    F1, n1 = curves.run_otoc_items(specs, t, str(tmp_path), dtype=syk.SYK_C128, tol=1e-12)
    assert n1 == 2 and syk.syk_counters(reset=True)["h_applies"] > 0
    F2, n2 = curves.run_otoc_items(specs, t, str(tmp_path), dtype=syk.SYK_C128, tol=1e-12)
    assert n2 == 0 and syk.syk_counters(reset=True)["h_applies"] == 0
    for s, a, b in zip(specs, F1, F2):
        assert np.array_equal(a, b)
        terms = syk.syk_build_terms(s["N"], inputs.couplings(s["N"], seed=s["seed"], realization=s["realization"]))
        psi = inputs.random_states(s["N"], s["states"], seed=s["seed"], realization=s["realization"])
        ref = syk.syk_otoc(terms, s["beta"], 0, 1, t, to_dev(torch, psi, "c128"), krylov_dim=40, tol=1e-12)
        assert np.max(np.abs(a - ref)) <= 1e-10 * np.max(np.abs(ref))
