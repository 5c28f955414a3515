"""Resumable curve files (paper_2002_05725_gb300/curves.py): host logic with a stand-in compute
function (no GPU): a second run loads every stored item and computes nothing; changed
settings, a changed time grid or a truncated file are recomputed; an interrupted run resumes."""
import os

import numpy as np
import pytest

from paper_2002_05725_gb300 import curves


class FakeCompute:
    def __init__(self, fail_after=None):
        self.calls = []
        self.fail_after = fail_after

    def __call__(self, specs, times, i, j, dtype, krylov_dim, tol, nworkers):
        if self.fail_after is not None and len(self.calls) >= self.fail_after:
            raise RuntimeError("interrupted")
        self.calls.append([dict(s) for s in specs])
        # a deterministic stand-in curve per item
        return [np.outer(np.asarray(times) + s["N"], np.arange(1, s["states"] + 1)) * (1 + 0.1j * s["beta"])
                for s in specs]


SPECS = [{"N": N, "seed": 7, "realization": r, "beta": b, "states": 2} for N in (20, 24) for r in (0, 1)
         for b in (1.0, 10.0)]
T = [0.0, 1.2, 2.4]


def test_second_run_loads_everything(tmp_path):
    fc = FakeCompute()
    F1, n1 = curves.run_otoc_items(SPECS, T, str(tmp_path), compute=fc, chunk=3)
    assert n1 == len(SPECS) and sum(len(c) for c in fc.calls) == len(SPECS)
    fc2 = FakeCompute()
    F2, n2 = curves.run_otoc_items(SPECS, T, str(tmp_path), compute=fc2)
    assert n2 == 0 and fc2.calls == []
    for a, b in zip(F1, F2):
        assert np.array_equal(a, b)
    assert len(os.listdir(tmp_path)) == len(SPECS)


def test_changed_settings_grid_or_bad_file_recomputed(tmp_path):
    curves.run_otoc_items(SPECS, T, str(tmp_path), compute=FakeCompute())
    fc = FakeCompute()
    _, n = curves.run_otoc_items(SPECS, T, str(tmp_path), tol=1e-9, compute=fc)
    assert n == len(SPECS)  # tolerance is part of the settings
    _, n = curves.run_otoc_items(SPECS, T + [3.6], str(tmp_path), tol=1e-9, compute=FakeCompute())
    assert n == len(SPECS)  # time grid changed
    path = curves.item_path(str(tmp_path), SPECS[0])
    with open(path, "wb") as f:
        f.write(b"truncated")
    fc = FakeCompute()
    _, n = curves.run_otoc_items(SPECS, T + [3.6], str(tmp_path), tol=1e-9, compute=fc)
    assert n == 1 and fc.calls[0][0] == SPECS[0]


def test_interrupted_run_resumes(tmp_path):
    with pytest.raises(RuntimeError):
        curves.run_otoc_items(SPECS, T, str(tmp_path), compute=FakeCompute(fail_after=2), chunk=3)
    assert len([f for f in os.listdir(tmp_path) if f.endswith(".npz") and ".tmp" not in f]) == 6
    fc = FakeCompute()
    F, n = curves.run_otoc_items(SPECS, T, str(tmp_path), compute=fc, chunk=3)
    assert n == len(SPECS) - 6
    ref, _ = curves.run_otoc_items(SPECS, T, str(tmp_path / "fresh"), compute=FakeCompute())
    for a, b in zip(F, ref):
        assert np.array_equal(a, b)
