"""The one-state complex64 matvec (k_apply_one): every CTA width and cluster size the
autotuner can pick, both sectors, against the oracle's sector matrix (N = 24, 28) and its
term-by-term row sums (N = 40), and inside a Krylov evolution (Lanczos epilogue) at N = 28."""
import json

import numpy as np
import pytest

from helpers import TOL, rel, to_dev, torch_or_skip
from oracle import evolve, hamiltonian as hm
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


def _force(N, ntb, cs):
    syk.syk_autotune_reset()
    syk.syk_autotune_import(json.dumps({"apply_tiles": [
        {"N": N, "dtype": syk.SYK_C64, "batch": 1, "ntb": ntb, "cluster": cs, "variant": 0}]}))


@pytest.mark.parametrize("N", [24, 28])
@pytest.mark.parametrize("ntb,cs", [(6, 1), (7, 2), (8, 1), (8, 4), (6, 8)])
def test_one_state_full_vs_oracle(N, ntb, cs):
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    J = inputs.couplings(N, 40)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 1, 41)
    try:
        _force(N, ntb, cs)
        for sector in (0, 1):
            syk.syk_matvec_launches(reset=True)
            y = syk.syk_apply_H(terms, sector, to_dev(torch, psi, "c64")).cpu().numpy()
            mv = syk.syk_matvec_launches(reset=True)
            assert mv["tiled"] == 1 and mv["rows"] == 0, mv
            ref = hm.H_sector_sparse(N, J, sector) @ psi.T
            assert rel(y, ref) < TOL["c64"], (sector, rel(y, ref))
    finally:
        syk.syk_autotune_reset()


def test_one_state_sampled_rows_N40():
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    N = 40
    J = inputs.couplings(N, 42)
    terms = syk.syk_build_terms(N, J)
    D = 1 << (N // 2 - 1)
    psi = inputs.random_states(N, 1, 43)
    rng = np.random.default_rng(44)
    rows = np.unique(np.concatenate([[0, 1, D - 1], rng.integers(0, D, 21)]))
    for sector in (0, 1):
        y = syk.syk_apply_H(terms, sector, to_dev(torch, psi, "c64")).cpu().numpy()
        ref = hm.apply_rows(N, J, sector, psi.T, rows)
        assert rel(y[rows], ref) < TOL["c64"], sector


def test_one_state_in_krylov_evolution_N28():
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    N = 28
    J = inputs.couplings(N, 45)
    psi = inputs.random_states(N, 1, 46)
    out, _ = syk.syk_expmv(syk.syk_build_terms(N, J), 0, complex(-0.5, -3.0), to_dev(torch, psi, "c64"),
                           krylov_dim=40, tol=1e-7)
    ref = evolve.SectorSystem(N, J).expmv(complex(-0.5, -3.0), psi.T, 0)
    assert rel(out.cpu().numpy(), ref) < TOL["c64"]
