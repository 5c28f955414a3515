"""Finite-size rescaling pipeline on GPU curves against the same analysis on the oracle's curves."""
import numpy as np
import pytest

from helpers import torch_or_skip
from oracle import correlators as co, evolve
from paper_2002_05725_gb300 import inputs, rescale, syk

pytestmark = pytest.mark.gpu


def test_rescaling_pipeline_vs_oracle_curves():
    """N = 12, 14, 16 at beta J = 1, two coupling draws x 3 states each, through the batched
    GPU workload (complex64) and through the oracle's exact chain: disorder averages, crossing
    times t*(N) of F~ = 0.75, lambda_fit and the linear extrapolation agree."""
    torch = torch_or_skip()
    syk.load(build_if_missing=True)
    Ns, beta, draws, B = [12, 14, 16], 1.0, 2, 3
    t = np.round(np.arange(0.0, 8.0001, 0.1), 12)
    items, keys, ref = [], [], {N: [] for N in Ns}
    for N in Ns:
        for r in range(draws):
            J = inputs.couplings(N, seed=3, realization=r)
            psi = inputs.random_states(N, B, 3, r)
            items.append((syk.syk_build_terms(N, J), beta,
                          torch.from_numpy(np.ascontiguousarray(psi.T)).to(torch.complex64).cuda()))
            keys.append(N)
            ref[N].append(co.F_state(evolve.SectorSystem(N, J), beta, 0, 1, t, psi.T))
    Fs = syk.syk_otoc_batch(items, 0, 1, t, syk.SYK_C64, 40, 1e-7)
    gpu = {N: rescale.disorder_average([F for F, k in zip(Fs, keys) if k == N]) for N in Ns}
    ora = {N: rescale.disorder_average(ref[N]) for N in Ns}
    for N in Ns:
        assert np.abs(gpu[N] - ora[N]).max() < 1e-5
    a = rescale.lyapunov(Ns, t, gpu, beta)
    b = rescale.lyapunov(Ns, t, ora, beta)
    assert np.allclose(a["t_star"], b["t_star"], rtol=1e-4)
    assert np.allclose(a["lambda_fit"], b["lambda_fit"], rtol=1e-3)
    # a two-point extrapolation to 1/N = 0 magnifies lambda_fit differences about 8x here
    assert abs(a["lambda"] - b["lambda"]) < 5e-3 * max(1.0, abs(b["lambda"]))
