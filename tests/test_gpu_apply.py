"""K1 (apply_H) and K5 (apply_chi) on the GPU against the CPU oracle."""
import numpy as np
import pytest

from helpers import TOL, rel, tdtype, to_dev, torch_or_skip
from oracle import hamiltonian as hm
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    return t


@pytest.mark.parametrize("N", [4, 8, 12, 16, 20])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_H_vs_oracle_full(torch, N, dt):
    J = inputs.couplings(N, 21)
    terms = syk.syk_build_terms(N, J)
    for sector in (0, 1):
        H = hm.H_sector_sparse(N, J, sector)
        for B in (1, 3, 19):
            psi = inputs.random_states(N, B, 100 + B)
            ref = H @ psi.T
            y = syk.syk_apply_H(terms, sector, to_dev(torch, psi, dt))
            assert rel(y.cpu().numpy(), ref) < TOL[dt], (N, sector, B)


@pytest.mark.parametrize("N", [28, 32, 40])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_H_sampled_rows(torch, N, dt):
    """Brute force over all C(N,4) terms on sampled rows (first, last, random)."""
    J = inputs.couplings(N, 5)
    terms = syk.syk_build_terms(N, J)
    D = 1 << (N // 2 - 1)
    psi = inputs.random_states(N, 2, 7)
    rng = np.random.default_rng(N)
    rows = np.unique(np.concatenate([[0, 1, D - 1], rng.integers(0, D, 21)]))
    for sector in (0, 1):
        y = syk.syk_apply_H(terms, sector, to_dev(torch, psi, dt)).cpu().numpy()
        ref = hm.apply_rows(N, J, sector, psi.T, rows)
        assert rel(y[rows], ref) < TOL[dt], (N, sector)


def test_apply_H_sampled_rows_N60(torch):
    """N = 60, even sector of dimension 2^29, complex64 (4 GiB per vector)."""
    N = 60
    J = inputs.couplings(N, 1)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states_device(N, 1, 60, "cuda", torch.complex64)
    y = syk.syk_apply_H(terms, 0, psi)
    torch.cuda.synchronize()
    rng = np.random.default_rng(60)
    D = 1 << (N // 2 - 1)
    rows = np.concatenate([[0, D - 1], rng.integers(0, D, 6)])
    m = hm.flip_mask(hm.quadruples(N))
    ys = y[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    for r, c in enumerate(rows):
        x = int(hm.full_index(N, 0, c))
        src = np.unique((np.int64(x) ^ m) & (D - 1))
        vals = psi[torch.as_tensor(src, device="cuda"), 0].cpu().numpy().astype(np.complex128)
        full = np.zeros(1, dtype=np.complex128)
        # oracle row over all terms, reading psi only at the sources it gathers
        lookup = dict(zip(src.tolist(), vals.tolist()))
        srcs = (np.int64(x) ^ m) & (D - 1)
        amp, xo = hm.term_action(hm.quadruples(N), np.int64(x) ^ m)
        assert np.all(xo == x)
        full[0] = np.sum(J * amp * np.array([lookup[s] for s in srcs.tolist()]))
        assert abs(ys[r, 0] - full[0]) < 4e-5 * max(1.0, abs(full[0])), (r, ys[r, 0], full[0])


def test_apply_H_hermitian(torch):
    N = 32
    J = inputs.couplings(N, 9)
    terms = syk.syk_build_terms(N, J)
    a = to_dev(torch, inputs.random_states(N, 3, 1), "c128")
    b = to_dev(torch, inputs.random_states(N, 3, 2), "c128")
    Ha = syk.syk_apply_H(terms, 0, a)
    Hb = syk.syk_apply_H(terms, 0, b)
    lhs = (a.conj() * Hb).sum(0)
    rhs = (Ha.conj() * b).sum(0)
    assert torch.max(torch.abs(lhs - rhs)).item() < 1e-11 * torch.max(torch.abs(lhs)).item()
    # <psi|H^2|psi>/<psi|psi> = sum J^2/16 up to the typicality error ~ D^{-1/2}
    e2 = (Ha.abs() ** 2).sum(0) / (a.abs() ** 2).sum(0)
    assert np.allclose(e2.cpu().numpy(), np.sum(J ** 2) / 16, rtol=0.05)


@pytest.mark.parametrize("N", [4, 12, 20])
@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_apply_chi_vs_oracle(torch, N, dt):
    psi = inputs.random_states(N, 3, 4)
    for sector in (0, 1):
        for i in range(N):
            ref = hm.chi_sector_sparse(N, i, sector) @ psi.T
            y = syk.syk_apply_chi(N, i, sector, to_dev(torch, psi, dt))
            assert rel(y.cpu().numpy(), ref) < (1e-15 if dt == "c128" else 1e-7), (i, sector)


def test_apply_chi_squares_to_half(torch):
    N = 36
    psi = inputs.random_states_device(N, 2, 3, "cuda", torch.complex128)
    for i in (0, 17, 35):
        y = syk.syk_apply_chi(N, i, 1, syk.syk_apply_chi(N, i, 0, psi))
        assert torch.max(torch.abs(y - psi / 2)).item() < 1e-15


def test_apply_H_invalid_args(torch):
    terms = syk.syk_build_terms(8, inputs.couplings(8, 0))
    psi = torch.zeros((8, 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(syk.SykError):
        syk.syk_apply_H(terms, 2, psi)
    with pytest.raises(syk.SykError):
        syk.syk_apply_H(terms, 0, psi[:, :0])


@pytest.mark.parametrize("dt,B", [("c64", 8), ("c64", 1), ("c128", 2)])
def test_apply_H_every_tile_configuration(torch, dt, B):
    """Every CTA width x cluster size of the tiled matvec (forced through the tuning table)
    against the oracle, then the autotuner's own choice and its JSON round trip."""
    N = 24
    J = inputs.couplings(N, 3)
    terms = syk.syk_build_terms(N, J)
    code = syk.SYK_C64 if dt == "c64" else syk.SYK_C128
    psi = inputs.random_states(N, B, 77)
    x = to_dev(torch, psi, dt)
    D = 1 << (N // 2 - 1)
    rows = np.unique(np.concatenate([[0, D - 1], np.random.default_rng(1).integers(0, D, 40)]))
    ref = hm.apply_rows(N, J, 0, psi.T, rows)
    for ntb in (6, 7, 8):
        for cs in (1, 2, 4, 8):
            syk.syk_autotune_import('{"apply_tiles": [{"N": %d, "dtype": %d, "batch": %d, "ntb": %d, "cluster": %d}]}'
                                    % (N, code, B, ntb, cs))
            y = syk.syk_apply_H(terms, 0, x).cpu().numpy().reshape(D, B)
            assert rel(y[rows], ref.reshape(len(rows), B)) < TOL[dt], (ntb, cs)
    best = syk.syk_autotune_apply(terms, code, B)
    assert best > 0
    js = syk.syk_autotune_export()
    assert '"N": 24' in js
    syk.syk_autotune_import(js)
    y = syk.syk_apply_H(terms, 0, x).cpu().numpy().reshape(D, B)
    assert rel(y[rows], ref.reshape(len(rows), B)) < TOL[dt]


@pytest.mark.parametrize("B,variants", [(16, (1, 2)), (8, (2, 3)), (4, (2, 3))])
def test_apply_H_coset_variants(torch, B, variants):
    """complex64 coset kernels (2, 4 or 8 rows per thread) at every CTA width x cluster size:
    full H at N = 20 (one or two tiles; both sectors) and sampled rows at N = 28."""
    code = syk.SYK_C64
    for N in (20, 28):
        J = inputs.couplings(N, 9)
        terms = syk.syk_build_terms(N, J)
        D = 1 << (N // 2 - 1)
        psi = inputs.random_states(N, B, 31)
        x = to_dev(torch, psi, "c64")
        rows = np.arange(D) if N == 20 else \
            np.unique(np.concatenate([[0, D - 1], np.random.default_rng(2).integers(0, D, 48)]))
        for sector in (0, 1):
            ref = hm.H_sector_sparse(N, J, sector) @ psi.T if N == 20 else hm.apply_rows(N, J, sector, psi.T, rows)
            for var in variants:
                for ntb in (6, 7, 8):
                    if (1 << var) << ntb > D:
                        continue
                    for cs in (1, 2, 4, 8):
                        syk.syk_autotune_import(
                            '{"apply_tiles": [{"N": %d, "dtype": %d, "batch": %d, "ntb": %d, "cluster": %d, '
                            '"variant": %d}]}' % (N, code, B, ntb, cs, var))
                        y = syk.syk_apply_H(terms, sector, x).cpu().numpy().reshape(D, B)
                        assert rel(y[rows], ref.reshape(len(rows), B)) < TOL["c64"], (N, sector, var, ntb, cs)
        best = syk.syk_autotune_apply(terms, code, B)
        assert best > 0
    syk.syk_autotune_import('{"apply_tiles": [{"N": 28, "dtype": 1, "batch": %d, "ntb": 8, "cluster": 1}]}' % B)


def test_apply_H_bench_size_launch_shapes(torch):
    """The benchmark's matvec at full size (N = 40, sector 2^19, 16 states, complex64) in the
    launch shapes it runs: the untuned default, the coset shapes the autotuner picks on GB300
    (2 rows per thread, 128-thread CTAs, cluster 1 and 2), the 4-row coset shape and the plain
    tiled kernel; sampled rows (first, last, random) against the oracle's term-by-term sum."""
    N, B = 40, 16
    J = inputs.couplings(N, 0)
    terms = syk.syk_build_terms(N, J)
    D = 1 << (N // 2 - 1)
    psi = inputs.random_states(N, B, 0)
    x = to_dev(torch, psi, "c64")
    rows = np.unique(np.concatenate([[0, 1, D - 1], np.random.default_rng(40).integers(0, D, 21)]))
    shapes = [None, (7, 1, 1), (7, 2, 1), (6, 1, 2), (6, 1, 0)]
    for sector in (0, 1):
        ref = hm.apply_rows(N, J, sector, psi.T, rows)
        for sh in shapes:
            syk.syk_autotune_reset()  # None: the built-in default shape
            if sh is not None:
                ntb, cs, var = sh
                syk.syk_autotune_import('{"apply_tiles": [{"N": 40, "dtype": 1, "batch": 16, "ntb": %d, '
                                        '"cluster": %d, "variant": %d}]}' % (ntb, cs, var))
            y = syk.syk_apply_H(terms, sector, x).cpu().numpy().reshape(D, B)
            assert rel(y[rows], ref.reshape(len(rows), B)) < TOL["c64"], (sector, sh)
    syk.syk_autotune_reset()


@pytest.mark.parametrize("B", [1, 8, 16])
def test_apply_H_misaligned_vectors(torch, B):
    """Vectors that start 8 bytes past a 16-byte boundary (views into a larger buffer): the
    bulk-copy kernels need 16-byte alignment and decline, the row kernel computes the result."""
    N = 20
    J = inputs.couplings(N, 8)
    terms = syk.syk_build_terms(N, J)
    D = 1 << (N // 2 - 1)
    psi = inputs.random_states(N, B, 12)
    big = torch.zeros(D * B + 1, dtype=torch.complex64, device="cuda")
    x = big[1:].view(D, B)
    x.copy_(to_dev(torch, psi, "c64").view(D, B))
    ybig = torch.zeros(D * B + 1, dtype=torch.complex64, device="cuda")
    y = ybig[1:].view(D, B)
    assert x.data_ptr() % 16 == 8 and y.data_ptr() % 16 == 8
    syk.syk_apply_H(terms, 0, x, out=y)
    ref = hm.H_sector_sparse(N, J, 0) @ psi.T
    assert rel(y.cpu().numpy().reshape(D, B), ref.reshape(D, B)) < TOL["c64"]
