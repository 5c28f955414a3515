"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics.

Every oracle function is checked here against something other than itself:
closed forms, algebraic identities, special cases with known spectra,
library routines for special cases, and brute-force alternatives.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import capply, correlators as co, evolve, hamiltonian as hm, jw
from paper_2002_05725_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- Majoranas

@pytest.mark.parametrize("N", [4, 8, 10])
def test_anticommutation(N):
    """{chi_a, chi_b} = delta_ab (Eq. 1 normalisation) for the JW map of Supp. Sec. I.A."""
    chis = [jw.chi_dense(N, i) for i in range(N)]
    eye = np.eye(chis[0].shape[0])
    for a in range(N):
        for b in range(N):
            ac = chis[a] @ chis[b] + chis[b] @ chis[a]
            assert np.abs(ac - (a == b) * eye).max() < 1e-14
        assert np.abs(chis[a] - chis[a].conj().T).max() == 0.0      # Hermitian


def test_chi_basis_matches_dense():
    N = 10
    x = np.arange(1 << (N // 2))
    for i in range(N):
        M = jw.chi_dense(N, i)
        amp, xo = jw.chi_basis(np.full(len(x), i), x)
        T = np.zeros_like(M)
        T[xo, x] = amp
        assert np.abs(T - M).max() < 1e-15


def test_jw_example_N4():
    """N=4: chi0 chi1 chi2 chi3 = -(1/4) Z_0 Z_1, so H = J P has eigenvalues +-J/4."""
    m, z, p = hm.term_table(4)
    assert (int(m[0]), int(z[0]), int(p[0])) == (0, 3, 2)
    J = np.array([0.7])
    ev = np.linalg.eigvalsh(hm.H_dense(4, J))
    assert np.allclose(np.sort(ev), [-0.175, -0.175, 0.175, 0.175], atol=1e-15)


# ----------------------------------------------------------------------------- H

def test_H_hermitian_and_parity():
    N = 10
    H = hm.H_dense(N, inputs.couplings(N, 5))
    assert np.abs(H - H.conj().T).max() == 0.0
    par = np.array([bin(v).count("1") & 1 for v in range(H.shape[0])])
    assert np.abs(H[np.ix_(par == 0, par == 1)]).max() == 0.0


@pytest.mark.parametrize("N", [8, 12])
def test_trace_H2_closed_form(N):
    """Distinct Majorana quartets are trace-orthogonal and (chi_i chi_j chi_k chi_l)^2 = 1/16,
    so Tr H^2 / 2^n = sum J^2 / 16 exactly (Eq. 1 with {chi_i, chi_j} = delta_ij)."""
    J = inputs.couplings(N, 2)
    if N <= 10:
        H = hm.H_dense(N, J)
        val = np.trace(H @ H).real / H.shape[0]
    else:
        val = sum(np.sum(np.abs(hm.H_sector_sparse(N, J, s).toarray()) ** 2) for s in (0, 1)) \
            / (1 << (N // 2))
    assert abs(val - np.sum(J ** 2) / 16) < 1e-14 * max(1.0, val)


def test_term_table_vs_dense_products():
    """Pauli form i^p X^m Z^z of 4 chi_i chi_j chi_k chi_l against dense Kronecker products."""
    N = 8
    n = N // 2
    chis = [jw.chi_dense(N, i) for i in range(N)]
    m, z, p = hm.term_table(N)
    for t, (i, j, k, l) in enumerate(hm.quadruples(N)):
        P = 4 * chis[i] @ chis[j] @ chis[k] @ chis[l]
        ops = []
        for s in range(n):
            A = jw.SX if (int(m[t]) >> s) & 1 else jw.I2
            B = jw.SZ if (int(z[t]) >> s) & 1 else jw.I2
            ops.append(A @ B)
        Q = np.ones((1, 1), dtype=np.complex128)
        for s in reversed(range(n)):
            Q = np.kron(Q, ops[s])
        assert np.abs(P - (1j ** int(p[t])) * Q).max() < 1e-14


@pytest.mark.parametrize("N", [8, 12, 20, 28, 40])
def test_term_and_mask_counts(N):
    """C(N,4) terms; masks of popcount 4, 2, 0 carry 16, 4(n-2), C(n,2) terms."""
    n = N // 2
    m, _, _ = hm.term_table(N) if N <= 28 else (hm.flip_mask(hm.quadruples(N)).astype(np.uint64), 0, 0)
    assert len(m) == math.comb(N, 4)
    masks, counts = np.unique(m, return_counts=True)
    assert len(masks) == math.comb(n, 4) + math.comb(n, 2) + 1
    pc = jw.popcount(masks)
    assert set(counts[pc == 4]) <= {16} and (pc == 4).sum() == math.comb(n, 4)
    assert set(counts[pc == 2]) == {4 * (n - 2)} and (pc == 2).sum() == math.comb(n, 2)
    assert counts[pc == 0].tolist() == [math.comb(n, 2)]


def test_memory_table_golden():
    """Supp. Table I memory columns follow from C(N,4) and 2^(N/2-1) (printed values rounded)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_memory.txt"), comments="#")
    for N, mf, fm in rows:
        N = int(N)
        D = 2 ** (N // 2 - 1)
        terms = len(hm.quadruples(N)) if N <= 40 else math.comb(N, 4)
        mf_calc = D * 5 * 16 + terms * 20
        fm_calc = D * (5 * 16 + terms * 24)
        assert 0.5 < mf_calc / mf < 1.5 and 0.5 < fm_calc / fm < 1.6


def test_sector_restriction():
    N = 10
    J = inputs.couplings(N, 3)
    H = hm.H_dense(N, J)
    for s in (0, 1):
        xs = hm.full_index(N, s, np.arange(1 << (N // 2 - 1)))
        assert np.all(hm.sector_of(xs) == s)
        assert np.abs(H[np.ix_(xs, xs)] - hm.H_sector_dense(N, J, s)).max() < 1e-15


def test_apply_rows_and_capply_vs_sparse():
    N = 12
    J = inputs.couplings(N, 4)
    psi = inputs.random_states(N, 3, 9).T
    for s in (0, 1):
        ref = hm.H_sector_sparse(N, J, s) @ psi
        rows = [0, 1, 5, 17, 31]
        assert np.abs(hm.apply_rows(N, J, s, psi, rows) - ref[rows]).max() < 1e-14
        tl = capply.TermList(N, J)
        assert np.abs(capply.apply_H(tl, s, psi) - ref).max() < 1e-14
        assert np.abs(capply.apply_H(tl, s, psi, rows=rows) - ref[rows]).max() < 1e-14


def test_chi_sector_squares_to_half():
    N = 12
    psi = inputs.random_states(N, 1, 2)[0]
    for i in (0, 5, 11):
        out = hm.apply_chi(N, i, 1, hm.apply_chi(N, i, 0, psi))
        assert np.abs(out - psi / 2).max() < 1e-15


# ----------------------------------------------------------------------------- evolution

def test_expmv_vs_scipy_expm():
    N = 10
    J = inputs.couplings(N, 6)
    sysm = evolve.SectorSystem(N, J)
    psi = inputs.random_states(N, 2, 1).T
    for s in (0, 1):
        Hs = sysm.H(s).toarray()
        for z in (-0.7j, -1.3, 0.4 - 2.5j):
            ref = sla.expm(z * Hs) @ psi
            assert np.abs(sysm.expmv(z, psi, s) - ref).max() < 1e-12
    out = sysm.expmv(-3.0j, psi, 0)
    assert np.allclose(np.linalg.norm(out, axis=0), np.linalg.norm(psi, axis=0), rtol=1e-13)


def test_expmv_N4_closed_form():
    """N=4 even sector: H = -J/4 (times identity), so e^{zH} psi = e^{-zJ/4} psi."""
    J = np.array([1.3])
    sysm = evolve.SectorSystem(4, J)
    psi = inputs.random_states(4, 1, 0)[0]
    for z in (-2j, -0.5, 1.0 - 1j):
        assert np.abs(sysm.expmv(z, psi, 0) - np.exp(-z * 1.3 / 4) * psi).max() < 1e-14


def test_expm_multiply_path_vs_dense():
    N = 14
    J = inputs.couplings(N, 8)
    psi = inputs.random_states(N, 1, 4)[0]
    dense = evolve.SectorSystem(N, J)
    sparse = evolve.SectorSystem(N, J, dense_max=1)
    for z in (-4.0j, -1.25):
        a = dense.expmv(z, psi, 0)
        b = sparse.expmv(z, psi, 0)
        assert np.abs(a - b).max() < 1e-11 * np.abs(a).max()


def test_tridiag_expm_special_cases():
    a = np.array([0.3, -1.1, 2.0])
    out = evolve.tridiag_expm_e1(a, np.zeros(2), -0.5j, beta0=2.0)
    assert np.allclose(out, [2.0 * np.exp(-0.5j * 0.3), 0, 0], atol=1e-15)
    # 2x2: T = [[0, b], [b, 0]]  ->  e^{zT} e1 = (cosh(zb), sinh(zb))
    b, z = 0.8, -1.7j
    out = evolve.tridiag_expm_e1(np.zeros(2), np.array([b]), z)
    assert np.allclose(out, [np.cosh(z * b), np.sinh(z * b)], atol=1e-15)
    al, be = inputs.random_tridiagonal(12, 3)
    T = np.diag(al) + np.diag(be, 1) + np.diag(be, -1)
    w, Q = np.linalg.eigh(T)
    z = 0.2 - 3.0j
    ref = Q @ (np.exp(z * w) * Q[0])
    assert np.abs(evolve.tridiag_expm_e1(al, be, z) - ref).max() < 1e-12


# ----------------------------------------------------------------------------- correlators

@pytest.mark.parametrize("beta", [0.0, 3.0])
def test_G_and_F_N4_closed_form(beta):
    """N=4, even sector: chi_0(t) chi_0 = e^{2iHt}/2 and the F chain reduces to
    -(1/4) e^{4iHt}; with H = -J/4 there, G = e^{-iJt/2}/2 and F~ = e^{-iJt}."""
    Jv = 0.9
    sysm = evolve.SectorSystem(4, np.array([Jv]))
    psi = inputs.random_states(4, 1, 5)[0]
    ts = np.linspace(0, 7, 8)
    G, Z = co.G_state(sysm, beta, 0, ts, psi)
    assert np.abs(G - 0.5 * np.exp(-0.5j * Jv * ts)).max() < 1e-14
    F = co.F_state(sysm, beta, 0, 1, ts, psi)
    nrm = np.vdot(psi, psi).real
    assert np.abs(F - (-0.25) * np.exp(-1j * Jv * ts) * nrm).max() < 1e-14 * nrm


def test_G_F_at_t0_beta0():
    """beta=0, t=0: chi_i^2 = 1/2 gives G(0) = 1/2; chi_i chi_j chi_i chi_j = -1/4 gives F(0)."""
    N = 12
    sysm = evolve.SectorSystem(N, inputs.couplings(N, 1))
    psi = inputs.random_states(N, 2, 2).T
    G, _ = co.G_state(sysm, 0.0, 3, [0.0], psi)
    assert np.abs(G - 0.5).max() < 1e-15
    F = co.F_state(sysm, 0.0, 0, 1, [0.0], psi)
    assert np.abs(F[0] + 0.25 * np.sum(np.abs(psi) ** 2, axis=0)).max() < 1e-13


def test_G_short_time_expansion():
    """Trace over the even sector at beta=0: G(t) = 1/2 - (t^2/16) sum_{T contains i} J_T^2 + O(t^4)."""
    N = 12
    J = inputs.couplings(N, 7)
    sysm = evolve.SectorSystem(N, J)
    basis = co.basis_states_even(N)
    i = 2
    q = hm.quadruples(N)
    s2 = np.sum(J[np.any(q == i, axis=1)] ** 2)
    for t in (0.05, 0.1):
        G, Z = co.G_state(sysm, 0.0, i, [t], basis)
        tr = np.sum(G[0] * Z) / np.sum(Z)
        assert abs(tr - (0.5 - t * t * s2 / 16)) < 0.05 * t ** 4 + 1e-14


def test_G_basis_sum_equals_trace():
    """Summing the one-state estimate over a basis of the even sector gives the trace form."""
    N = 8
    J = inputs.couplings(N, 11) * 3.0
    sysm = evolve.SectorSystem(N, J)
    ts = [0.0, 0.6, 2.5]
    G, Z = co.G_state(sysm, 1.5, 5, ts, co.basis_states_even(N))
    est = np.sum(G * Z[None, :], axis=1) / np.sum(Z)
    assert np.abs(est - co.G_trace_even(N, J, 1.5, 5, ts)).max() < 1e-13


def test_F_basis_sum_equals_trace_and_is_real():
    N = 8
    J = inputs.couplings(N, 12) * 3.0
    sysm = evolve.SectorSystem(N, J)
    ts = [0.0, 0.9, 3.0]
    F = co.F_state(sysm, 2.0, 1, 6, ts, co.basis_states_even(N))
    tr = co.F_trace_even(N, J, 2.0, 1, 6, ts)
    assert np.abs(np.sum(F, axis=1) - tr).max() < 1e-13
    # Eq. F_reg is Hermitian, so its full trace is real.  The one-sector trace is
    # not: chi_i and chi_j flip the parity, which breaks the cyclic argument.
    full = co.F_trace_even(N, J, 2.0, 1, 6, ts, sector=None)
    assert np.abs(full.imag).max() < 1e-14 * np.abs(full).max()
    assert np.abs(full - tr - co.F_trace_even(N, J, 2.0, 1, 6, ts, sector=1)).max() < 1e-13


# ----------------------------------------------------------------------------- regularization family, G(tau)

@pytest.mark.parametrize("x", [(0.25, 0.25, 0.25, 0.25), (0.0, 0.0, 0.0, 1.0), (0.1, 0.4, 0.2, 0.3)])
def test_F_split_N4_closed_form(x):
    """N=4 even sector (H = -J/4 there, +J/4 in the odd sector): for every split of rho,
    F(t) = -(1/4)|psi|^2 e^{beta J (x2 + x4 - x1 - x3)/4} e^{-iJt}, so F~(t) = e^{-iJt}."""
    Jv, beta = 0.9, 2.3
    sysm = evolve.SectorSystem(4, np.array([Jv]))
    psi = inputs.random_states(4, 1, 5)[0]
    ts = np.linspace(0, 6, 7)
    F = co.F_state_split(sysm, beta, x, 0, 1, ts, psi)
    nrm = np.vdot(psi, psi).real
    ref = -0.25 * nrm * np.exp(beta * Jv * (x[1] + x[3] - x[0] - x[2]) / 4) * np.exp(-1j * Jv * ts)
    assert np.abs(F - ref).max() < 1e-13 * np.abs(ref).max()


def test_F_split_regularized_is_F_reg_and_basis_sum_is_trace():
    N = 8
    J = inputs.couplings(N, 12) * 3.0
    sysm = evolve.SectorSystem(N, J)
    psi = inputs.random_states(N, 2, 3).T
    ts = [0.0, 0.9, 3.0]
    assert np.abs(co.F_state_split(sysm, 2.0, (0.25,) * 4, 1, 6, ts, psi)
                  - co.F_state(sysm, 2.0, 1, 6, ts, psi)).max() < 1e-13
    x = (0.0, 0.0, 0.0, 1.0)
    F = co.F_state_split(sysm, 2.0, x, 1, 6, ts, co.basis_states_even(N))
    tr = co.F_trace_split(N, J, 2.0, x, 1, 6, ts)
    assert np.abs(np.sum(F, axis=1) - tr).max() < 1e-12 * np.abs(tr).max()
    # t = 0: chi_i chi_j chi_i chi_j = -1/4, so the full trace is -Tr[rho]/4
    full = co.F_trace_split(N, J, 2.0, x, 1, 6, ts, sector=None)
    assert abs(full[0] + 0.25 * np.trace(sla.expm(-2.0 * hm.H_dense(N, J))).real) < 1e-12


def test_G_imag_N4_and_definitions():
    """N=4: chi_0(tau) chi_0 = e^{2 tau H}/2, so G(tau) = e^{-J tau/2}/2 in the even sector;
    G(0) = 1/2 at any N; the basis sum equals the dense trace form."""
    Jv, beta = 0.8, 3.0
    sysm = evolve.SectorSystem(4, np.array([Jv]))
    psi = inputs.random_states(4, 1, 2)[0]
    taus = np.linspace(0, beta, 5)
    G, _ = co.G_imag_state(sysm, beta, 0, taus, psi)
    assert np.abs(G - 0.5 * np.exp(-Jv * taus / 2)).max() < 1e-14
    N = 8
    J = inputs.couplings(N, 4) * 3.0
    sysm = evolve.SectorSystem(N, J)
    G, Z = co.G_imag_state(sysm, 2.0, 3, [0.0, 0.7, 2.0], co.basis_states_even(N))
    assert np.abs(G[0] - 0.5).max() < 1e-14
    est = np.sum(G * Z[None, :], axis=1) / np.sum(Z)
    assert np.abs(est - co.G_imag_trace_even(N, J, 2.0, 3, [0.0, 0.7, 2.0])).max() < 1e-13
