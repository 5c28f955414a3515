"""Gradients of F~(t) and G(t) w.r.t. every coupling and beta on the GPU."""
import numpy as np
import pytest

from helpers import rel, to_dev, torch_or_skip
from oracle import gradient as gr
from paper_2002_05725_gb300 import inputs, syk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_or_skip()
    syk.load(build_if_missing=True)
    return t


@pytest.mark.parametrize("N", [8, 12])
def test_otoc_grad_vs_daleckii_krein(torch, N):
    J = inputs.couplings(N, 5) * (2.0 if N == 8 else 1.0)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 2, 9)
    beta, t, i, j = 3.0, 2.2, 0, 1
    F, dJ, db = syk.syk_otoc_grad(terms, beta, i, j, t, to_dev(torch, psi, "c128"), krylov_dim=30, tol=1e-13,
                                  quad_dz=0.1)
    Fr, dJr, dbr = gr.otoc_tilde_grad(N, J, beta, i, j, t, psi.T)
    assert rel(F, Fr) < 1e-11
    assert rel(dJ, dJr) < 1e-8
    assert rel(db, dbr) < 1e-8 * max(1.0, np.abs(dJr).max() / max(np.abs(dbr).max(), 1e-30))


@pytest.mark.parametrize("N", [8, 12])
def test_G_grad_vs_daleckii_krein(torch, N):
    J = inputs.couplings(N, 6) * (2.0 if N == 8 else 1.0)
    terms = syk.syk_build_terms(N, J)
    psi = inputs.random_states(N, 3, 2)
    beta, t, i = 2.0, 3.1, 3
    G, dJ, db = syk.syk_correlator_G_grad(terms, beta, i, t, to_dev(torch, psi, "c128"), krylov_dim=30, tol=1e-13,
                                          quad_dz=0.1)
    Gr, dJr, dbr = gr.g_grad(N, J, beta, i, t, psi.T)
    assert rel(G, Gr) < 1e-11
    assert rel(dJ, dJr) < 1e-8
    assert np.abs(db - dbr).max() < 1e-8 * max(np.abs(dJr).max(), np.abs(dbr).max())


def _fd_checks(fun, J, beta, dJ, db, rng, ncoup=50, ndir=4, h=1e-6):
    """Central differences (h = 1e-6) of fun(J, beta) on ncoup sampled couplings, ndir random
    unit directions in coupling space and beta, against the adjoint gradient (per state)."""
    sample = rng.choice(len(J), ncoup, replace=False)
    fdJ, fdb = gr.fd_grad(fun, J, beta, sample, h=h)
    dirs = rng.standard_normal((ndir, len(J)))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    fdd = np.array([(fun(J + h * d, beta) - fun(J - h * d, beta)) / (2 * h) for d in dirs])
    scale = np.abs(dJ).max()
    errs = {"couplings": float(np.abs(dJ[sample] - fdJ).max() / scale),
            "directions": float(np.abs(dirs @ dJ - fdd).max() / max(np.abs(dirs @ dJ).max(), scale)),
            "beta": float(np.abs(db - fdb).max() / max(np.abs(db).max(), scale))}
    return errs


@pytest.fixture(scope="module")
def n28_config():
    """The gradient workload's own settings: N = 28 (20475 couplings), beta J = 5, t* = 5,
    Gauss-Legendre sub-intervals of |z| rho <= 0.05 (about 200 time steps), two states."""
    N = 28
    J = inputs.couplings(N, 0)
    return {"N": N, "J": J, "terms": syk.syk_build_terms(N, J), "psi": inputs.random_states(N, 2, 0),
            "beta": 5.0, "t": 5.0, "quad_dz": 0.05}


def test_otoc_grad_N28_config_vs_finite_differences(torch, n28_config):
    """dF~(t*)/dJ and dF~/dbeta (c128) against central differences of the GPU F~ (c128) on 50
    sampled couplings, 4 random directions and beta, within 1e-4 of the gradient's scale; the
    c64 gradient against the c128 one within 1e-4."""
    c = n28_config
    dev = to_dev(torch, c["psi"], "c128")
    F, dJ, db = syk.syk_otoc_grad(c["terms"], c["beta"], 0, 1, c["t"], dev, krylov_dim=40, tol=1e-13,
                                  quad_dz=c["quad_dz"])

    def Ftil(Jx, b):
        Fx = syk.syk_otoc(syk.syk_build_terms(c["N"], Jx), b, 0, 1, [0.0, c["t"]], dev, krylov_dim=40, tol=1e-13)
        return Fx[1] / Fx[0]

    assert rel(F, Ftil(c["J"], c["beta"])) < 1e-10
    errs = _fd_checks(Ftil, c["J"], c["beta"], dJ, db, np.random.default_rng(28))
    assert max(errs.values()) < 1e-4, errs
    F64, dJ64, db64 = syk.syk_otoc_grad(c["terms"], c["beta"], 0, 1, c["t"], to_dev(torch, c["psi"], "c64"),
                                        krylov_dim=40, tol=1e-7, quad_dz=c["quad_dz"])
    assert rel(F64, F) < 1e-5
    assert rel(dJ64, dJ) < 1e-4
    assert np.abs(db64 - db).max() < 1e-4 * max(np.abs(db).max(), np.abs(dJ).max())


def test_G_grad_N28_config_vs_finite_differences(torch, n28_config):
    """dG(t*)/dJ and dG/dbeta (G normalised by Z = <phi|phi>) at the same settings."""
    c = n28_config
    dev = to_dev(torch, c["psi"], "c128")
    G, dJ, db = syk.syk_correlator_G_grad(c["terms"], c["beta"], 0, c["t"], dev, krylov_dim=40, tol=1e-13,
                                          quad_dz=c["quad_dz"])

    def Gt(Jx, b):
        Gx, _ = syk.syk_correlator_G(syk.syk_build_terms(c["N"], Jx), b, 0, [c["t"]], dev, krylov_dim=40, tol=1e-13)
        return Gx[0]

    assert rel(G, Gt(c["J"], c["beta"])) < 1e-10
    errs = _fd_checks(Gt, c["J"], c["beta"], dJ, db, np.random.default_rng(29))
    assert max(errs.values()) < 1e-4, errs
    G64, dJ64, db64 = syk.syk_correlator_G_grad(c["terms"], c["beta"], 0, c["t"], to_dev(torch, c["psi"], "c64"),
                                                krylov_dim=40, tol=1e-7, quad_dz=c["quad_dz"])
    assert rel(G64, G) < 1e-5
    assert rel(dJ64, dJ) < 1e-4


def test_autograd_function_matches_jacobian(torch):
    from paper_2002_05725_gb300 import autograd as sa
    N = 12
    Jn = inputs.couplings(N, 2)
    psi = to_dev(torch, inputs.random_states(N, 3, 4), "c128")
    J = torch.tensor(Jn, dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    out = sa.otoc_tilde(J, beta, N, 0, 1, 1.5, psi, krylov_dim=30, quad_dz=0.2)
    w = torch.tensor([[1.0, -0.5], [0.25, 2.0], [-1.0, 0.3]], dtype=torch.float64)
    (out * w).sum().backward()
    _, dJ, db = gr.otoc_tilde_grad(N, Jn, 2.0, 0, 1, 1.5, psi.cpu().numpy())
    refJ = dJ.real @ w[:, 0].numpy() + dJ.imag @ w[:, 1].numpy()
    refb = float(db.real @ w[:, 0].numpy() + db.imag @ w[:, 1].numpy())
    assert np.abs(J.grad.numpy() - refJ).max() < 1e-8 * np.abs(refJ).max()
    assert abs(beta.grad.item() - refb) < 1e-8 * max(1.0, abs(refb))
