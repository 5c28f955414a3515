"""torch.autograd wrappers of the C-ABI gradient entry points.

``otoc_tilde(J, beta, ...)`` and ``g_t(J, beta, ...)`` return the real and
imaginary parts (shape (B, 2), float64) of F~(t) = F(t)/F(0) (Eq. F_reg) or G(t)
(Eq. G) for B random states, as differentiable functions of the couplings J
(C(N,4), float64) and beta (0-d float64).  The forward pass calls
syk_otoc_grad / syk_correlator_G_grad, which return the value and the full
Jacobian in one call; backward contracts that Jacobian with the incoming
gradient (chain rule only).
"""
from __future__ import annotations

import numpy as np
import torch

from . import syk


class _CorrelatorFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, beta, kind, args, psi0, opts):
        N = args["N"]
        terms = syk.syk_build_terms(N, J.detach().cpu().numpy())
        b = float(beta.detach().cpu())
        if kind == "otoc":
            val, dJ, db = syk.syk_otoc_grad(terms, b, args["i"], args["j"], args["t"], psi0, **opts)
        else:
            val, dJ, db = syk.syk_correlator_G_grad(terms, b, args["i"], args["t"], psi0, **opts)
        ctx.save_for_backward(torch.from_numpy(np.stack([dJ.real, dJ.imag], -1)),
                              torch.from_numpy(np.stack([db.real, db.imag], -1)))
        ctx.dev = J.device
        return torch.from_numpy(np.stack([val.real, val.imag], -1)).to(J.device)

    @staticmethod
    def backward(ctx, gout):
        dJ, db = ctx.saved_tensors                     # (T, B, 2), (B, 2)
        g = gout.detach().to("cpu", torch.float64)     # (B, 2)
        gJ = torch.einsum("tbc,bc->t", dJ, g).to(ctx.dev)
        gb = torch.einsum("bc,bc->", db, g).to(ctx.dev)
        return gJ, gb, None, None, None, None


def otoc_tilde(J, beta, N, i, j, t, psi0, krylov_dim=40, tol=1e-12, quad_dz=0.25):
    """Differentiable (Re, Im) of F~(t) per state, shape (B, 2)."""
    return _CorrelatorFn.apply(J, beta, "otoc", {"N": N, "i": i, "j": j, "t": t}, psi0,
                               {"krylov_dim": krylov_dim, "tol": tol, "quad_dz": quad_dz})


def g_t(J, beta, N, i, t, psi0, krylov_dim=30, tol=1e-12, quad_dz=0.25):
    """Differentiable (Re, Im) of G(t) per state, shape (B, 2)."""
    return _CorrelatorFn.apply(J, beta, "g", {"N": N, "i": i, "t": t}, psi0,
                               {"krylov_dim": krylov_dim, "tol": tol, "quad_dz": quad_dz})
