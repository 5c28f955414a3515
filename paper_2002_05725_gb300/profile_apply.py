"""Times syk_apply_H on one configuration (for profilers and quick measurements), and with
--expmv one real-time evolution step through syk_expmv.

    python -m paper_2002_05725_gb300.profile_apply --N 40 --batch 8 --dtype c64 --reps 3

Autotunes the launch shape for the configuration first (as the benchmark does),
then prints one JSON line with the mean time per apply (CUDA events, after one
warm-up apply) and the FP32/FP64 and effective-gather rates.
"""
from __future__ import annotations

import argparse
import json

from . import inputs, syk


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sector", type=int, default=0)
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch-shape heuristic")
    ap.add_argument("--expmv", type=float, default=None, metavar="T",
                    help="also time one real-time step e^{-iHT} psi (Krylov dimension --krylov, tol --tol) and "
                         "check that it preserves the norm")
    ap.add_argument("--krylov", type=int, default=20)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--tile", default=None,
                    help="force the launch shape 'ntb,cluster[,variant]' (no tuning sweep; variant 0 = k_apply_tiled, "
                         "1..3 = k_apply_coset with 2^variant rows per thread)")
    ap.add_argument("--grad", type=float, default=None, metavar="TSTAR",
                    help="also time one gradient call syk_otoc_grad (beta J = 5, t* = TSTAR, quad_dz 0.05, "
                         "tol 1e-7 for c64 and 1e-12 for c128), as the benchmark's gradient workload runs it")
    ap.add_argument("--c128-arith", default="df", choices=["df", "fp64"],
                    help="complex128 matvec arithmetic: double-float (default) or native FP64")
    a = ap.parse_args()
    import torch
    syk.load()
    syk.syk_c128_arith(syk.C128_DOUBLE_FLOAT if a.c128_arith == "df" else syk.C128_FP64)
    dt = torch.complex64 if a.dtype == "c64" else torch.complex128
    terms = syk.syk_build_terms(a.N, inputs.couplings(a.N, 0))
    psi = inputs.random_states_device(a.N, a.batch, 1, "cuda", dt)
    y = torch.empty_like(psi)
    tile = None
    code = syk.SYK_C64 if a.dtype == "c64" else syk.SYK_C128
    if a.tile:
        v = [int(t) for t in a.tile.split(",")]
        ntb, cs, var = v[0], v[1], (v[2] if len(v) > 2 else 0)
        syk.syk_autotune_import(json.dumps({"apply_tiles": [{"N": a.N, "dtype": code, "batch": a.batch,
                                                             "ntb": ntb, "cluster": cs, "variant": var}]}))
        tile = {"ntb": ntb, "cluster": cs, "variant": var, "forced": True}
    elif not a.no_tune and a.batch in (1, 2, 4, 8, 16):
        syk.syk_autotune_apply(terms, code, a.batch)
        tile = [e for e in json.loads(syk.syk_autotune_export())["apply_tiles"]
                if e["N"] == a.N and e["batch"] == a.batch]
    syk.syk_apply_H(terms, a.sector, psi, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        syk.syk_apply_H(terms, a.sector, psi, out=y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    nnz = terms.D * terms.nmasks
    s = 8 if a.dtype == "c64" else 16
    out = {"N": a.N, "batch": a.batch, "dtype": a.dtype, "c128_arith": a.c128_arith, "ms_per_apply": ms,
           "tflops": 8.0 * nnz * a.batch / (ms * 1e-3) / 1e12,
           "gather_GBps": nnz * a.batch * s / (ms * 1e-3) / 1e9, "nnz": nnz, "tile": tile}
    if a.expmv is not None:
        # one output step of the real-time evolution, workspace allocated by the call
        syk.syk_counters(reset=True)
        e0.record()
        phi, nb = syk.syk_expmv(terms, a.sector, complex(0.0, -a.expmv), psi, krylov_dim=a.krylov, tol=a.tol,
                                out=y)
        e1.record()
        torch.cuda.synchronize()
        cnt = syk.syk_counters(reset=True)
        n0 = torch.linalg.vector_norm(psi.to(torch.complex128), dim=0)
        n1 = torch.linalg.vector_norm(phi.to(torch.complex128), dim=0)
        out["expmv"] = {"t": a.expmv, "krylov_dim": a.krylov, "tol": a.tol, "seconds": e0.elapsed_time(e1) / 1e3,
                        "krylov_bases": nb, "h_applies": cnt["h_applies"] // a.batch,
                        "workspace_bytes": syk.syk_workspace_bytes(a.N, code, a.krylov, a.batch),
                        "max_norm_change": float(((n1 - n0).abs() / n0).max())}
    if a.grad is not None:
        x = psi.clone()
        tol = 1e-7 if a.dtype == "c64" else 1e-12
        syk.syk_counters(reset=True)
        e0.record()
        syk.syk_otoc_grad(terms, 5.0, 0, 1, a.grad, x, krylov_dim=40, tol=tol, quad_dz=0.05)
        e1.record()
        torch.cuda.synchronize()
        cnt = syk.syk_counters(reset=True)
        out["grad"] = {"tstar": a.grad, "seconds": e0.elapsed_time(e1) / 1e3, "h_applies": cnt["h_applies"] // a.batch,
                       "launches": cnt["launches"]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
