"""Resumable sets of OTOC curves: one .npz file per work item on the host.

A disorder average needs many independent items (coupling draw, beta, random states; Supp.
Sec. I.C), and a run over all of them can last hours.  `run_otoc_items` computes the items in
chunks through `syk_otoc_batch` and writes each item's curves to its own file as soon as its
chunk is done (written to a temporary name, then renamed, so a file is either complete or
absent).  Run again with the same directory, it loads every item whose file exists with the
same settings and computes only the rest: an interrupted run resumes where it stopped.

File name: otoc_N{N}_seed{seed}_r{realization}_beta{beta}.npz; contents: F (nt x states, the
unnormalised F(t) of each state), t, and the settings that produced it (N, seed,
realization, beta, states, i, j, dtype, krylov_dim, tol).  A file whose settings differ from
the request is recomputed and overwritten.
"""
from __future__ import annotations

import os

import numpy as np

SETTINGS = ("N", "seed", "realization", "beta", "states", "i", "j", "dtype", "krylov_dim", "tol")


def item_path(out_dir: str, spec: dict) -> str:
    return os.path.join(out_dir, f"otoc_N{spec['N']}_seed{spec['seed']}_r{spec['realization']}"
                                 f"_beta{float(spec['beta']):g}.npz")


def _settings(spec, i, j, dtype, krylov_dim, tol):
    return {"N": int(spec["N"]), "seed": int(spec["seed"]), "realization": int(spec["realization"]),
            "beta": float(spec["beta"]), "states": int(spec["states"]), "i": int(i), "j": int(j),
            "dtype": int(dtype), "krylov_dim": int(krylov_dim), "tol": float(tol)}


def load_item(path: str, settings: dict, times):
    """The stored curves if the file exists and matches the settings and time grid, else None."""
    if not os.path.exists(path):
        return None
    try:
        with np.load(path) as z:
            for k in SETTINGS:
                if k not in z or z[k].item() != settings[k]:
                    return None
            if z["t"].shape != (len(times),) or not np.array_equal(z["t"], np.asarray(times, dtype=np.float64)):
                return None
            return np.array(z["F"])
    except (OSError, ValueError, KeyError):
        return None  # unreadable or truncated: recompute


def save_item(path: str, settings: dict, times, F) -> None:
    tmp = path + ".tmp.npz"
    np.savez(tmp, F=np.asarray(F), t=np.asarray(times, dtype=np.float64),
             **{k: np.asarray(v) for k, v in settings.items()})
    os.replace(tmp, path)


def gpu_compute(specs, times, i, j, dtype, krylov_dim, tol, nworkers):
    """Curves of the given items on the GPU (seeded couplings and states from `inputs`)."""
    import torch

    from . import inputs, syk
    items = []
    for s in specs:
        terms = syk.syk_build_terms(s["N"], inputs.couplings(s["N"], seed=s["seed"], realization=s["realization"]))
        psi = inputs.random_states(s["N"], s["states"], seed=s["seed"], realization=s["realization"])
        cdt = torch.complex64 if dtype == syk.SYK_C64 else torch.complex128
        x = torch.from_numpy(np.ascontiguousarray(psi.T)).to(cdt).cuda()
        items.append((terms, s["beta"], x))
    return syk.syk_otoc_batch(items, i, j, times, dtype=dtype, krylov_dim=krylov_dim, tol=tol, nworkers=nworkers)


def run_otoc_items(specs, times, out_dir, i=0, j=1, dtype=1, krylov_dim=40, tol=1e-7, nworkers=4, chunk=16,
                   compute=None):
    """F (nt x states) of every item spec ({N, seed, realization, beta, states}), loaded from
    out_dir where present, otherwise computed `chunk` items at a time and stored.  Returns
    (list of F in the order of specs, number of items computed now)."""
    compute = compute or gpu_compute
    os.makedirs(out_dir, exist_ok=True)
    out = [None] * len(specs)
    todo = []
    for k, s in enumerate(specs):
        st = _settings(s, i, j, dtype, krylov_dim, tol)
        F = load_item(item_path(out_dir, s), st, times)
        if F is None:
            todo.append(k)
        else:
            out[k] = F
    for c0 in range(0, len(todo), chunk):
        ks = todo[c0:c0 + chunk]
        Fs = compute([specs[k] for k in ks], times, i, j, dtype, krylov_dim, tol, nworkers)
        for k, F in zip(ks, Fs):
            save_item(item_path(out_dir, specs[k]), _settings(specs[k], i, j, dtype, krylov_dim, tol), times, F)
            out[k] = np.asarray(F)
    return out, len(todo)
