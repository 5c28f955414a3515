"""Writes tests/golden/oracle_N28_curves.json: G(t) and the regularized OTOC F(t) at N = 28
(sector dimension 2^13) from the CPU oracle alone.

At this size the oracle evolves with scipy's expm_multiply on the sector's CSR matrix
(Al-Mohy & Higham), which takes minutes per state, too long to repeat inside every GPU test
run; the values are therefore computed once by this script, which imports only `oracle/`
and the seeded input generators, and stored.  The GPU parity tests read them.

Workload: couplings `inputs.couplings(28, 0)` (Eq. 1, variance 6/N^3), states
`inputs.random_states(28, 2, 0)` (Supp. Sec. I.C), the OTOC of Eq. F_reg at beta J = 10 with
W = chi_0, V = chi_1, and G(t) of Eq. G at beta J = 5 for chi_2, on t = 0, 3, 6, 12.

    python tests/golden/make_oracle_curves.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, SEED, NSTATES = 28, 0, 2
BETA_F, BETA_G, I_G = 10.0, 5.0, 2
TIMES = [0.0, 3.0, 6.0, 12.0]
OUT = os.path.join(HERE, "oracle_N28_curves.json")


def _task(args):
    kind, s = args
    from oracle import correlators as co, evolve
    from paper_2002_05725_gb300 import inputs
    J = inputs.couplings(N, SEED)
    psi = inputs.random_states(N, NSTATES, SEED)[s]
    sysm = evolve.SectorSystem(N, J)
    t0 = time.time()
    if kind == "F":
        F = co.F_state(sysm, BETA_F, 0, 1, TIMES, psi)
        return kind, s, [[float(v.real), float(v.imag)] for v in F], None, time.time() - t0
    G, Z = co.G_state(sysm, BETA_G, I_G, TIMES, psi)
    return kind, s, [[float(v.real), float(v.imag)] for v in G], float(Z), time.time() - t0


def main():
    tasks = [(k, s) for k in ("F", "G") for s in range(NSTATES)]
    with mp.get_context("spawn").Pool(len(tasks)) as pool:
        res = pool.map(_task, tasks)
    out = {"N": N, "seed": SEED, "nstates": NSTATES, "t": TIMES,
           "F": {"beta": BETA_F, "i": 0, "j": 1, "values": [None] * NSTATES},
           "G": {"beta": BETA_G, "i": I_G, "values": [None] * NSTATES, "Z": [None] * NSTATES},
           "seconds": {}}
    for kind, s, vals, Z, sec in res:
        out[kind]["values"][s] = vals
        if kind == "G":
            out["G"]["Z"][s] = Z
        out["seconds"][f"{kind}{s}"] = round(sec, 1)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}: {out['seconds']}")


if __name__ == "__main__":
    main()
