#!/usr/bin/env python3
"""Benchmark: regularized-OTOC curves per hour at N = 40 on GB300.

One step = the regularized OTOC F~(t) (Eq. F_reg, rho^{1/4} between the
operators, W = chi_0, V = chi_1, beta J = 10) of B = 16 random states of one
coupling draw on a 10-point time grid t = 1.2, 2.4, ..., 12 plus t = 0 (the
10-point curves of Supp. Table I, to the t = 12 of the batched workload),
Krylov dimension 40, tolerance 1e-7, complex64 vectors with FP64 Lanczos
scalars.  value = curves (states) per hour over all ranks; each rank runs its
own coupling draw (independent replicas, weak scaling, no collective on the
data path).  Inputs are synthetic (Gaussian couplings and states, seeded).

--impl reference times the CPU oracle (plain-C term-at-a-time H|psi>) on a
bounded sample of rows and converts it to the same metric with a modelled
count of H applications per curve (see applies_model).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--N", type=int, default=40)
    ap.add_argument("--states", type=int, default=16)
    ap.add_argument("--beta", type=float, default=10.0)
    ap.add_argument("--npts", type=int, default=10)
    ap.add_argument("--tmax", type=float, default=12.0)
    ap.add_argument("--krylov", type=int, default=40)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--dtype", default="c64", choices=["c64", "c128"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", action="store_true",
                    help="mixed-N batched workload (N 20..40, beta J 1/3/10, 8 states per draw)")
    ap.add_argument("--draws", type=int, default=1, help="coupling draws per (N, beta) in --batched mode")
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--batched-Ns", default="20,24,28,32,36,40", help="sizes of the --batched workload")
    ap.add_argument("--graphs", default="segments", choices=["off", "segments", "device"],
                    help="launch mode of the Krylov evolutions of the --batched workload (syk_use_graphs 0/1/2)")
    ap.add_argument("--persistent", default="on", choices=["on", "off", "split"],
                    help="run the --batched items that fit one CTA in the persistent launch (on) or every item on "
                         "the per-item streams (off)")
    ap.add_argument("--grad", action="store_true",
                    help="gradient workload: dF~(t*)/dJ for all couplings and dF~/dbeta at N=28, beta J=5, "
                         "t*=5, about 200 quadrature sub-intervals, 8 states, c64 and c128")
    ap.add_argument("--grad-N", type=int, default=28, help="system size of the --grad workload")
    ap.add_argument("--grad-t", type=float, default=5.0, help="t* of the --grad workload")
    ap.add_argument("--c128-states", type=int, default=2,
                    help="states of the timed complex64 batch also evaluated in the plain complex128 form "
                         "(one state per step), for the c128 arm of the metric and the c64 accuracy (0: skip)")
    ap.add_argument("--orth", default="default", choices=["default", "full", "local"],
                    help="Lanczos orthogonalisation of the evolutions (library default, full Gram-Schmidt, or the "
                         "three-term recurrence)")
    ap.add_argument("--n32-curves", action="store_true",
                    help="the N=32 curve workload at its own size: F~(t) for W=chi_1, V=chi_2 at beta J=10, "
                         "t in [0, 15] step 0.05 (301 points), 16 states per coupling draw, Krylov 40, in c64 "
                         "and c128, with the per-curve c64 error against c128")
    ap.add_argument("--seeds", type=int, default=4, help="coupling draws of the --n32-curves workload")
    ap.add_argument("--no-batched-extra", action="store_true",
                    help="skip the mixed-N batch figure that the default line carries")
    return ap.parse_args()


def time_grid(npts, tmax):
    return [0.0] + [round(tmax * k / npts, 12) for k in range(1, npts + 1)]


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def matvec_kernel(tile, states, dtype):
    """Name and source file of the matvec kernel a tuned launch shape selects."""
    if tile and tile.get("variant", 0) > 0:
        return (f"k_apply_coset<{states}, RB={tile['variant']}, ntb={tile['ntb']}> (cluster {tile['cluster']})",
                "coset", "syk_apply_coset.cu")
    R = "float" if dtype == "c64" else "double"
    shape = f" (ntb={tile['ntb']}, cluster {tile['cluster']})" if tile else ""
    return f"k_apply_tiled<{R}, {states}>" + shape, "tiled", "syk_apply.cu"


def ncu_traffic(N, states, dtype, kind="tiled", source="syk_apply.cu"):
    """DRAM bytes per matvec launch from the committed ncu summary of this configuration,
    or None if there is none or the kernel source changed since it was captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"apply_{kind}_N{N}_B{states}_{dtype}.md")
    src = os.path.join(ROOT, "paper_2002_05725_gb300", "csrc", source)
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None, None
    vals = {}
    keys = ("traffic_bytes_per_launch", "kernel_source_sha256", "smem_wavefronts_per_launch",
            "tma_fill_bytes_per_launch")
    for line in text.splitlines():
        if ":" in line and line.strip().startswith(keys):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != sha or "traffic_bytes_per_launch" not in vals:
        return None, os.path.relpath(path, ROOT)
    out = {k: float(v) for k, v in vals.items() if k != "kernel_source_sha256"}
    return out, os.path.relpath(path, ROOT)


def fp32_peak_tflops(sm_mhz, n_sm):
    """FP32 FMA peak from unit counts: SMs x 128 lanes x 2 flop x clock."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def curve_error(F, Fref):
    """Largest over states of max_t |F~ - F~ref| / max_t |F~ref| with F~ = F / F(t=0)."""
    a = np.asarray(F) / np.asarray(F)[0]
    b = np.asarray(Fref) / np.asarray(Fref)[0]
    return float(np.max(np.max(np.abs(a - b), axis=0) / np.max(np.abs(b), axis=0)))


# ------------------------------------------------------------------ cost model
def applies_model(N, beta, times, m=40, tol=1e-7):
    """Modelled H applications per state for one OTOC curve (Lanczos, checked every 2 vectors).

    A Krylov step of length tau needs the smallest m with (e rho tau / 2m)^m <= tol,
    rho = an effective half spectral width; 0.036 N J reproduces the count measured on
    the GPU path at N = 40 (808 per curve); longer steps are split.
    """
    rho = 0.036 * N

    def m_needed(tau):
        if tau <= 0:
            return 0
        for mm in range(1, 400):
            if (math.e * rho * tau / (2 * mm)) ** mm <= tol:
                return mm
        return 400

    def applies(tau):
        if tau <= 0:
            return 0
        k = 1
        while m_needed(tau / k) > m:
            k += 1
        return k * min(m, 2 * math.ceil(m_needed(tau / k) / 2))

    total = applies(beta / 8) + applies(beta / 4)
    prev = 0.0
    for t in times:
        # forward increments of both chains, then rho^{1/4} U(t)^dag as one evolution of |z|
        total += 2 * applies(t - prev) + 2 * applies(math.hypot(t, beta / 4))
        prev = t
    return total


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons, util = [], 0.0, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                if int(f[0]) != self.index:
                    continue
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            try:
                util.append(float(f[9]))
            except (IndexError, ValueError):
                pass
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}
        if util:
            # nvidia-smi utilization.gpu: percent of the sample period in which a kernel ran
            out["gpu_busy_pct_mean"] = statistics.fmean(util)
        return out


# ------------------------------------------------------------------ CPU oracle
def oracle_apply_seconds(N, states, budget_s, seed=0):
    """Times the oracle's plain-C H|psi> on sampled rows; returns (s per full apply, info)."""
    from oracle import capply
    from paper_2002_05725_gb300 import inputs
    cores = os.cpu_count() or 1
    J = inputs.couplings(N, seed)
    tl = capply.TermList(N, J)
    D = inputs.sector_dim(N)
    rng = np.random.default_rng(1)
    psi = (rng.standard_normal((D, states)) + 1j * rng.standard_normal((D, states))).astype(np.complex128)
    capply.apply_H(tl, 0, psi, rows=rng.integers(0, D, 4 * cores), nthreads=cores)  # warm-up (threads, caches)
    nrows, dt, batch = 0, 0.0, 16 * cores
    while dt < budget_s and nrows < D:
        rows = rng.integers(0, D, batch)
        t0 = time.perf_counter()
        capply.apply_H(tl, 0, psi, rows=rows, nthreads=cores)
        dt += time.perf_counter() - t0
        nrows += batch
        batch = min(2 * batch, 1 << 16)
    per_apply = dt * D / nrows
    return per_apply, {"rows": nrows, "seconds": dt, "cores": cores, "terms": len(tl.m)}


def reference_main(a, rank, world):
    times = time_grid(a.npts, a.tmax)
    A = applies_model(a.N, a.beta, times[1:], a.krylov, a.tol)
    if rank != 0:
        return
    budget = max(2.0, min(30.0, 120.0 / max(1, a.steps + a.warmup)))
    vals, step_s = [], []
    info = None
    for s in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        per_apply, info = oracle_apply_seconds(a.N, a.states, budget, seed=s)
        if s >= a.warmup:
            vals.append(per_apply)
            step_s.append(time.perf_counter() - t0)
    per_apply = statistics.median(vals)
    curve_s = per_apply * A  # all states of the batch advance together in one apply
    value = a.states * 3600.0 / curve_s
    # a step is the bounded sample actually run (its wall time is ms_per_step); the metric is
    # extrapolated from it to whole curves, as `extrapolation` states
    line = {
        "impl": "reference", "metric": "OTOC curves/hour at N=40", "value": value, "unit": "curves/hour",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": statistics.median(step_s) * 1e3,
        "extrapolation": {"seconds_per_full_apply": per_apply, "applies_per_curve": A,
                          "seconds_per_curve_set": curve_s, "states_per_curve_set": a.states},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(a, times),
        "cpu_baseline": {"value": value, "unit": "curves/hour", "cores": info["cores"], "kind": "oracle",
                         "sample": f"plain-C fp64 term-at-a-time H|psi> on {info['rows']} sampled rows x "
                                   f"{a.states} states per step (of {inputs_dim(a.N)}), scaled to full applies x "
                                   f"{A} modelled H applications per curve"},
        "e2e": {"value": value, "unit": "curves/hour", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def inputs_dim(N):
    return 1 << (N // 2 - 1)


def config_dict(a, times):
    return {"workload": f"regularized OTOC F~(t), N={a.N} (sector dim 2^{a.N // 2 - 1}), beta*J={a.beta:g}, "
                        f"W=chi_0 V=chi_1, {a.states} Gaussian random states per coupling draw, "
                        f"t=0 and {a.npts} points to t={a.tmax:g}, Krylov dim {a.krylov}, tol {a.tol:g}",
            "N": a.N, "beta_J": a.beta, "states_per_step": a.states, "t_grid": times, "krylov_dim": a.krylov,
            "tol": a.tol, "vector_dtype": a.dtype, "scalars": "f64",
            "l2": "flushed between timed steps (256 MiB write)"}


# ------------------------------------------------------------------ ranks
def max_over_ranks(value, device, world):
    """Largest value over the ranks (timing is the slowest rank's); no-op for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def curves_per_hour(world, states, steps, t_max_ms):
    """Whole-job throughput: every rank evaluates `states` curves per step (weak scaling)."""
    return world * states * steps * 3600.0 / (t_max_ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def c128_plain_arm(a, terms, host, times, dev, F64):
    """The plain complex128 form (the paper's precision) of the same curves: one state per
    step, states 0..K-1 of the timed batch.  Returns the c128 arm and the accuracy of the
    timed complex64 curves of those states against it."""
    import torch

    from paper_2002_05725_gb300 import syk
    K = min(a.c128_states, a.states)
    cols = [torch.from_numpy(np.ascontiguousarray(host[s][:, None])).to(torch.complex128).to(dev) for s in range(K)]
    stream = torch.cuda.current_stream(dev)
    syk.syk_autotune_apply(terms, syk.SYK_C128, 1)
    syk.syk_otoc(terms, a.beta, 0, 1, times[:2], cols[0], krylov_dim=a.krylov, tol=1e-12)  # warm-up
    torch.cuda.synchronize(dev)
    syk.syk_counters(reset=True)
    clk = ClockSampler(dev.index)
    clk.start()
    total_ms, curves = 0.0, []
    for x in cols:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        curves.append(syk.syk_otoc(terms, a.beta, 0, 1, times, x, krylov_dim=a.krylov, tol=1e-12))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
    clocks = clk.stop()
    cnt = syk.syk_counters(reset=True)
    F128 = np.concatenate(curves, axis=1)
    arm = {"value": K * 3600.0 / (total_ms / 1e3), "unit": "curves/hour", "steps": K, "states_per_step": 1,
           "ms_per_step": total_ms / K, "dtype": "c128", "tol": 1e-12,
           "applies_per_curve": cnt["h_applies"] / K, "clocks": clocks,
           "note": "same coupling draw, grid and Krylov dimension; one state per step; untimed warm-up of "
                   "two points; L2 not flushed (each step runs for seconds)"}
    acc = {"max_t_rel_err_c64_vs_c128": curve_error(F64[:, :K], F128), "states": K, "bound": 1e-5,
           "definition": "per state max_t |F~_c64 - F~_c128| / max_t |F~_c128|, largest over the states; "
                         "F~_c64 from the last timed complex64 step"}
    return arm, acc


def gpu_main(a, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2002_05725_gb300 import inputs, syk
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    syk.load()
    if a.orth != "default":
        for code in (syk.SYK_C64, syk.SYK_C128):
            syk.syk_lanczos_orth(code, syk.ORTH_FULL if a.orth == "full" else syk.ORTH_LOCAL)
    times = time_grid(a.npts, a.tmax)
    realization = rank
    J = inputs.couplings(a.N, seed=0, realization=realization)
    terms = syk.syk_build_terms(a.N, J)
    host = inputs.random_states(a.N, a.states, seed=0, realization=realization)
    cdt = torch.complex64 if a.dtype == "c64" else torch.complex128
    psi_host = torch.from_numpy(np.ascontiguousarray(host.T)).to(cdt).pin_memory()
    psi_dev = psi_host.to(dev).contiguous()
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # untimed: pick the matvec launch shape for this (N, dtype, batch)
    code = syk.SYK_C64 if a.dtype == "c64" else syk.SYK_C128
    if a.states in (1, 2, 4, 8, 16):
        syk.syk_autotune_apply(terms, code, a.states)
    tuned = json.loads(syk.syk_autotune_export())["apply_tiles"]

    def step(src):
        return syk.syk_otoc(terms, a.beta, 0, 1, times, src, krylov_dim=a.krylov, tol=a.tol)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(a.warmup):
        F = step(psi_dev)
    # the matvec's roofline: FMA throughput measured on this device just before the timed region
    fma = {32: syk.syk_fma_peak(32, 8192), 64: syk.syk_fma_peak(64, 256)}
    barrier()

    # timed region: device-resident inputs
    syk.syk_counters(reset=True)
    syk.syk_matvec_launches(reset=True)
    syk.syk_profile_read(reset=True)
    syk.syk_profile_enable(True)
    clk = ClockSampler(local_rank)
    clk.start()
    total_ms = 0.0
    for _ in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        F = step(psi_dev)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
    clocks = clk.stop()
    syk.syk_profile_enable(False)
    prof = syk.syk_profile_read(reset=True)
    cnt = syk.syk_counters(reset=True)
    mv = syk.syk_matvec_launches(reset=True)
    F_timed = F
    barrier()
    t_max = max_over_ranks(total_ms, dev, world)
    value = curves_per_hour(world, a.states, a.steps, t_max)

    # end to end: host (pinned) inputs through the C ABI, result read back to host
    e2e_ms = 0.0
    for _ in range(a.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        F = step(psi_host.numpy())
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_max = max_over_ranks(e2e_ms, dev, world)
    e2e_val = curves_per_hour(world, a.states, a.e2e_steps, e2e_max) if a.e2e_steps else None

    if rank != 0:
        return
    Ft = F_timed / F_timed[0]
    applies_per_state = cnt["h_applies"] / max(1, a.steps) / a.states
    D = terms.D
    nnz = D * terms.nmasks
    avg_ms = prof["total_ms"] / max(1, prof["launches"])
    flops = 8.0 * nnz * a.states
    pk, pk_kind = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    bits = 32 if a.dtype == "c64" else 64
    peak = fma[bits]["tflops"]
    derived = fp32_peak_tflops(sm_mhz, n_sm) / (1.0 if bits == 32 else 64.0)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    tile = next((e for e in tuned if e["N"] == a.N and e["batch"] == a.states and e["dtype"] == code), None)
    kname, kind, ksrc = matvec_kernel(tile, a.states, a.dtype)
    ncu_vals, traffic_src = ncu_traffic(a.N, a.states, a.dtype, kind, ksrc)
    traffic = ncu_vals["traffic_bytes_per_launch"] if ncu_vals else None
    smem = None
    if ncu_vals and "smem_wavefronts_per_launch" in ncu_vals:
        # the matvec's binding unit: the SMs' shared-memory port (128 B per cycle per SM)
        sbytes = ncu_vals["smem_wavefronts_per_launch"] * 128 + ncu_vals.get("tma_fill_bytes_per_launch", 0.0)
        speak = n_sm * 128 * sm_mhz * 1e6 / 1e9
        sach = sbytes / (avg_ms * 1e-3) / 1e9
        smem = {"achieved": sach, "peak": speak, "unit": "GB/s", "frac": sach / speak, "bytes": sbytes,
                "source": "ncu LSU shared-memory wavefronts x 128 B + bulk-copy fill bytes, per launch",
                "peak_kind": f"derived: {n_sm} SMs x 128 B/cycle x {sm_mhz:.0f} MHz"}
    esz = 8 if a.dtype == "c64" else 16
    gather = nnz * a.states * esz / (avg_ms * 1e-3) / 1e9
    orth_names = {syk.ORTH_FULL: "full Gram-Schmidt", syk.ORTH_LOCAL: "three-term recurrence"}
    line = {
        "metric": "OTOC curves/hour at N=40", "value": value, "unit": "curves/hour", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": a.dtype, "data": "synthetic",
        "config": config_dict(a, times),
        "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                     "peak_kind": f"measured: syk_fma_peak({bits}) on this device before the timed region "
                                  f"({'FFMA' if bits == 32 else 'DFMA'} chains, {n_sm} SMs, "
                                  f"{fma[bits]['ms']:.2f} ms); unit-count figure {derived:.2f} TFLOP/s at "
                                  f"{sm_mhz:.0f} MHz",
                     "fma_peaks_measured": {"fp32_tflops": fma[32]["tflops"], "fp64_tflops": fma[64]["tflops"],
                                            "sms": n_sm},
                     "per_launch": {"flops": flops, "avg_ms": avg_ms, "launches": prof["launches"]},
                     "shared_memory": smem},
        "hpsi": {"gather_GBps": gather, "hbm_peak_GBps": pk.get("hbm_gbs"), "gather_frac_of_hbm":
                 gather / float(pk.get("hbm_gbs", 6800.0)), "peak_kind": pk_kind},
        "apply_tile": tile,
        "lanczos_orthogonalisation": {"c64": orth_names[syk.syk_lanczos_orth(syk.SYK_C64)],
                                      "c128": orth_names[syk.syk_lanczos_orth(syk.SYK_C128)]},
        "matvec_launches_by_kernel": mv,
        "applies_per_curve": applies_per_state,
        "applies_per_curve_model": applies_model(a.N, a.beta, times[1:], a.krylov, a.tol),
        "krylov_bases_per_step": cnt["krylov_bases"] / max(1, a.steps),
        "gpu_launches": cnt["launches"],
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "curves/hour", "h2d_bytes_per_step": int(D * a.states * esz),
                "d2h_bytes_per_step": int(len(times) * a.states * 16)},
        "result_check": {"Ftilde_t0": float(np.real(Ft[0, 0])), "Ftilde_tmax_mean": float(np.mean(np.real(Ft[-1])))},
    }
    if world == 1 and a.dtype == "c64" and a.c128_states > 0:
        line["c128_plain"], line["accuracy"] = c128_plain_arm(a, terms, host, times, dev, F_timed)
    if world == 1 and not a.no_batched_extra:
        line["batched"] = run_batched(a, 0, 1, local_rank, draws=1)
    if not a.no_cpu_baseline and world == 1:
        per_apply, info = oracle_apply_seconds(a.N, a.states, a.cpu_seconds)
        curve_s = per_apply * applies_per_state
        line["cpu_baseline"] = {
            "value": a.states * 3600.0 / curve_s, "unit": "curves/hour", "cores": info["cores"], "kind": "oracle",
            "sample": f"plain-C fp64 term-at-a-time H|psi> (oracle/c/apply_terms.c) on {info['rows']} sampled rows "
                      f"x {a.states} states ({info['seconds']:.1f} s), scaled to full applies x "
                      f"{applies_per_state:.0f} H applications per curve counted on the GPU path"}
    print(json.dumps(line), flush=True)


def persistent_summary(rep, hz):
    """The `persistent` object of a --batched line from syk_batch_report's counters: where the
    persistent launch's CTAs spent their SM clock cycles (hz: the SM clock sampled during the
    run), and their matvec rate per SM against one SM's FP32 lane rate (128 lanes x 2 flop per
    cycle): algorithmic flops (8 per nonzero of H_s per state) over the cycles in matvecs.
    Convergence checks that run the full eigendecomposition leave no separate ones
    (ms_per_full_eig None); the last share then holds only the combination coefficients."""
    cyc = max(rep["cycles_items"], 1)
    return {"items": rep["persistent_items"], "per_item_path_items": rep["stream_items"],
            "subitems": rep["persistent_subitems"], "ctas": rep["persistent_ctas"],
            "h_applies": rep["h_applies"], "convergence_checks": rep["checks"],
            "full_eigendecompositions": rep["full_eigs"],
            "seconds_per_subitem": rep["cycles_items"] / hz / max(rep["persistent_subitems"], 1),
            "ms_per_check": rep["cycles_check"] / hz * 1e3 / rep["checks"] if rep["checks"] else None,
            "ms_per_full_eig": rep["cycles_eig"] / hz * 1e3 / rep["full_eigs"] if rep["full_eigs"] else None,
            "matvec_roofline": {
                "achieved_tflops_per_sm": rep["matvec_flops"] * hz / max(rep["cycles_matvec"], 1) / 1e12,
                "peak_tflops_per_sm": 128 * 2 * hz / 1e12,
                "frac": rep["matvec_flops"] / max(rep["cycles_matvec"], 1) / 256.0,
                "peak_kind": "unit count (128 FP32 lanes x 2 flop per cycle per SM)"},
            "cycle_shares": {"matvec": rep["cycles_matvec"] / cyc, "convergence_checks": rep["cycles_check"] / cyc,
                             "eigendecompositions_and_coefficients": rep["cycles_eig"] / cyc},
            "note": "items whose sector vector fits one CTA's shared memory (or whose states split over CTAs) "
                    "run as one persistent launch, a CTA per sub-item running its whole chain on the device; "
                    "cycle shares are SM clock cycles summed over those sub-items"}


def run_batched(a, rank, world, local_rank, draws):
    """Mixed-N batch: draws x (N in 20..40) x (beta J in 1, 3, 10), 8 states each, 10 points to t=12.
    Returns the throughput figure (curves/hour over the wall time of one syk_otoc_batch call)."""
    import torch

    from paper_2002_05725_gb300 import inputs, syk
    torch.cuda.set_device(local_rank)
    syk.load()
    times = time_grid(a.npts, a.tmax)
    Ns, betas = [int(v) for v in a.batched_Ns.split(",")], [1.0, 3.0, 10.0]
    syk.syk_use_graphs({"off": 0, "segments": 1, "device": 2}[a.graphs])
    prev_persistent = syk.syk_batch_persistent({"off": 0, "on": 1, "split": 2}[a.persistent])
    items = []
    for d in range(draws):
        for N in Ns:
            for b in betas:
                r = rank * 100000 + d * 100 + N
                terms = syk.syk_build_terms(N, inputs.couplings(N, seed=7, realization=r))
                psi = inputs.random_states(N, 8, seed=7, realization=r)
                x = torch.from_numpy(np.ascontiguousarray(psi.T)).to(torch.complex64).cuda()
                items.append((terms, b, x))
    syk.syk_otoc_batch(items[:len(Ns)], 0, 1, [0.0, 1.0], dtype=syk.SYK_C64, nworkers=a.workers)  # warm-up/tune
    syk.syk_counters(reset=True)
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    t0 = time.perf_counter()
    out = syk.syk_otoc_batch(items, 0, 1, times, dtype=syk.SYK_C64, krylov_dim=a.krylov, tol=a.tol,
                             nworkers=a.workers)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    cnt = syk.syk_counters(reset=True)
    rep = syk.syk_batch_report()
    syk.syk_use_graphs(True)
    syk.syk_batch_persistent(prev_persistent)
    curves = 8 * len(items)
    persistent = persistent_summary(rep, (clocks.get("sm_mhz") or 2070.0) * 1e6)
    return {"metric": "OTOC curves/hour, mixed-N batch", "value": world * curves * 3600.0 / wall,
            "unit": "curves/hour", "wall_s": wall, "dtype": "c64",
            "config": {"workload": f"{draws} draw(s) x N in {Ns} x beta J in {betas}, 8 states each, "
                                   f"F~ at t=0 and {a.npts} points to t={a.tmax:g}, Krylov {a.krylov}, "
                                   f"tol {a.tol:g}, {a.workers} host workers / streams for the items outside "
                                   f"the persistent launch (persistent {a.persistent})",
                       "items": len(items), "curves": curves,
                       "evolutions": {"off": "host-driven, direct launches", "segments": "host-driven, segment graphs",
                                      "device": "device-driven graphs"}[a.graphs]},
            "clocks": clocks, "persistent": persistent,
            "gpu_launches": cnt["launches"], "h_applies": cnt["h_applies"],
            "result_check": {"Ftilde_t0_all_one": bool(all(np.allclose(F[0] / F[0], 1) for F in out))}}


def batched_main(a, rank, world, local_rank):
    res = run_batched(a, rank, world, local_rank, a.draws)
    if rank == 0:
        line = {"metric": res["metric"], "value": res["value"], "unit": res["unit"], "n_gpus": world, "steps": 1,
                "warmup": 1, "ms_per_step": res["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64", "data": "synthetic"}
        line.update({k: v for k, v in res.items() if k not in line and k not in ("metric", "wall_s")})
        print(json.dumps(line), flush=True)


def grad_main(a, rank, world, local_rank):
    """Gradient workload: F~(t*) and its derivatives w.r.t. all C(N,4) couplings and beta by the
    adjoint chain (syk_otoc_grad), timed per call after a warm-up call, in c64 and c128."""
    import torch

    from paper_2002_05725_gb300 import inputs, syk
    torch.cuda.set_device(local_rank)
    syk.load()
    N, beta, tstar, states = a.grad_N, 5.0, a.grad_t, 8
    quad_dz = 0.05  # |z| rho_est per Gauss-Legendre sub-interval: about 180 sub-intervals for t* = 5
    terms = syk.syk_build_terms(N, inputs.couplings(N, seed=0, realization=rank))
    psi = inputs.random_states(N, states, seed=0, realization=rank)
    res = {}
    for dt in ("c64", "c128"):
        x = torch.from_numpy(np.ascontiguousarray(psi.T)).to(
            torch.complex64 if dt == "c64" else torch.complex128).cuda()
        tol = 1e-7 if dt == "c64" else 1e-12
        syk.syk_otoc_grad(terms, beta, 0, 1, tstar, x, krylov_dim=40, tol=tol, quad_dz=quad_dz)  # warm-up
        syk.syk_counters(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F, dJ, db = syk.syk_otoc_grad(terms, beta, 0, 1, tstar, x, krylov_dim=40, tol=tol, quad_dz=quad_dz)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        cnt = syk.syk_counters(reset=True)
        res[dt] = {"seconds": wall, "F": F, "dJ": dJ, "db": db, "h_applies": cnt["h_applies"] // states,
                   "launches": cnt["launches"]}
    ref = res["c128"]
    rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    if rank == 0:
        print(json.dumps({
            "metric": f"gradient evaluations/hour at N={N} (all couplings and beta, one state each)",
            "value": world * states * 3600.0 / res["c64"]["seconds"], "unit": "gradients/hour", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": res["c64"]["seconds"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"dF~(t*)/dJ_ijkl (C({N},4) = {inputs.n_terms(N)}) and dF~/dbeta, N={N}, "
                                   f"beta J={beta:g}, t*={tstar:g}, Gauss-Legendre sub-intervals of |z| rho_est <= {quad_dz:g}, "
                                   f"{states} states, Krylov 40", "N": N},
            "c128": {"seconds": ref["seconds"], "gradients_per_hour": states * 3600.0 / ref["seconds"],
                     "h_applies_per_state": ref["h_applies"]},
            "c64_h_applies_per_state": res["c64"]["h_applies"],
            "c64_vs_c128": {"F": rel(res["c64"]["F"], ref["F"]), "dJ": rel(res["c64"]["dJ"], ref["dJ"]),
                            "dbeta": rel(res["c64"]["db"], ref["db"])}}), flush=True)


def n32_main(a, rank, world, local_rank):
    """N=32 curve workload at its own size: 301-point F~(t) curves of 16 states per coupling
    draw in c64 (FP64 Lanczos scalars) and c128, each draw's two calls timed with CUDA events;
    reports curves/hour of both forms and the largest c64 curve error against c128."""
    import torch

    from paper_2002_05725_gb300 import inputs, syk
    torch.cuda.set_device(local_rank)
    syk.load()
    N, beta, states = 32, 10.0, 16
    times = [round(0.05 * k, 12) for k in range(301)]
    sec = {"c64": 0.0, "c128": 0.0}
    applies = {"c64": 0, "c128": 0}
    errs = []
    for d in range(a.seeds):
        seed = 1000 * rank + d
        terms = syk.syk_build_terms(N, inputs.couplings(N, seed=seed))
        psi = inputs.random_states(N, states, seed=seed)
        F = {}
        for dt, tol in (("c64", 1e-7), ("c128", 1e-12)):
            code = syk.SYK_C64 if dt == "c64" else syk.SYK_C128
            if d == 0:
                syk.syk_autotune_apply(terms, code, states)
            x = torch.from_numpy(np.ascontiguousarray(psi.T)).to(
                torch.complex64 if dt == "c64" else torch.complex128).cuda()
            syk.syk_counters(reset=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            F[dt] = syk.syk_otoc(terms, beta, 0, 1, times, x, krylov_dim=40, tol=tol)
            e1.record()
            torch.cuda.synchronize()
            sec[dt] += e0.elapsed_time(e1) / 1e3
            applies[dt] += syk.syk_counters(reset=True)["h_applies"] // states
        errs.append(curve_error(F["c64"], F["c128"]))
    if rank == 0:
        n = world * a.seeds * states
        print(json.dumps({
            "metric": "OTOC curves/hour at N=32 (301 points to t=15), c64 vs c128",
            "value": n * 3600.0 / sec["c64"], "unit": "curves/hour", "n_gpus": world, "steps": a.seeds,
            "warmup": 0, "ms_per_step": sec["c64"] * 1e3 / a.seeds, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"regularized OTOC F~(t), N=32 (sector dim 2^15), beta*J={beta:g}, W=chi_0 "
                                   f"V=chi_1, t in [0, 15] step 0.05 (301 points), {states} Gaussian random states "
                                   f"per draw, {a.seeds} coupling draws, Krylov dim 40, tol 1e-7 (c64) / 1e-12 (c128)",
                       "N": N, "seeds": a.seeds, "states_per_draw": states},
            "c128": {"value": n * 3600.0 / sec["c128"], "seconds": sec["c128"],
                     "applies_per_curve": applies["c128"] / a.seeds},
            "c64_seconds": sec["c64"], "c64_applies_per_curve": applies["c64"] / a.seeds,
            "accuracy": {"max_t_rel_err_c64_vs_c128_per_draw": errs, "max": max(errs)}}), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        if world > 1 and rank != 0:
            return
        reference_main(a, rank, world)
        return
    if a.batched:
        batched_main(a, rank, world, local_rank)
        return
    if a.grad:
        grad_main(a, rank, world, local_rank)
        return
    if a.n32_curves:
        n32_main(a, rank, world, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        gpu_main(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
