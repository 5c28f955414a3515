"""Host logic of bench.py: time grid, throughput, peaks, kernel naming and ncu-summary parsing."""
import hashlib
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_time_grid_and_throughput():
    assert bench.time_grid(10, 12.0) == [0.0] + [round(1.2 * k, 12) for k in range(1, 11)]
    # 2 ranks x 16 curves x 2 steps in 20 s -> 64 curves per 20 s
    assert bench.curves_per_hour(2, 16, 2, 20000.0) == pytest.approx(64 * 3600 / 20.0)
    assert bench.max_over_ranks(3.5, None, 1) == 3.5


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)


def test_matvec_kernel_names():
    name, kind, src = bench.matvec_kernel({"ntb": 7, "cluster": 2, "variant": 1}, 16, "c64")
    assert kind == "coset" and src == "syk_apply_coset.cu" and "RB=1" in name and "cluster 2" in name
    name, kind, src = bench.matvec_kernel({"ntb": 6, "cluster": 1, "variant": 0}, 8, "c128")
    assert kind == "tiled" and src == "syk_apply.cu" and name.startswith("k_apply_tiled<double, 8>")
    assert bench.matvec_kernel(None, 1, "c64")[0] == "k_apply_tiled<float, 1>"


def test_ncu_summary_parsing_follows_the_source_hash(tmp_path, monkeypatch):
    """Traffic is taken from a committed summary only while the kernel source is unchanged."""
    src_dir = tmp_path / "paper_2002_05725_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = src_dir / "k.cu"
    src.write_text("kernel source v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "apply_coset_N40_B16_c64.md").write_text(
        "# summary\n\ntraffic_bytes_per_launch: 123\nsmem_wavefronts_per_launch: 10\n"
        f"tma_fill_bytes_per_launch: 5\nkernel_source_sha256: `{sha}`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    vals, path = bench.ncu_traffic(40, 16, "c64", "coset", "k.cu")
    assert vals == {"traffic_bytes_per_launch": 123.0, "smem_wavefronts_per_launch": 10.0,
                    "tma_fill_bytes_per_launch": 5.0}
    assert path == os.path.join("profiles", "apply_coset_N40_B16_c64.md")
    src.write_text("kernel source v2\n")  # the kernel changed since the capture
    assert bench.ncu_traffic(40, 16, "c64", "coset", "k.cu")[0] is None
    assert bench.ncu_traffic(40, 8, "c64", "coset", "k.cu") == (None, None)  # no summary at all


def test_applies_model_is_calibrated():
    assert bench.applies_model(40, 10.0, bench.time_grid(10, 12.0)[1:]) == 808


def test_curve_error_is_per_state_max_t_norm():
    """max_t |F~ - F~ref| / max_t |F~ref| per state (F~ = F / F(0)), largest over the states."""
    t = np.linspace(0.0, 1.0, 5)
    ref = np.stack([np.exp(-t), 2.0 * np.exp(-2 * t)], axis=1)
    F = ref.copy()
    F[3, 1] += 2e-3 * 2.0  # state 1: F~ off by 2e-3 at one time, max_t |F~ref| = 1
    assert bench.curve_error(F, ref) == pytest.approx(2e-3)
    assert bench.curve_error(3.0 * ref, ref) == pytest.approx(0.0, abs=1e-15)  # scale cancels in F~


def test_persistent_summary_shares_and_matvec_rate():
    """The --batched line's persistent object from syk_batch_report counters: shares of the
    CTAs' cycles, per-check time, and the matvec rate per SM against 128 lanes x 2 flop x clock."""
    hz = 2.0e9
    rep = {"persistent_items": 4, "stream_items": 1, "persistent_subitems": 8, "persistent_ctas": 8,
           "cycles_matvec": 6e9, "cycles_check": 2e9, "cycles_eig": 0, "cycles_items": 8e9,
           "h_applies": 1000, "checks": 400, "full_eigs": 0, "matvec_flops": int(0.25 * 256 * 6e9)}
    p = bench.persistent_summary(rep, hz)
    assert p["seconds_per_subitem"] == pytest.approx(8e9 / hz / 8)
    assert p["ms_per_check"] == pytest.approx(2e9 / hz * 1e3 / 400)
    assert p["ms_per_full_eig"] is None  # checks fused with the full eigendecomposition
    assert p["cycle_shares"]["matvec"] == pytest.approx(0.75)
    assert p["matvec_roofline"]["frac"] == pytest.approx(0.25)
    assert p["matvec_roofline"]["achieved_tflops_per_sm"] == pytest.approx(0.25 * 256 * hz / 1e12)
    assert p["matvec_roofline"]["peak_tflops_per_sm"] == pytest.approx(256 * hz / 1e12)
