"""Host-side arithmetic of bench.py's roofline fields: algorithmic bytes per zone-update for
the workload shapes (n_v w per access: one read of the stage input and one write every
stage, one read of U^n in combining stages), the ghost-inflated figure, the derived FP32 /
FP64 peaks, and the measured-traffic guard (a figure only while the kernel sources hash to
the captured version)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("nvar,w,rk,expect", [(5, 8, 2, 100.0), (5, 4, 2, 50.0), (9, 8, 3, 192.0),
                                               (9, 4, 3, 96.0), (5, 4, 3, 160.0 / 3.0)])
def test_algorithmic_bytes(nvar, w, rk, expect):
    assert bench.algorithmic_bytes_per_zone(nvar, w, rk) == pytest.approx(expect, rel=1e-15)


def test_ghost_inflated_bytes():
    # 9 vars x 4 B: halo read (8000/4096 - 1) + ghost write and fill read (3904/4096 each)
    extra = 36.0 * (8000.0 / 4096.0 - 1.0) + 2 * 36.0 * 3904.0 / 4096.0
    assert bench.ghost_inflated_bytes_per_zone(9, 4, 3) == pytest.approx(96.0 + extra, rel=1e-15)


def test_derived_alu_peaks():
    assert bench.alu_peak_tflops(bench.FP32_LANES, 2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert bench.alu_peak_tflops(bench.FP64_LANES, 2070.0) == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)


def test_traffic_only_for_the_captured_sources(monkeypatch):
    import hashlib
    h = hashlib.sha256()
    for f in bench.STAGE_SRC:
        with open(os.path.join(ROOT, "paper_2607_19277_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setattr(bench, "STAGE_SRC_DIGEST", h.hexdigest()[:16])
    assert bench.stage_traffic() == pytest.approx(bench.STAGE_TRAFFIC_BYTES)
    monkeypatch.setattr(bench, "STAGE_SRC_DIGEST", "0" * 16)
    assert bench.stage_traffic() is None


def test_summary_collects_the_legs_and_drops_missing_ones():
    line = {"value": 1.0, "roofline": {"frac": 0.3, "launch_ms": 0.9, "alu": {"frac": 0.4}},
            "fp64": {"value": 2.0, "roofline": {"frac": 0.5}},
            "error_vs_fp64": {"max_rel_l1_rho_m_e_B": 1e-6, "rel_l1": {"psi": 1e-4}},
            "serving": {"fp32_batched": {"latency_p99_s": 0.2}}}
    s = bench.summary_of(line)
    assert s == {"fp32_value": 1.0, "fp32_hbm_frac": 0.3, "fp32_alu_frac": 0.4, "fp32_stage_launch_ms": 0.9,
                 "fp64_value": 2.0, "fp64_alu_frac": 0.5, "fp32_max_rel_l1_vs_fp64": 1e-6,
                 "fp32_psi_rel_l1_vs_fp64": 1e-4, "serving_fp32_batched_p99_s": 0.2}


def test_average_to_base_grid_is_volume_weighted():
    """Leaves of level 1 and 2 averaged onto a 32^3 base grid (2 base blocks per edge): a
    level-2 block covers 8 base cells per edge, each the mean of 2^3 fine cells."""
    import numpy as np
    rng = np.random.default_rng(3)
    lev = np.array([1, 2])
    ijk = np.array([[0, 0, 0], [2, 0, 0]])      # level-2 block (2,0,0) sits in base block (1,0,0)
    cons = rng.random((2, 5, 16, 16, 16))
    out = bench._average_to_base(lev, ijk, cons, 32)
    assert np.array_equal(out[:, :16, :16, :16], cons[0])
    fine = cons[1].reshape(5, 8, 2, 8, 2, 8, 2).mean(axis=(2, 4, 6))
    assert np.allclose(out[:, :8, :8, 16:24], fine, rtol=0, atol=1e-15)
    assert not out[:, 16:, :, :].any()
