"""Host logic of bench.py that needs no GPU: the split of the library's profile records into
kernels, phases and per-phase kernel times, and the DRAM-traffic records (taken only while
their sources are unchanged; scaled by algorithmic bytes where the record says so)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rec(launches, ms, flops=0.0, by=0.0):
    return {"launches": launches, "ms": ms, "flops": flops, "bytes": by}


def test_split_profile_separates_kernels_phases_and_per_phase_kernels():
    prof = {
        "k_cpqr": _rec(8, 40.0, 1e9, 1e8),
        "k_fill_y": _rec(4, 8.0),
        "phase:build:level_11": _rec(0, 60.0),
        "phase:solve:schur": _rec(0, 20.0),
        "in:build:level_11:k_cpqr": _rec(2, 11.0),
        "in:build:level_10:k_cpqr": _rec(2, 9.0),
        "in:build:level_11:k_fill_y": _rec(4, 8.0),
    }
    kern, phases, by_phase = bench.split_profile(prof, 2)
    assert set(kern) == {"k_cpqr", "k_fill_y"}
    assert phases == {"build:level_11": 30.0, "solve:schur": 10.0}
    assert by_phase["build:level_11"]["k_cpqr"] == {"ms": 5.5, "launches": 1.0}
    assert by_phase["build:level_11"]["k_fill_y"] == {"ms": 4.0, "launches": 2.0}
    assert by_phase["build:level_10"] == {"k_cpqr": {"ms": 4.5, "launches": 1.0}}
    # a kernel's per-phase times never exceed its total
    tot = sum(v["ms"] for ph in by_phase.values() for k, v in ph.items() if k == "k_cpqr")
    assert tot <= kern["k_cpqr"]["ms"] / 2 + 1e-12


def test_traffic_records_follow_their_sources(monkeypatch, tmp_path):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    rel = os.path.relpath(str(src), bench.ROOT)
    digest = bench._sources_digest([rel])
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {
        ("w", "k_fixed"): {"bytes_per_launch": 5.0e8, "note": "capture", "sources": [rel], "digest": digest},
        ("w", "k_scaled"): {"ratio_to_algorithmic": 0.5, "note": "scaled", "sources": [rel], "digest": digest},
    })
    assert bench.measured_traffic("w", "k_fixed") == (5.0e8, "capture")
    assert bench.measured_traffic("w", "k_scaled", 2.0e8) == (1.0e8, "scaled")
    b, why = bench.measured_traffic("w", "k_scaled")
    assert b is None and "algorithmic" in why
    b, why = bench.measured_traffic("w", "k_other")
    assert b is None and "no ncu capture" in why
    src.write_text("// kernel v2\n")  # the kernel changed since the capture
    b, why = bench.measured_traffic("w", "k_fixed")
    assert b is None and "predates" in why


def test_committed_traffic_records_name_existing_sources():
    for rec in bench.NCU_TRAFFIC.values():
        for p in rec["sources"]:
            assert os.path.exists(os.path.join(bench.ROOT, p)), p
        assert len(rec["digest"]) == 16


def test_kernel_peaks_follow_the_precision_mode():
    # FP64 handles: the FP64 unit; double-float and tensor precision: the FP32 pipes for every
    # kernel whose updates run in double-float, so no kernel's fraction can exceed its unit
    fp64 = bench.kernel_peak("k_schur_solve", 0)[1]
    for name in ("k_schur_solve", "k_pgj", "k_gj_inverse", "k_bgj_panel", "k_pqr", "k_cpqr"):
        assert bench.kernel_peak(name, 0)[1] == fp64
        for prec in (1, 2):
            bound, peak, note = bench.kernel_peak(name, prec)
            assert bound == "alu" and peak > 4.0 * fp64 and "double-float" in note
    assert bench.kernel_peak("k_zgemm_batched_df", 0)[1] > 4.0 * fp64
    assert bench.kernel_peak("k_oz_mma", 2)[0] == "tensor"
