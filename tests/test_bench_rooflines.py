"""The roofline records of bench.py from per-phase times (host logic, no GPU).

Both factorisation schedules must give well-formed records: the separate
kernels (a diagonal-inverse phase and an update phase per block) and the fused
launch (one update-phase span per inversion, no diagonal-inverse spans).  The
DRAM-traffic figures come from ncu captures and are used only while each
kernel's source file is unchanged.
"""

import hashlib
import os
import types

import pytest

import bench

PHASES = ("kinematics", "nearest", "segments", "assemble", "border", "convert", "lu_panel",
          "lu_update", "trsv", "gemv", "krylov", "update", "lu_diag", "assemble32")
PEAKS = {"hbm_gbs": 6688.0, "bf16_tflops": 1963.0, "bf16_tflops_sustained": 1700.0,
         "sm_max_mhz": 2070.0}
PROBLEM = types.SimpleNamespace(n=2406, pairs=800 * 8000)
CLOCKS = {"sm_mhz": 2070.0}
SOLVE = {"outer_mean": 3.0, "inner_mean": 3.85}


def _phases(**ms_spans):
    ms = {p: 0.0 for p in PHASES}
    spans = {p: 0 for p in PHASES}
    for p, (m, k) in ms_spans.items():
        ms[p], spans[p] = m, k
    return ms, spans


def _check(rec):
    for key in ("kernel", "bound", "achieved", "peak", "unit", "frac", "work_per_launch",
                "launches"):
        assert key in rec, key
    assert rec["achieved"] > 0 and rec["peak"] > 0
    assert rec["frac"] == pytest.approx(rec["achieved"] / rec["peak"])


def test_separate_kernel_schedule():
    ms, spans = _phases(lu_diag=(0.9, 38), lu_update=(0.65, 38), lu_panel=(0.5, 76),
                        assemble=(0.47, 1), krylov=(0.3, 1))
    recs = bench._rooflines(ms, spans, PROBLEM, PEAKS, "measured", CLOCKS, SOLVE)
    assert {"lu_diag", "lu_update", "assemble", "solve"} <= set(recs)
    for r in recs.values():
        _check(r)
    # per launch: 0.9 ms / 38 diagonal inverses; the first of a factorisation is the
    # inverse alone (2 * 64^3 flops), the other 37 add the lookahead and staged-tile
    # products (8 * 64^3 flops)
    w = (2 * 64 ** 3 + 37 * 8 * 64 ** 3) / 38
    assert recs["lu_diag"]["work_per_launch"] == pytest.approx(w)
    assert recs["lu_diag"]["achieved"] == pytest.approx(w / (0.9e-3 / 38) / 1e12)


def test_fused_schedule():
    ms, spans = _phases(lu_update=(1.05, 1), assemble=(0.47, 1), krylov=(0.3, 1))
    recs = bench._rooflines(ms, spans, PROBLEM, PEAKS, "measured", CLOCKS, SOLVE)
    assert "lu_diag" not in recs
    rec = recs["lu_update"]
    _check(rec)
    assert rec["kernel"].startswith("k_gj_fused")
    nblk = -(-PROBLEM.n // 64)
    assert rec["blocks"] == nblk
    assert rec["us_per_block"] == pytest.approx(1.05e3 / nblk)
    assert rec["work_per_launch"] == pytest.approx(8.0 * PROBLEM.n ** 2 * nblk)


def test_traffic_record_follows_its_source(tmp_path, monkeypatch):
    # DRAM bytes from an ncu capture are reported only while the kernel's
    # source file is the one captured (SHA-1 prefix); n^2 scaling from the
    # captured size
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel, as captured")
    sha = hashlib.sha1(b"kernel, as captured").hexdigest()[:12]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.NCU_TRAFFIC, "k_test", {"bytes": 1000.0, "file": "k.cu",
                                                      "sha1": sha, "n": 100})
    assert bench._traffic("k_test", 200) == pytest.approx(4000.0)
    src.write_bytes(b"kernel, edited since")
    assert bench._traffic("k_test", 200) is None
    assert bench._traffic("k_unknown", 200) is None


def test_traffic_records_name_existing_sources():
    for kernel, rec in bench.NCU_TRAFFIC.items():
        assert os.path.exists(os.path.join(bench.ROOT, rec["file"])), kernel
        if rec["bytes"] is not None:
            assert len(rec["sha1"]) == 12, kernel
