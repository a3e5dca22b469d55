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
N_SYS, PAIRS = 27648, 9200 * 92000
SM_MHZ = 2070.0
SOLVE = {"outer_mean": 3.5, "inner_mean": 20.0}


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


def test_records_of_every_kernel_family():
    nblk = -(-N_SYS // 64)
    ms, spans = _phases(lu_diag=(15.0, nblk), lu_update=(660.0, nblk), lu_panel=(28.0, 2 * nblk),
                        assemble=(220.0, 2), assemble32=(2.2, 1), krylov=(180.0, 2))
    recs = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, SOLVE)
    assert {"lu_diag", "lu_update", "assemble", "assemble32", "krylov"} <= set(recs)
    for r in recs.values():
        _check(r)
    # per launch: the first diagonal inverse of a factorisation is the inverse
    # alone (2 * 64^3 flops), the others add the lookahead and staged-tile
    # products (8 * 64^3 flops); the peak is the whole GPU's FP32 rate
    w = (2 * 64 ** 3 + (nblk - 1) * 8 * 64 ** 3) / nblk
    assert recs["lu_diag"]["work_per_launch"] == pytest.approx(w)
    assert recs["lu_diag"]["achieved"] == pytest.approx(w / (15e-3 / nblk) / 1e12)
    assert recs["lu_diag"]["peak"] == pytest.approx(152 * 128 * 2 * SM_MHZ * 1e6 / 1e12)
    # the update: 8 n^2 bytes per launch against the measured HBM copy rate
    assert recs["lu_update"]["work_per_launch"] == pytest.approx(8.0 * N_SYS ** 2)
    assert recs["lu_update"]["peak"] == PEAKS["hbm_gbs"]
    # FP64 assembly: 40 operations per pair against 2 FP64 lanes per SM per clock
    a = recs["assemble"]
    assert a["work_per_launch"] == pytest.approx(40.0 * PAIRS)
    assert a["peak"] == pytest.approx(625.0)
    assert a["pairs_per_s"] == pytest.approx(PAIRS / 0.110)
    # FP32 copy: pairs against the pair peak 152 x 128 x clock / 20
    assert recs["assemble32"]["peak"] == pytest.approx(152 * 128 * SM_MHZ * 1e6 / 20)
    # solve: (outer + inner + 1) FP64 matrix passes (the extra one for the
    # extended residual's ||A||_inf) and (outer + inner + 1) FP32 ones; FP64
    # operations: 3 per entry and outer step, 1 per entry and inner step + 1
    k = recs["krylov"]
    assert k["work_per_launch"] == pytest.approx(8.0 * N_SYS ** 2 * 24.5 + 4.0 * N_SYS ** 2 * 24.5)
    assert k["fp64_gops"] * 1e9 * (k["ms_per_launch"] / 1e3) == pytest.approx(
        (3 * SOLVE["outer_mean"] + SOLVE["inner_mean"] + 1) * N_SYS ** 2)


@pytest.mark.parametrize("f16", [True, False])
def test_two_level_factorisation_is_rated_against_its_closer_roofline(f16):
    # the two-level schedule has one panel span and one update span per
    # 256-column block and no diagonal-inverse spans; its update is a rank-256
    # product, 3 passes x 2 n^2 256 tensor flops per launch (FP16 pairs at the
    # BF16 rate, or split TF32 at the derived TF32 rate), which also reads and
    # writes the FP32 matrix (8 n^2 bytes); the record takes the larger fraction
    nb = -(-N_SYS // 256)
    for upd_ms in (265.0, 40.0):
        ms, spans = _phases(lu_panel=(40.0, nb), lu_update=(upd_ms, nb), assemble=(220.0, 2))
        recs = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, SOLVE,
                               update_f16=f16)
        u = recs["lu_update"]
        _check(u)
        t = upd_ms * 1e-3 / nb
        fl = 3 * 2.0 * N_SYS ** 2 * 256
        tp = PEAKS["bf16_tflops_sustained"] * (1.0 if f16 else 1.1 / 2.25)
        assert u["tensor_tflops"] == pytest.approx(fl / t / 1e12)
        assert u["tensor_peak"] == pytest.approx(tp)
        assert u["hbm_gbs"] == pytest.approx(8.0 * N_SYS ** 2 / t / 1e9)
        tfrac, hfrac = fl / t / 1e12 / tp, 8.0 * N_SYS ** 2 / t / 1e9 / PEAKS["hbm_gbs"]
        assert u["frac"] == pytest.approx(max(tfrac, hfrac))
        assert u["bound"] == ("hbm" if hfrac >= tfrac else "tensor")
        assert "lu_diag" not in recs and "lu_panel" in recs


def test_records_are_skipped_for_phases_that_did_not_run():
    ms, spans = _phases(assemble=(80.0, 1), krylov=(100.0, 1))
    recs = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, SOLVE)
    assert set(recs) == {"assemble", "krylov"}


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


def test_spans_alone_excludes_overlapping_launches():
    tr = [("assemble", 0.0, 10.0), ("lu_update", 5.0, 20.0), ("assemble", 30.0, 40.0),
          ("krylov", 35.0, 50.0), ("assemble", 60.0, 65.0), ("lu_panel", 65.0, 70.0)]
    assert bench.spans_alone(tr, "assemble", ("lu_update", "lu_panel")) == [10.0, 5.0]


def test_float_pair_gmres_products_leave_the_fp64_count():
    ms, spans = _phases(assemble=(80.0, 1), krylov=(100.0, 1))
    a = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, SOLVE)["krylov"]
    b = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, SOLVE,
                        arnoldi_df=True)["krylov"]
    assert a["work_per_launch"] == b["work_per_launch"]  # the same bytes either way
    t = a["ms_per_launch"] / 1e3
    assert (a["fp64_gops"] - b["fp64_gops"]) * 1e9 * t == pytest.approx(
        SOLVE["inner_mean"] * N_SYS ** 2)


def test_working_precision_residuals_are_counted_as_what_they_are():
    # 3.5 refinement steps a solve, 2 of them on an exact residual and 2.5
    # working-precision residuals formed (1.5 kept, 1 rejected): 4.5 + 20 + 1
    # passes over an 8-byte matrix, 24.5 over M; FP64 work only in the exact
    # residuals and the ||A||_inf pass when the other products use the
    # float-pair copy, the working-precision products added when they do not
    ms, spans = _phases(assemble=(80.0, 1), krylov=(100.0, 1))
    st = dict(SOLVE, exact_mean=2.0, working_mean=2.5)
    k = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, st,
                        arnoldi_df=True)["krylov"]
    assert k["work_per_launch"] == pytest.approx(8.0 * N_SYS ** 2 * 25.5 + 4.0 * N_SYS ** 2 * 24.5)
    t = k["ms_per_launch"] / 1e3
    assert k["fp64_gops"] * 1e9 * t == pytest.approx((3 * 2.0 + 1) * N_SYS ** 2)
    f = bench.rooflines(ms, spans, N_SYS, PAIRS, PEAKS, "measured", SM_MHZ, st)["krylov"]
    assert f["fp64_gops"] * 1e9 * t == pytest.approx((3 * 2.0 + 1 + 20.0 + 2.5) * N_SYS ** 2)


def test_critical_path_charges_overlap_to_the_work_that_ends_last():
    # the factorisation (a chain: update 0-20 and panel 18-30, one run) with the
    # FP64 assembly beside it (5-25 ms, ends first: off the critical path),
    # then the assembly alone (30-40) and the solve (40-60, 62-70); the gap
    # (60-62) is charged to nothing
    tr = [("lu_update", 0.0, 20.0), ("lu_panel", 18.0, 30.0), ("assemble", 5.0, 25.0),
          ("assemble", 30.0, 40.0), ("krylov", 40.0, 60.0), ("krylov", 62.0, 70.0)]
    c = bench.critical_ms(tr)
    assert c["lu"] == pytest.approx(30.0)
    assert c["assemble"] == pytest.approx(10.0)
    assert c["krylov"] == pytest.approx(28.0)
    assert sum(c.values()) == pytest.approx(68.0)
    # an assembly that outlasts the factorisation is on the path for its tail
    c2 = bench.critical_ms([("lu_update", 0.0, 10.0), ("lu_panel", 10.1, 20.0),
                            ("assemble", 5.0, 26.0)])
    assert c2["lu"] == pytest.approx(5.0)
    assert c2["assemble"] == pytest.approx(21.0)
