"""Host-side helpers of bench.py (no GPU): the work counts the roofline divides by, and the DRAM
traffic record's key and scaling."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench


def _log(rows):
    """A bond log [steps=1][layers=6][bonds][8] with the given (mD, nD, l, sweeps, flags, chi) rows
    on layer 0 and nothing elsewhere."""
    rec = np.zeros((1, 6, max(1, len(rows)), 8), dtype=np.int32)
    for b, r in enumerate(rows):
        rec[0, 0, b, :len(r)] = r
    return rec


def test_sketch_elements_counts_both_sketches_per_power_iteration():
    q = bench.RSVD_POWER
    rec = _log([(512, 300, 160, 8, 0, 128), (0, 0, 0, 0, 0, 0), (100, 400, 96, 8, 0, 64)])
    want = ((1 + q) * 512 + (q + 1) * 300) * 160 + ((1 + q) * 400 + (q + 1) * 100) * 96
    assert bench.sketch_elements(rec) == want


def test_hqr_and_rsvd_flops_follow_the_householder_counts():
    m, l = 700, 160
    assert bench.hqr_flops(m, l) == pytest.approx(16.0 * (m * l * l - l ** 3 / 3.0))
    assert bench.hqr_flops(10, 20) == 0.0                        # wide: not a QR the kernel runs
    q = bench.RSVD_POWER
    rec = _log([(m, 400, l, 8, 0, 128)])
    fl_qr, fl_gemm = bench.rsvd_flops(rec)
    assert fl_qr == pytest.approx((1 + q) * bench.hqr_flops(m, l) + (q + 1) * bench.hqr_flops(400, l))
    assert fl_gemm == pytest.approx(8.0 * m * 400 * l * (2 * q + 3) + 8.0 * (m + 400) * l * 128)


def test_svd_flops_with_rank_reduce_to_the_full_count():
    m, n = 300, 200
    full = bench.svd_flops_full(m, n)
    # the rank-k count at k = n: QR 4(4mn^2 - 2n^2(m+n) + 4n^3/3), the n x n SVD and U = D V
    k = n
    qr = 4.0 * (4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k ** 3 / 3.0)
    small = 4.0 * (4.0 * n * n * k + 8.0 * n * k * k + 9.0 * k ** 3)
    assert bench.svd_flops(m, n, 0) == pytest.approx(qr + small + 8.0 * m * n * k)
    assert bench.svd_flops(m, n, 50) < bench.svd_flops(m, n, 0) and full > 0


def test_traffic_record_scales_per_element_and_checks_the_source(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2201_05529_gb300", "csrc", "hqr_grid.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    rec = tmp_path / "traffic.json"
    rec.write_text(json.dumps({"sources": ["hqr_grid.cu"], "sha": {"hqr_grid.cu": sha},
                               "dram_bytes_per_sketch_element": 18.0, "how": "test"}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(rec))
    assert bench.traffic_record(["hqr_grid.cu"], 1000.0) == (18000.0, "test")
    # another kernel's sources, or a stale hash: no traffic figure
    assert bench.traffic_record(["qrcp.cu"])[0] is None
    rec.write_text(json.dumps({"sources": ["hqr_grid.cu"], "sha": {"hqr_grid.cu": "0" * 16},
                               "dram_bytes_per_sketch_element": 18.0}))
    assert bench.traffic_record(["hqr_grid.cu"], 1000.0)[0] is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.json"))
    assert bench.traffic_record(["hqr_grid.cu"], 1000.0)[0] is None
