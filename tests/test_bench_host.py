"""bench.py's host-side arithmetic (CPU): the roofline entries built from
per-launch times, the choice of the dominant kernel, the traffic lookup and
the launch and rate bookkeeping of the JSON line."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

PEAKS = dict(hbm_gbs=6697.2, sm_max_mhz=2070.0, source="measured")


def phases(**ms):
    return [ms.get(k, 0.0) for k in bench.KERNELS]


def test_alu_entries_count_pairs_against_the_fp32_lane_rate():
    M = N = 20000
    r = bench.roofline_entries(phases(e_pass_a=0.1, e_pass_b=0.2), M, N, M, PEAKS)
    # pass A: 7 FP32 ops per pair -> 128 / 7 pairs per clock per SM
    peak_a = 152 * 2070e6 * 128 / 7
    assert r["e_pass_a"]["achieved"] == pytest.approx(M * N / 1e-4 / 1e9)
    assert r["e_pass_a"]["frac"] == pytest.approx(M * N / 1e-4 / peak_a)
    # pass B: 12 ops per pair
    assert r["e_pass_b"]["peak"] == pytest.approx(152 * 2070e6 * 128 / 12 / 1e9)
    assert r["e_pass_a"]["bound"] == r["e_pass_b"]["bound"] == "alu"
    # kernels that did not run are absent
    assert "m_project" not in r


def test_hbm_entries_count_the_basis_once_per_product():
    M, N, K = 20000, 20000, 20000
    r = bench.roofline_entries(phases(m_project=0.24, m_expand=0.25), M, N, K, PEAKS)
    assert r["m_project"]["bytes"] == M * K * 4 + M * 16
    assert r["m_expand"]["bytes"] == M * K * 4 + K * 16
    gbs = (M * K * 4 + M * 16) / 0.24e-3 / 1e9
    assert r["m_project"]["achieved"] == pytest.approx(gbs)
    assert r["m_project"]["frac"] == pytest.approx(gbs / 6697.2)
    # an FP16 basis streams half the bytes
    r16 = bench.roofline_entries(phases(m_project=0.24), M, N, K, PEAKS, es=2)
    assert r16["m_project"]["bytes"] == M * K * 2 + M * 16


def test_dominant_kernel_counts_both_products_of_the_streaming_kernel():
    M = N = K = 20000
    r = bench.roofline_entries(phases(e_pass_a=0.10, e_pass_b=0.17, m_project=0.24, m_expand=0.25), M, N, K, PEAKS)
    name, d = bench.dominant_kernel(r)
    assert name == "colsum_bulk"
    assert d["launches_per_iter"] == 2
    assert d["ms"] == pytest.approx(0.245)
    # with a small basis the E-step passes dominate
    r = bench.roofline_entries(phases(e_pass_a=0.10, e_pass_b=0.17, m_project=0.01, m_expand=0.01), M, N, 200,
                               PEAKS)
    assert bench.dominant_kernel(r)[0] == "e_pass_b"


def test_traffic_is_reported_only_for_the_recorded_workload_and_source():
    rec = bench.traffic_for("colsum_bulk", "fp32_m20000_full")
    assert rec is None or rec > 1.6e9          # null once the kernel's source has changed
    assert bench.traffic_for("colsum_bulk", "fp32_m8000_full") is None
    assert bench.traffic_for("no_such_kernel", "fp32_m20000_full") is None


def test_job_rate_is_all_ranks_steps_over_the_slowest_rank():
    assert bench.job_rate(100, 1, 50.0) == pytest.approx(2000.0)
    assert bench.job_rate(100, 4, 200.0) == pytest.approx(2000.0)


def test_timed_launch_count():
    # one piece: 11 launches per iteration + 5 per registration
    assert bench.timed_launches(100, 30, 1) == 30 * (100 * 11 + 5)
    # 3 pieces: 19 per iteration except the 11 evented ones (0, 10, .., 90, 99)
    assert bench.timed_launches(100, 30, 3) == 30 * (11 * 11 + 19 * 89 + 5) == 54510
    # a registration of 1 iteration: that iteration carries the events
    assert bench.timed_launches(1, 4, 3) == 4 * (11 + 5)
