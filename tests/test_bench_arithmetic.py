"""The bench's roofline arithmetic, on the CPU (no device: the functions take the library's
reported times and schedules as plain numbers).

The reported fractions rest on three things pinned here: the algorithmic bytes of a pass for
each read of K (4 n^2 + n for the full square, 4 n (n + 1) / 2 + n for the packed triangle,
half of each for a half-precision K), which launch time each form divides them by (the stream
without its fold for the symmetric pass, the whole reduction for the full square, the loop
time for the one-launch fit), and that an ncu traffic record is used only for the workload
and kernel source it was taken on.
"""
import types

import pytest

import bench

PK = {"hbm": 6681.5, "bf16": 1945.3, "sm_mhz": 2070.0, "source": "measured"}
N, K = 70000, 10
WL = types.SimpleNamespace(n=N, k=K, name="images_n70000_d784_k10_gauss_fp32")


def _prof(k_pass_used, sym_form, schedule, passes=50, reduce_ms=0.0, fold_ms=0.0, loop_ms=0.0, assign_ms=1.0):
    info = {"k_pass_used": k_pass_used, "sym_form": sym_form, "schedule": schedule, "reduce_ms": reduce_ms,
            "fold_ms": fold_ms, "loop_ms": loop_ms, "assign_ms": assign_ms}
    return [{"iterations": passes, "info": info}]


def test_algorithmic_bytes_of_the_packed_triangle():
    b = bench.sym_bytes(N, K, 138, True, 4)
    assert b["algorithmic"] == 2 * N * (N + 1) + N                 # 9.80 GB: unique FP32 entries + labels
    h = bench.sym_bytes(N, K, 70, True, 2)
    assert h["algorithmic"] == N * (N + 1) + N                     # 4.90 GB at 2 bytes an entry
    T = (N + 127) // 128
    assert b["packed_tiles"] == 65536 * T * (T + 1) / 2 and h["packed_tiles"] == 32768 * T * (T + 1) / 2
    assert b["slot_stores"] == 4 * 138 * K * N


def test_symmetric_pass_divides_by_the_stream_without_its_fold():
    prof = _prof(1, 2, [4, 3, 138, 12], reduce_ms=50 * 1.78, fold_ms=50 * 0.09)
    r = bench.pass_roofline(WL, prof, PK)
    assert r["kernel"] == "reduce_sym_sorted_kernel"
    assert r["avg_launch_ms"] == pytest.approx(1.69)
    assert r["achieved"] == pytest.approx((2 * N * (N + 1) + N) / 1.69e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PK["hbm"])


def test_tensor_core_symmetric_form_counts_two_bytes_an_entry():
    prof = _prof(1, 3, [8, 5, 70, 16], reduce_ms=50 * 0.883, fold_ms=50 * 0.06)
    r = bench.pass_roofline(WL, prof, PK, "fp16")
    assert r["kernel"] == "reduce_sym_mma_kernel"
    assert r["algorithmic_bytes_per_launch"] == N * (N + 1) + N
    T = (N + 127) // 128
    assert r["moved_bytes_per_launch"]["labels"] == 2 * 256 * 16 * T * (T + 1) / 2   # one-hot operands
    assert r["frac"] == pytest.approx((N * (N + 1) + N) / 0.823e-3 / 1e9 / PK["hbm"])


def test_full_square_forms():
    r = bench.pass_roofline(WL, _prof(2, 0, [0, 0, 0, 0], reduce_ms=50 * 3.0), PK)
    assert r["kernel"] == "reduce_kernel" and r["algorithmic_bytes_per_launch"] == 4 * N * N + N
    h = bench.pass_roofline(WL, _prof(2, 0, [0, 4, 0, 16], reduce_ms=50 * 1.51), PK, "fp16")
    assert h["kernel"] == "batched_mma_kernel" and h["algorithmic_bytes_per_launch"] == 2 * N * N + N
    assert h["traffic"] is None                                     # no record for this kernel
    assert h["frac"] == pytest.approx((2 * N * N + N) / 1.51e-3 / 1e9 / PK["hbm"])


def test_one_launch_fit_is_measured_against_l2_ingest():
    wl = types.SimpleNamespace(n=2000, k=8, name="blobs_n2000_d16_k8_poly")
    r = bench.pass_roofline(wl, _prof(3, 0, [0, 0, 0, 0], passes=30, loop_ms=30 * 0.02), PK)
    peak = bench.L2_INGEST_B_PER_CLK_SM * bench.GB300_SMS * PK["sm_mhz"] * 1e6 / 1e9
    assert r["bound"] == "l2" and r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx((4 * 2000 * 2000 + 2000) / 0.02e-3 / 1e9)


def test_traffic_records_apply_only_to_their_workload_and_source():
    got = bench.recorded_traffic("reduce_sym_sorted_kernel", "reduce_sym.cu", WL.name)
    assert got is not None and got > 2 * N * (N + 1)                 # a launch moves at least the triangle
    assert bench.recorded_traffic("reduce_sym_sorted_kernel", "reduce_sym.cu", "rings_n20000_d8_k4_gauss") is None
    # a record checked against another source file's hash is stale, and is not used
    assert bench.recorded_traffic("reduce_sym_sorted_kernel", "iterate.cu", WL.name) is None
    assert bench.recorded_traffic("no_such_kernel", "reduce_sym.cu", WL.name) is None
