"""Host logic of bench.py on the CPU: the algorithmic work model of the
gather/FFT stages, the roofline arithmetic built on it, the scaling of the
committed ncu traffic, the stage-to-kernel map and the end-to-end timing
helper (the L2 flush stays outside the timed call)."""
import time

import pytest

import bench


def test_stage_model_counts_the_fft_butterflies():
    """exact-2^22 level 0: two shifts of M = 8192 points; an M-point radix-2
    FFT has (M/2) log2 M = 4096 * 13 butterflies, 68 FP32 instructions each
    in float-float, and reads 8192 complex64 samples per shift."""
    wl = bench.WORKLOADS["exact-2^22"]
    m = wl.stage_model("gather_fft_l0")
    assert m == {"bytes": 2 * 8192 * 8, "fft_ops": 2 * 4096 * 13 * 68}
    m3 = wl.stage_model("gather_fft_l3")  # M = 1024 at level 3
    assert m3 == {"bytes": 2 * 1024 * 8, "fft_ops": 2 * 512 * 10 * 68}
    assert wl.stage_model("decode_l2") is None


def test_stage_model_of_the_four_step_fft():
    """exact-2^27: M = 2^18 runs as columns of 2^9 points (reading the
    input) then rows of 2^9 points."""
    wl = bench.WORKLOADS["exact-2^27"]
    cols, rows = wl.stage_model("gather_cols_l0"), wl.stage_model("fft_rows_l0")
    half = 2 * (1 << 17)  # two shifts x M/2 butterflies per radix-2 stage
    assert cols == {"bytes": 2 * (1 << 18) * 8, "fft_ops": half * 9 * 68}
    assert rows == {"bytes": 0, "fft_ops": half * 9 * 68}


def test_roofline_of_the_dominant_gather_fft():
    wl = bench.WORKLOADS["exact-2^22"]
    stages = {"gather_fft_l0": (2.0, 1), "decode_l3": (1.0, 1)}  # ms in all, launches
    roof = bench.roofline(wl, stages, 152, {"sm_mhz": 2000.0})
    assert roof["kernel"] == "k_gather_fft" and roof["bound"] == "alu"
    assert roof["share"] == pytest.approx(2.0 / 3.0)
    ops = 2 * 4096 * 13 * 68 * 152
    assert roof["achieved"] == pytest.approx(ops / 2e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    hbm = roof["hbm_view"]
    assert hbm["achieved_gbs"] == pytest.approx(2 * 8192 * 8 * 152 / 2e-3 / 1e9)
    assert hbm["frac"] == pytest.approx(hbm["achieved_gbs"] / hbm["peak_gbs"])


def test_roofline_claims_no_model_for_the_solvers():
    wl = bench.WORKLOADS["exact-2^22"]
    roof = bench.roofline(wl, {"decode_l3": (3.0, 1), "gather_fft_l0": (1.0, 1)}, 152, None)
    assert roof["kernel"] == "k_iter_decode<a=4>"
    assert roof["frac"] is None and roof["achieved"] is None


def test_ncu_traffic_scales_with_the_signals():
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        ent = json.load(f)["exact-2^22"]["k_gather_fft"]
    got = bench.ncu_traffic("exact-2^22", "k_gather_fft", 76)
    if ent["source_sha"] == bench.kernel_source_hash("k_gather_fft"):
        assert got == pytest.approx(ent["dram_bytes_per_launch"] * 76 / ent["signals_per_launch"])
    else:  # counters taken on other kernel text are not reported
        assert got is None
    assert bench.ncu_traffic("exact-2^22", "k_iter_fold<a=2>", 152) is None
    assert bench.ncu_traffic("no-such-workload", "k_gather_fft", 152) is None


def test_kernel_of_maps_stages_to_kernels():
    assert bench.kernel_of("gather_fft_l1") == "k_gather_fft"
    assert bench.kernel_of("gather_fft_consecutive", 1 << 15) == "k_fft4_cols"
    assert bench.kernel_of("gather_fft_consecutive", 1 << 13) == "k_gather_fft"
    assert bench.kernel_of("gather_cols_l2") == "k_fft4_cols"
    assert bench.kernel_of("fft_rows_l0") == "k_fft4_rows"
    assert bench.kernel_of("fold_l2") == "k_iter_fold<a=3>"
    assert bench.kernel_of("decode_l0") == "k_iter_decode<a=1>"
    assert bench.kernel_of("finalize") == "k_finalize"


def test_host_timed_steps_leaves_the_flush_out():
    class _Cuda:
        calls = 0

        @staticmethod
        def synchronize():
            _Cuda.calls += 1

    class _Torch:
        cuda = _Cuda

    seen = []
    t = bench.host_timed_steps(_Torch, lambda i: (seen.append(i), time.sleep(0.01)), 3,
                               lambda: time.sleep(0.05))
    assert seen == [0, 1, 2] and _Cuda.calls == 3
    assert 0.03 <= t < 0.1  # three 10 ms calls, none of the three 50 ms flushes
