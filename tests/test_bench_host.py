"""Host logic of bench.py on the CPU: the algorithmic work model of the
gather/FFT stages and of the decoders, the roofline arithmetic built on it,
the scaling of the committed ncu traffic, the stage-to-kernel map, the bytes
that cross the host link and the end-to-end timing helper (the L2 flush
stays outside the timed call)."""
import time

import pytest

import bench


def test_stage_model_counts_the_fft_work():
    """exact-2^22 level 0: two shifts of M = 8192 points read 8192 complex64
    samples each; the FFT's flops are 5 M log2 M per shift; an M-point
    radix-2 FFT has (M/2) log2 M = 4096 * 13 butterflies, 68 FP32
    instructions each in float-float."""
    wl = bench.WORKLOADS["exact-2^22"]
    m = wl.stage_model("gather_fft_l0")
    assert m == {"bytes": 2 * 8192 * 8, "fft_flops": 5 * 2 * 8192 * 13,
                 "ff_instr": 2 * 4096 * 13 * 68}
    m3 = wl.stage_model("gather_fft_l3")  # M = 1024 at level 3
    assert m3 == {"bytes": 2 * 1024 * 8, "fft_flops": 5 * 2 * 1024 * 10,
                  "ff_instr": 2 * 512 * 10 * 68}
    assert wl.stage_model("decode_l2") is None
    # the four levels read 8 B x (2 + 1 + 1/2 + 1/4) = 30 B per level-0 row
    assert wl.h2d_per_signal() == 30 * 8192


def test_stage_model_of_the_four_step_fft():
    """exact-2^27: M = 2^18 runs as columns of 2^9 points (reading the
    input) then rows of 2^9 points; together 5 M log2 M flops per shift."""
    wl = bench.WORKLOADS["exact-2^27"]
    cols, rows = wl.stage_model("gather_cols_l0"), wl.stage_model("fft_rows_l0")
    half = 2 * (1 << 17)  # two shifts x M/2 butterflies per radix-2 stage
    assert cols["bytes"] == 2 * (1 << 18) * 8 and rows["bytes"] == 0
    assert cols["ff_instr"] == rows["ff_instr"] == half * 9 * 68
    assert cols["fft_flops"] + rows["fft_flops"] == 5 * 2 * (1 << 18) * 18


def test_roofline_of_a_dominant_gather_fft_counts_input_bytes():
    """The gather/FFT kernels are bound by HBM on the method's input bytes;
    the FFT flops against the FP32 peak and the float-float issue rate are
    reported beside the fraction, not as it."""
    wl = bench.WORKLOADS["exact-2^22"]
    stages = {"gather_fft_l0": (2.0, 1), "gather_fft_l1": (0.5, 1), "decode_l3": (1.0, 1)}
    roof = bench.roofline(wl, stages, 152, {"sm_mhz": 2000.0}, [9000, 5000, 3000, 1000])
    assert roof["kernel"] == "k_gather_fft<FF, 8>" and roof["bound"] == "hbm"
    assert roof["share"] == pytest.approx(2.5 / 3.5)
    byts = (2 * 8192 * 8 + 2 * 4096 * 8) * 152
    assert roof["achieved"] == pytest.approx(byts / 2.5e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["peak"] == bench.measured_peaks()[0]["hbm_gbs"]
    fl = roof["fp32_flop_view"]
    assert fl["peak_tflops"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert fl["achieved_tflops"] == pytest.approx(5 * (2 * 8192 * 13 + 2 * 4096 * 12) * 152
                                                  / 2.5e-3 / 1e12)
    diag = roof["ff_issue_diag"]
    assert diag["peak_tinstr"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert set(roof["by_kernel"]) == {"k_gather_fft<FF, 8>", "k_iter_decode<FF, 4>"}


def test_roofline_of_a_dominant_decoder_counts_fp64_flops_per_bin():
    """A decoder dominating is reported against the FP64 peak derived from
    the unit counts, on decode_flops() per queued bin of its level."""
    wl = bench.WORKLOADS["exact-2^22"]
    roof = bench.roofline(wl, {"decode_l3": (3.0, 2), "gather_fft_l0": (1.0, 2)}, 152,
                          {"sm_mhz": 2070.0}, [9000, 5000, 3000, 1000])
    assert roof["kernel"] == "k_iter_decode<FF, 4>" and roof["bound"] == "alu"
    fl = bench.decode_flops(4, 8) * 1000 * 2
    assert roof["achieved"] == pytest.approx(fl / 3e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
    assert roof["bins_per_launch"] == 1000
    # without the queue lengths no flop model is claimed
    bare = bench.roofline(wl, {"decode_l3": (3.0, 1)}, 152, None)
    assert bare["frac"] is None and bare["achieved"] is None


def test_float_float_decoders_are_measured_against_the_fp32_issue_rate():
    """The mixed path decodes one and two aliases in float-float on the FP32
    pipes: those decoders are reported against the FP32 issue rate on
    decode_ff_instr() per bin; three and four aliases (FP64) and the FP64
    path's decoders stay against the FP64 peak."""
    wl = bench.WORKLOADS["exact-2^22"]
    roof = bench.roofline(wl, {"decode_l0": (2.0, 1), "decode_l2": (1.0, 1)}, 152,
                          {"sm_mhz": 2000.0}, [900000, 90000, 15000, 2000])
    assert roof["kernel"] == "k_iter_decode<FF, 1>" and roof["unit"] == "Tinstr/s"
    assert roof["achieved"] == pytest.approx(bench.decode_ff_instr(1, 2) * 900000 / 2e-3 / 1e12)
    assert roof["peak"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert "FP32 issue" in roof["peak_note"]
    assert roof["by_kernel"]["k_iter_decode<FF, 3>"]["bound"] == "alu"
    f64 = bench.roofline(bench.WORKLOADS["exact-2^16-fp64"], {"decode_l0": (2.0, 1)}, 152,
                         {"sm_mhz": 2000.0}, [900000, 90000, 15000, 2000])
    assert f64["unit"] == "TFLOP/s"
    assert f64["achieved"] == pytest.approx(bench.decode_flops(1, 2) * 900000 / 2e-3 / 1e12)
    # one complex float-float multiply-add per complex multiply-add of the
    # flop model, one snap per root
    assert bench.decode_ff_instr(2, 4) == pytest.approx(
        bench.FF_CMA_INSTR * (bench.decode_flops(2, 4) - 8) / 8 + 2 * bench.FF_SNAP_INSTR)
    assert bench.ff_decoder("mixed", 2) and not bench.ff_decoder("mixed", 3)
    assert not bench.ff_decoder("fp64", 1)


def test_decode_flops_grow_with_the_alias_count():
    """One alias: 8 complex multiply-adds and change; four aliases with 8
    syndromes: about 1.8 kflop per bin."""
    f = [bench.decode_flops(a, 2 * a) for a in (1, 2, 3, 4)]
    assert f == sorted(f)
    assert bench.decode_flops(1, 2) == pytest.approx(8 * (2 / 3 + 1 + 1 + 2 + 2 + 2 / 3 + 1 + 2)
                                                     + 4)
    assert 1700 < bench.decode_flops(4, 8) < 2000


def test_general_path_solvers_have_flop_models():
    """The general path's singular values and per-bin solves are reported
    against the FP64 peak on their work per bin (bins from the plan's
    counts: SVD bins, voted one-alias bins, voted multi-alias bins)."""
    wl = bench.WORKLOADS["general-2^27"]
    stages = {"gen_svals": (7.0, 1), "gen_solve": (6.0, 1), "gather_fft_random": (0.4, 1)}
    roof = bench.roofline(wl, stages, 4, {"sm_mhz": 2070.0}, [800000, 200000, 50000])
    assert roof["kernel"] == "k_gen_svals" and roof["bound"] == "alu"
    assert roof["achieved"] == pytest.approx(bench.svals_flops(4) * 800000 / 7e-3 / 1e12)
    sol = roof["by_kernel"]["k_gen_solve"]
    assert sol["bound"] == "alu" and sol["frac"] > 0
    # 4 x 4 Hankel, 5 sweeps of 6 pairs at 140 flops
    assert bench.svals_flops(4) == 5 * 6 * 140
    assert bench.solve_flops(1, 32, 9) > 32 * 14


def test_ncu_traffic_scales_with_the_signals():
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        ent = json.load(f)["exact-2^22"]["k_gather_fft"]
    got = bench.ncu_traffic("exact-2^22", "k_gather_fft<FF, 8>", 76)
    if ent["source_sha"] == bench.kernel_source_hash("k_gather_fft"):
        assert got == pytest.approx(ent["dram_bytes_per_launch"] * 76 / ent["signals_per_launch"])
    else:  # counters taken on other kernel text are not reported
        assert got is None
    assert bench.ncu_traffic("exact-2^22", "k_iter_fold<FF, 2>", 152) is None
    assert bench.ncu_traffic("no-such-workload", "k_gather_fft", 152) is None


def test_kernel_of_maps_stages_to_template_instances():
    k = bench.kernel_of
    assert k("gather_fft_l1") == k("gather_fft_l3") == "k_gather_fft<FF, 8>"
    assert k("gather_fft_l0", 8192, "fp64") == "k_gather_fft<F64, 8>"
    assert k("gather_fft_consecutive", 1 << 15) == "k_fft4_cols<FF, 8>"
    assert k("gather_fft_consecutive", 1 << 13) == "k_gather_fft<FF, 8>"
    assert k("gather_cols_l2") == "k_fft4_cols<FF, 8>"
    assert k("fft_rows_l0") == "k_fft4_rows<FF, 8>"
    assert k("fold_l2") == "k_iter_fold<FF, 3>"
    assert k("decode_l0") == "k_iter_decode<FF, 1>"
    assert k("decode_fixed_a3", 8192, "mixed", 4) == "k_fixed_round<FF, 3, 8>"
    assert k("extract") == "k_extract<float2, 1>"
    assert k("finalize") == "k_finalize<FF, 0>"


def test_link_bytes_count_what_crosses_the_host_link():
    """At least 64 B per level-0 row for the exact paths (above the
    algorithmic 30 B), one sector per gathered sample on the general path."""
    assert bench.WORKLOADS["exact-2^22"].link_bytes_per_signal() == 64 * 8192
    g = bench.WORKLOADS["general-2^20"]
    assert g.link_bytes_per_signal() == (6 + 9) * (1 << 15) * 32


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
