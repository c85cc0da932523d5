"""GPU parity of the exactly K-sparse transform against the FP64 oracle, through
the C ABI.  Supports must match bit-exactly; values within 1e-10 relative on
the FP64 path and 1e-4 relative (the bulk-FP32 bound) on the mixed path."""
import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

FP64_VAL_TOL = 1e-10
MIXED_VAL_TOL = 1e-4


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


def _tol_of(plan):
    p = plan.params
    return dict(zero_tol=p.zero_tol, root_tol=p.root_tol, res_tol=p.res_tol)


def _run_gpu(torch, plan, xs, cap):
    x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    out = plan.exact(x, cap)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _compare(orc, plan, xs, mode, cap, val_tol, mmax=None, scale_rel=False):
    """Run the oracle on every signal of xs and compare with the GPU result
    (value errors relative to each value, or with scale_rel to the signal's
    largest value)."""
    import torch
    idx, val, cnt, unres, ovf = _run_gpu(torch, plan, xs, cap)
    om = orc.ITER if mode == "iter" else orc.FIXED
    tol = _tol_of(plan)
    worst = 0.0
    for b in range(xs.shape[0]):
        oi, ov, ou = orc.exact(xs[b], plan.M, plan.params.a_max, om,
                               max_iters=plan.params.max_iters, cap=cap, **tol)
        n = int(cnt[b])
        gi, gv = idx[b, :n], val[b, :n]
        order = np.argsort(gi, kind="stable")
        gi, gv = gi[order], gv[order]
        assert ovf[b] == 0
        np.testing.assert_array_equal(gi, oi, err_msg=f"signal {b}: supports differ")
        assert unres[b] == ou, f"signal {b}: unresolved {unres[b]} vs {ou}"
        if n:
            den = np.abs(ov).max() if scale_rel else np.maximum(np.abs(ov), 1e-300)
            rel = np.abs(gv - ov) / den
            worst = max(worst, float(rel.max()))
    assert worst <= val_tol, worst
    return worst


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_plain_fp64_unit_magnitudes(gpu, orc, mode):
    """N = 2^16 complex128, K = 64, |X| = 1, M = 256 (d = 256), FP64 path."""
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 16, 64, 256
    plan = Plan(N, K, N // M, mode, "fp64", max_signals=8)
    xs = np.stack([siggen.exact_signal(N, K, s)[0] for s in range(8)])
    _compare(orc, plan, xs, mode, cap=4 * M, val_tol=FP64_VAL_TOL)


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_mixed_full_size(gpu, orc, mode):
    """N = 2^22 complex64, K = 4096, |X| ~ U[1,10], M = 2^13: the headline
    configuration, four signals in one batch."""
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 22, 4096, 1 << 13
    plan = Plan(N, K, N // M, mode, "mixed", max_signals=4)
    xs, _, _ = siggen.batch_exact(N, K, range(100, 104), mag=(1, 10), dtype=np.complex64)
    _compare(orc, plan, xs, mode, cap=2 * K, val_tol=MIXED_VAL_TOL)


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_fp64_full_size(gpu, orc, mode):
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 22, 4096, 1 << 13
    plan = Plan(N, K, N // M, mode, "fp64", max_signals=2)
    xs = np.stack([siggen.exact_signal(N, K, s, mag=(1, 10))[0] for s in (7, 8)])
    _compare(orc, plan, xs, mode, cap=2 * K, val_tol=FP64_VAL_TOL)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("N,K,M", [(1 << 10, 6, 32), (1 << 12, 100, 256), (1 << 14, 600, 1024),
                                   (1 << 18, 2048, 4096), (1 << 13, 2000, 8192),
                                   (1 << 17, 6000, 1 << 14), (1 << 18, 7000, 1 << 15),
                                   (1 << 20, 30000, 1 << 16)])
def test_sizes_span_tiles(gpu, orc, prec, N, K, M):
    """Fold blocks of 256 bins: M = 32 is a partial block; M = 8192 is the
    largest one-CTA FFT and M >= 2^14 goes through the four-step FFT (every
    level of M = 2^16 does); K / M from 0.2 to 0.5 exercises every level."""
    from paper_1407_8315_gb300 import Plan
    dt = np.complex128 if prec == "fp64" else np.complex64
    for mode in ("iter", "fixed"):
        plan = Plan(N, K, N // M, mode, prec, max_signals=3)
        xs, _, _ = siggen.batch_exact(N, K, [N + K + i for i in range(3)], mag=(1, 10), dtype=dt)
        _compare(orc, plan, xs, mode, cap=4 * M,
                 val_tol=FP64_VAL_TOL if prec == "fp64" else MIXED_VAL_TOL)


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_large_single_signal(gpu, orc, mode):
    """N = 2^27 complex64 (1 GiB), K = 2^16, M = 2^18 (d = 512): four-step
    FFTs at every level."""
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 27, 1 << 16, 1 << 18
    plan = Plan(N, K, N // M, mode, "mixed", max_signals=1)
    xs = siggen.exact_signal(N, K, 2027, mag=(1, 10), dtype=np.complex64)[0][None, :]
    _compare(orc, plan, xs, mode, cap=2 * K, val_tol=MIXED_VAL_TOL)


def test_fig1_worked_example_on_gpu(gpu, orc):
    from paper_1407_8315_gb300 import Plan
    x = siggen.tone_signal(8, [0, 2, 4], [1.0, 2.0j, -3.0 + 0.5j])[None, :]
    plan = Plan(8, 3, 2, "iter", "fp64", a_max=2, max_iters=1)
    idx, val, cnt, unres, _ = _run_gpu(gpu, plan, x, 8)
    assert idx[0, :cnt[0]].tolist() == [2] and unres[0] == 1
    plan = Plan(8, 3, 2, "iter", "fp64", a_max=2, max_iters=2)
    idx, val, cnt, unres, _ = _run_gpu(gpu, plan, x, 8)
    assert sorted(idx[0, :cnt[0]].tolist()) == [0, 2, 4] and unres[0] == 0
    plan = Plan(8, 3, 2, "fixed", "fp64", a_max=2)
    idx, val, cnt, unres, _ = _run_gpu(gpu, plan, x, 8)
    assert sorted(idx[0, :cnt[0]].tolist()) == [0, 2, 4] and unres[0] == 0


def test_zero_signal_and_single_tone(gpu):
    from paper_1407_8315_gb300 import Plan
    N, M = 1 << 12, 64
    plan = Plan(N, 4, N // M, "iter", "mixed", max_signals=2)
    xs = np.zeros((2, N), np.complex64)
    xs[1] = siggen.tone_signal(N, [1234], [3 - 4j], np.complex64)
    idx, val, cnt, unres, ovf = _run_gpu(gpu, plan, xs, 4)
    assert cnt[0] == 0 and unres[0] == 0
    assert cnt[1] == 1 and idx[1, 0] == 1234 and abs(val[1, 0] - (3 - 4j)) < 1e-5


def test_capacity_overflow_is_flagged(gpu):
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 14, 200, 1024
    plan = Plan(N, K, N // M, "iter", "fp64")
    x = siggen.exact_signal(N, K, 5, mag=(1, 10))[0][None, :]
    import torch
    xt = torch.from_numpy(x).cuda()
    full = plan.exact(xt, 1024)
    small = plan.exact(xt, 256)  # cap >= K still required
    torch.cuda.synchronize()
    n_full = int(full.count[0])
    assert n_full > 150
    # a plan whose K promises more than cap is rejected up front
    with pytest.raises(Exception):
        plan.exact(xt, 100)
    assert int(small.count[0]) == min(n_full, 256)
    assert int(small.overflow[0]) == (1 if n_full > 256 else 0)


def test_batch_equals_single(gpu):
    """Signals in one batch do not interact."""
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 16, 512, 1024
    plan = Plan(N, K, N // M, "iter", "mixed", max_signals=5)
    xs, _, _ = siggen.batch_exact(N, K, range(5), mag=(1, 10), dtype=np.complex64)
    bi, bv, bc, bu, _ = _run_gpu(gpu, plan, xs, 2048)
    for b in range(5):
        si, sv, sc, su, _ = _run_gpu(gpu, plan, xs[b:b + 1], 2048)
        assert sc[0] == bc[b] and su[0] == bu[b]
        np.testing.assert_array_equal(si[0, :sc[0]], bi[b, :bc[b]])
        np.testing.assert_array_equal(sv[0, :sc[0]], bv[b, :bc[b]])


def test_host_entry_matches_device_entry(gpu):
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 18, 1024, 2048
    plan = Plan(N, K, N // M, "iter", "mixed", max_signals=3)
    xs, _, _ = siggen.batch_exact(N, K, range(3), mag=(1, 10), dtype=np.complex64)
    di, dv, dc, du, do = _run_gpu(gpu, plan, xs, 2 * K)
    h = plan.exact_host(xs, 2 * K)
    np.testing.assert_array_equal(h.count, dc)
    np.testing.assert_array_equal(h.unresolved, du)
    for b in range(3):
        np.testing.assert_array_equal(h.idx[b, :dc[b]], di[b, :dc[b]])
        np.testing.assert_array_equal(h.val[b, :dc[b]], dv[b, :dc[b]])


def test_host_entry_page_locked_in_place(gpu):
    """Page-locked inputs and results: the kernels read the samples and write
    the results in place in host memory; identical to the device entry."""
    import torch
    from paper_1407_8315_gb300 import Plan, sft
    N, K, M = 1 << 18, 1024, 2048
    plan = Plan(N, K, N // M, "iter", "mixed", max_signals=3)
    xs, _, _ = siggen.batch_exact(N, K, range(3), mag=(1, 10), dtype=np.complex64)
    di, dv, dc, du, do = _run_gpu(gpu, plan, xs, 2 * K)
    px = torch.empty((3, N), dtype=torch.complex64, pin_memory=True)
    px.numpy()[:] = xs
    cap = 2 * K
    out = sft.Result(torch.empty((3, cap), dtype=torch.int64, pin_memory=True).numpy(),
                     torch.empty((3, cap), dtype=torch.complex128, pin_memory=True).numpy(),
                     torch.empty(3, dtype=torch.int64, pin_memory=True).numpy(),
                     torch.empty(3, dtype=torch.int32, pin_memory=True).numpy(),
                     torch.empty(3, dtype=torch.int32, pin_memory=True).numpy())
    for S in (1, 3):
        plan.set_sub_batches(S)  # one sub-batch per signal in the second pass
        h = plan.exact_host(px.numpy(), cap, out)
        np.testing.assert_array_equal(h.count, dc)
        np.testing.assert_array_equal(h.unresolved, du)
        for b in range(3):
            np.testing.assert_array_equal(h.idx[b, :dc[b]], di[b, :dc[b]])
            np.testing.assert_array_equal(h.val[b, :dc[b]], dv[b, :dc[b]])


def test_strided_batch(gpu, orc):
    """x_stride > N: signals read from a wider row pitch."""
    from paper_1407_8315_gb300 import Plan
    import torch
    N, K, M = 1 << 14, 300, 1024
    plan = Plan(N, K, N // M, "iter", "fp64", max_signals=2)
    xs = np.stack([siggen.exact_signal(N, K, s, mag=(1, 10))[0] for s in (1, 2)])
    wide = np.zeros((2, N + 96), np.complex128)
    wide[:, :N] = xs
    xt = torch.from_numpy(wide).cuda()[:, :N]
    out = plan.exact(xt, 4 * M)
    torch.cuda.synchronize()
    for b in range(2):
        oi, _, _ = orc.exact(xs[b], M, 4, orc.ITER, **_tol_of(plan), cap=4 * M)
        gi = np.sort(out.idx[b, :int(out.count[b])].cpu().numpy())
        np.testing.assert_array_equal(gi, oi)


def test_plans_of_different_sizes_coexist(gpu, orc):
    """A plan created after a larger one must not shrink the larger plan's
    FFT tile: both run correctly in either order."""
    from paper_1407_8315_gb300 import Plan
    big = Plan(1 << 16, 512, (1 << 16) // 4096, "iter", "mixed", max_signals=1)
    small = Plan(1 << 12, 16, (1 << 12) // 64, "iter", "mixed", max_signals=1)
    xb = siggen.exact_signal(1 << 16, 512, 3, mag=(1, 10), dtype=np.complex64)[0][None, :]
    xs = siggen.exact_signal(1 << 12, 16, 4, mag=(1, 10), dtype=np.complex64)[0][None, :]
    for _ in range(2):
        _compare(orc, big, xb, "iter", 2048, MIXED_VAL_TOL)
        _compare(orc, small, xs, "iter", 256, MIXED_VAL_TOL)


@pytest.mark.parametrize("mode,prec", [("iter", "mixed"), ("fixed", "mixed"), ("iter", "fp64")])
def test_sub_batches_give_identical_results(gpu, mode, prec):
    """A call split into 1..4 sub-batches on forked streams returns bitwise
    the same results (each sub-batch works in its own workspace slice); 70
    signals, so the sub-batches differ in size."""
    import torch
    from paper_1407_8315_gb300 import Plan
    N, K, M, B = 1 << 14, 60, 256, 70
    dt = np.complex128 if prec == "fp64" else np.complex64
    xs, _, _ = siggen.batch_exact(N, K, [9000 + i for i in range(B)], mag=(1, 10), dtype=dt)
    plan = Plan(N, K, N // M, mode, prec, max_signals=B)
    x = torch.from_numpy(xs).cuda()
    ref = None
    for S in (1, 2, 3, 4):
        plan.set_sub_batches(S)
        assert plan.sub_batches(B) == S
        out = plan.exact(x, 2 * K)
        torch.cuda.synchronize()
        got = [t.cpu().numpy() for t in out]
        if ref is None:
            ref = got
        else:
            for j in (2, 3, 4):  # counts, unresolved, overflow
                np.testing.assert_array_equal(ref[j], got[j])
            for b in range(B):  # the written entries (the rest is uninitialised)
                n = int(ref[2][b])
                np.testing.assert_array_equal(ref[0][b, :n], got[0][b, :n])
                np.testing.assert_array_equal(ref[1][b, :n], got[1][b, :n])
    plan.set_sub_batches(0)
    assert plan.sub_batches(B) == 2 and plan.sub_batches(31) == 1
    assert plan.sub_batches(96) == 3 and plan.sub_batches(1000) == 4


def _same_supports_close_values(ref, got, B, rel):
    """Equal counts, flags and supports; values within rel of each signal's
    largest value."""
    for j in (2, 3, 4):
        np.testing.assert_array_equal(ref[j], got[j])
    for b in range(B):
        n = int(ref[2][b])
        o1, o2 = np.argsort(ref[0][b, :n]), np.argsort(got[0][b, :n])
        np.testing.assert_array_equal(ref[0][b, :n][o1], got[0][b, :n][o2])
        if n:
            v1, v2 = ref[1][b, :n][o1], got[1][b, :n][o2]
            assert np.abs(v1 - v2).max() <= rel * np.abs(v1).max()


@pytest.mark.parametrize("mode", ["iter", "fixed"])
@pytest.mark.parametrize("a_max", [3, 4])
def test_quad_decoders_match_the_oracle(gpu, orc, mode, a_max):
    """The four-lane decoders of three and four aliases (a plan option, used
    on calls that run as one sub-batch): supports bit-exact with the oracle
    and values within the mixed bound; against the one-lane decoder the same
    supports and values within float-float rounding.  N = 2^18, K = M = 1024
    (many bins of three and four aliases), 16 signals."""
    import torch
    from paper_1407_8315_gb300 import Plan
    N, K, M, B = 1 << 18, 1024, 1024, 16
    xs, _, _ = siggen.batch_exact(N, K, range(500, 500 + B), mag=(1, 10), dtype=np.complex64)
    plan = Plan(N, K, N // M, mode, "mixed", max_signals=B, a_max=a_max)
    ref = _run_gpu(torch, plan, xs, 2 * K)
    plan.set_quad_decoders(True)
    _compare(orc, plan, xs, mode, cap=2 * K, val_tol=MIXED_VAL_TOL)
    _same_supports_close_values(ref, _run_gpu(torch, plan, xs, 2 * K), B, 1e-9)


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_quad_decoders_with_long_queues_in_one_sub_batch(gpu, orc, mode):
    """128 signals in one sub-batch with the four-lane decoders enabled: the
    queues of the later levels may exceed the four-lane limit (64 bins per
    SM), so one call can use either decoder per level; the results still
    match the oracle and the one-lane call."""
    import torch
    from paper_1407_8315_gb300 import Plan
    N, K, M, B = 1 << 18, 1024, 1024, 128
    xs, _, _ = siggen.batch_exact(N, K, range(900, 900 + B), mag=(1, 10), dtype=np.complex64)
    plan = Plan(N, K, N // M, mode, "mixed", max_signals=B, a_max=4)
    plan.set_sub_batches(1)
    ref = _run_gpu(torch, plan, xs, 2 * K)
    plan.set_quad_decoders(True)
    _compare(orc, plan, xs, mode, cap=2 * K, val_tol=MIXED_VAL_TOL)
    _same_supports_close_values(ref, _run_gpu(torch, plan, xs, 2 * K), B, 1e-9)


@pytest.mark.parametrize("mode,prec", [("iter", "fp64"), ("fixed", "fp64"), ("fixed", "mixed")])
@pytest.mark.parametrize("N,K,M", [(1 << 18, 1024, 1024), (1 << 20, 8192, 4096)])
def test_up_to_eight_aliases_matches_oracle(gpu, orc, mode, prec, N, K, M):
    """a_max = 8 (above four aliases: Berlekamp-Massey locator and the
    candidate search, one warp per bin): at K/M = 1 and 2 the GPU recovers
    exactly the oracle's set (ITER runs 8 levels; FIXED decodes from 16
    syndromes) with values within the precision's tolerance of the signal's
    largest value (a least-squares solve over up to 8 nearby candidates
    amplifies the input's rounding in the small values)."""
    from paper_1407_8315_gb300 import Plan
    dt = np.complex128 if prec == "fp64" else np.complex64
    plan = Plan(N, K, N // M, mode, prec, max_signals=3, a_max=8)
    xs, _, _ = siggen.batch_exact(N, K, [77 + K + i for i in range(3)], mag=(1, 10), dtype=dt)
    if prec == "fp64":
        _compare(orc, plan, xs, mode, cap=8 * M, val_tol=FP64_VAL_TOL, scale_rel=True)
        return
    # complex64 input: the supports must agree; the values of a bin holding
    # five or more nearby aliases are ill-determined (the least-squares
    # problem amplifies the input's 6e-8 rounding), so there both value
    # sets must fit the bin's 16 equations of Eq. (3) equally well, and the
    # values of the other bins must agree to the usual tolerance
    idx, val, cnt, unres, ovf = _run_gpu(gpu, plan, xs, 8 * M)
    tol = _tol_of(plan)
    d = N // M
    for b in range(3):
        oi, ov, ou = orc.exact(xs[b], M, 8, orc.FIXED, cap=8 * M, **tol)
        n = int(cnt[b])
        o = np.argsort(idx[b, :n], kind="stable")
        gi, gv = idx[b, :n][o], val[b, :n][o]
        assert ovf[b] == 0 and unres[b] == ou
        np.testing.assert_array_equal(gi, oi)
        x = xs[b].astype(np.complex128)
        Y = np.stack([d * np.fft.fft(x[(np.arange(M) * d + j) % N]) for j in range(16)])
        bins = gi % M
        counts = np.bincount(bins, minlength=M)
        small = counts[bins] <= 4
        scale = np.abs(ov).max()
        assert np.abs(gv[small] - ov[small]).max() <= MIXED_VAL_TOL * scale
        for k in np.unique(bins[~small]):
            sel = bins == k
            Z = np.exp(2j * np.pi * np.outer(np.arange(16), gi[sel]) / N)
            rg = np.abs(Y[:, k] - Z @ gv[sel]).max()
            ro = np.abs(Y[:, k] - Z @ ov[sel]).max()
            assert rg <= max(2 * ro, tol["res_tol"] * np.abs(Y[:, k]).max()), (b, k, rg, ro)


def test_stage_timeline_shows_every_sub_batch(gpu):
    """With profiling on, a call split into four sub-batches reports every
    launch once in the timeline, on its sub-batch, with ordered times; the
    per-stage sums match the stage names of sft_plan_stage_times."""
    from paper_1407_8315_gb300 import Plan
    N, K, M = 1 << 16, 64, 1 << 10
    plan = Plan(N, K, N // M, "iter", "mixed", max_signals=8)
    plan.set_sub_batches(4)
    xs = np.stack([siggen.exact_signal(N, K, s)[0] for s in range(8)]).astype(np.complex64)
    x = gpu.from_numpy(xs).cuda()
    plan.set_profiling(True)
    plan.exact(x, 4 * M)
    tl = plan.stage_timeline()
    plan.exact(x, 4 * M)
    st = plan.stage_times()
    plan.set_profiling(False)
    assert {s for _, s, _, _ in tl} == {0, 1, 2, 3}
    assert all(0.0 <= t0 <= t1 for _, _, t0, t1 in tl)
    assert min(t0 for _, _, t0, _ in tl) == 0.0
    assert {n for n, _, _, _ in tl} == set(st)
    for name, (ms, launches) in st.items():
        assert sum(1 for n, _, _, _ in tl if n == name) == launches
    # each sub-batch runs its stages in order on its own stream
    for s in range(4):
        mine = [(t0, t1) for _, q, t0, t1 in tl if q == s]
        assert all(a[1] <= b[0] + 1e-3 for a, b in zip(mine, mine[1:]))
