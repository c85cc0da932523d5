"""GPU parity of the generally K-sparse transform (Algorithm 2) against the
FP64 oracle, through the C ABI: the random shifts, the votes (supports) and
the Subspace Pursuit values."""
import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

MIXED_VAL_TOL = 1e-4
FP64_VAL_TOL = 1e-10


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


def _run(torch, plan, xs, cap):
    x = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    out = plan.general(x, cap)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _compare(orc, plan, xs, seed, val_tol, a_max=3):
    import torch
    cap = 2 * plan.K + 16
    idx, val, cnt, unres, ovf = _run(torch, plan, xs, cap)
    worst = 0.0
    for b in range(xs.shape[0]):
        oi, ov, _ = orc.general(xs[b], plan.M, plan.K, a_max=a_max, seed=seed, cap=cap)
        n = int(cnt[b])
        gi, gv = idx[b, :n], val[b, :n]
        o = np.argsort(gi, kind="stable")
        gi, gv = gi[o], gv[o]
        assert ovf[b] == 0 and unres[b] == 0
        np.testing.assert_array_equal(gi, oi, err_msg=f"signal {b}: supports differ")
        if n:
            worst = max(worst, float((np.abs(gv - ov) / np.abs(ov)).max()))
    assert worst <= val_tol, worst
    return worst


def test_cs_shifts_match_the_oracle(gpu, orc):
    from paper_1407_8315_gb300 import Plan
    for seed in (0, 1, 12345, 2**63 + 7):
        plan = Plan(1 << 20, 1024, 32, "general", "mixed", seed=seed)
        np.testing.assert_array_equal(plan.cs_shifts, orc.cs_shifts(seed, 32, 9))


@pytest.mark.parametrize("snr", [20, 30, 40])
def test_noisy_full_size(gpu, orc, snr):
    """N = 2^20 complex64, K = 1024, |X| ~ U[1,10], white noise at 20/30/40 dB;
    the paper's setting d = N/(32K) = 32 (M = 2^15, four-step FFT), a_m = 3,
    r = 9.  Three signals per batch."""
    from paper_1407_8315_gb300 import Plan
    N, K = 1 << 20, 1024
    d = N // (32 * K)
    plan = Plan(N, K, d, "general", "mixed", max_signals=3, seed=snr)
    xs = np.stack([siggen.noisy_signal(N, K, 300 + 10 * snr + i, snr, mag=(1, 10))[0]
                   for i in range(3)])
    _compare(orc, plan, xs, snr, MIXED_VAL_TOL)


def test_noiseless_equals_planted(gpu, orc):
    from paper_1407_8315_gb300 import Plan
    N, K = 1 << 16, 128
    M = N // 16
    plan = Plan(N, K, 16, "general", "fp64", max_signals=2, seed=3)
    xs = np.stack([siggen.exact_signal(N, K, s, mag=(1, 10))[0] for s in (0, 5)])
    _compare(orc, plan, xs, 3, FP64_VAL_TOL)
    idx, val, cnt, _, _ = _run(gpu, plan, xs, 2 * K)
    for b, s in enumerate((0, 5)):
        _, supp, vals = siggen.exact_signal(N, K, s, mag=(1, 10))
        if np.bincount(supp % M).max() <= 3:
            np.testing.assert_array_equal(np.sort(idx[b, :cnt[b]]), supp)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("N,K,d,a_max", [(1 << 14, 64, 8, 2), (1 << 16, 300, 16, 2),
                                         (1 << 17, 700, 16, 4), (1 << 18, 1 << 9, 16, 3)])
def test_sizes(gpu, orc, prec, N, K, d, a_max):
    from paper_1407_8315_gb300 import Plan
    dt = np.complex128 if prec == "fp64" else np.complex64
    plan = Plan(N, K, d, "general", prec, max_signals=2, seed=N + K, a_max=a_max)
    xs = np.stack([siggen.noisy_signal(N, K, 7 * N + i, 25, mag=(1, 10), dtype=dt)[0]
                   for i in range(2)])
    _compare(orc, plan, xs, N + K, FP64_VAL_TOL if prec == "fp64" else MIXED_VAL_TOL,
             a_max=a_max)


def test_exact_entry_rejects_general_plan(gpu):
    from paper_1407_8315_gb300 import Plan, SftError
    import torch
    plan = Plan(1 << 14, 64, 16, "general", "mixed")
    x = torch.zeros((1, 1 << 14), dtype=torch.complex64, device="cuda")
    with pytest.raises(SftError):
        plan.exact(x, 64)


@pytest.mark.parametrize("N,K,d,a_max,prec,snr", [
    (1 << 14, 32, 16, 3, "mixed", 20),
    (1 << 16, 16, 128, 3, "fp64", 30),
    (1 << 16, 64, 64, 4, "mixed", 30),
    (1 << 18, 8, 2048, 3, "mixed", 10),
    (1 << 20, 1024, 32, 3, "mixed", 30),
])
def test_unpruned_matches_oracle(gpu, orc, N, K, d, a_max, prec, snr):
    """The CS model without pruning (Sec. III-B): every bin by Subspace
    Pursuit at sparsity a_m over all d candidates, against the oracle's
    prune=False path -- identical supports (every non-zero coefficient of
    every bin), values within the precision's tolerance.  d from 16 to 2048
    (the shared-memory root table), M = 2^15 runs the four-step FFT."""
    from paper_1407_8315_gb300 import Plan
    M = N // d
    plan = Plan(N, K, d, "general-unpruned", prec, max_signals=2, a_max=a_max, seed=snr + d)
    dt = np.complex128 if prec == "fp64" else np.complex64
    xs = np.stack([siggen.noisy_signal(N, K, 500 + d + i, snr, mag=(1, 10), dtype=dt)[0]
                   for i in range(2)])
    cap = M * a_max
    idx, val, cnt, unres, ovf = _run(gpu, plan, xs, cap)
    tol = FP64_VAL_TOL if prec == "fp64" else MIXED_VAL_TOL
    for b in range(2):
        oi, ov, _ = orc.general(xs[b], M, K, a_max=a_max, seed=snr + d, cap=cap, prune=False)
        n = int(cnt[b])
        o = np.argsort(idx[b, :n], kind="stable")
        gi, gv = idx[b, :n][o], val[b, :n][o]
        assert ovf[b] == 0 and unres[b] == 0
        np.testing.assert_array_equal(gi, oi, err_msg=f"signal {b}: supports differ")
        scale = np.abs(ov).max()
        assert np.abs(gv - ov).max() <= tol * scale


def test_unpruned_overflow_keeps_cap_entries(gpu):
    """A result capacity below a_m N/d sets the overflow flag and fills the
    capacity."""
    from paper_1407_8315_gb300 import Plan
    N, K, d = 1 << 14, 32, 16
    plan = Plan(N, K, d, "general-unpruned", "mixed", seed=1)
    x = siggen.noisy_signal(N, K, 7, 20, mag=(1, 10))[0][None, :]
    idx, val, cnt, unres, ovf = _run(gpu, plan, x, 64)
    assert int(ovf[0]) == 1 and int(cnt[0]) == 64


@pytest.mark.parametrize("mode", ["general", "general-unpruned"])
def test_sub_batches_give_identical_results(gpu, mode):
    """The general paths split into 1..4 sub-batches return bitwise the same
    results as one launch sequence."""
    from paper_1407_8315_gb300 import Plan
    N, K, d, B = 1 << 14, 16, 32, 37
    xs = np.stack([siggen.noisy_signal(N, K, 700 + i, 25, mag=(1, 10))[0] for i in range(B)])
    plan = Plan(N, K, d, mode, "mixed", max_signals=B, seed=4)
    cap = 3 * (N // d)
    ref = None
    for S in (1, 2, 3, 4):
        plan.set_sub_batches(S)
        got = _run(gpu, plan, xs, cap)
        if ref is None:
            ref = got
        else:
            for j in (2, 3, 4):  # counts, unresolved, overflow
                np.testing.assert_array_equal(ref[j], got[j])
            for b in range(B):  # the written entries (the rest is uninitialised)
                n = int(ref[2][b])
                np.testing.assert_array_equal(ref[0][b, :n], got[0][b, :n])
                np.testing.assert_array_equal(ref[1][b, :n], got[1][b, :n])
