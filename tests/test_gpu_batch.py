"""Heterogeneous batches (sft_batch): signals of uneven N, K and kind in one
graph-captured call.  Every signal's result is compared with the FP64
oracle (Algorithm 1 for the exactly sparse signals, Algorithm 2 for the noisy
ones): supports bit-exact, values within the mixed form's 1e-4.  The batch
must also give exactly the results of transforming each signal on its own
(same kernels, same per-signal arithmetic).  Both hold on the first call
(capture), on a replay with new data, and without the graph."""
import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

MIXED_VAL_TOL = 1e-4


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


def _make(n_signals, seed):
    """The heterogeneous workload's signal kinds and bin counts, with N capped
    at 2^16 (K and M scaled with it) to keep the test short."""
    from paper_1407_8315_gb300 import sft
    specs = siggen.hetero_batch_spec(n_signals, seed)
    params, xs = [], []
    for sp in specs:
        scale = max(1, sp["N"] >> 16)
        N, K = sp["N"] // scale, max(1, sp["K"] // scale)
        M = max(32, sp["M"] // scale)
        if sp["kind"] == "exact":
            p = sft.sft_params_default(N, K, N // M, "iter", "mixed")
            x = siggen.exact_signal(N, K, sp["seed"], mag=(1, 10), dtype=np.complex64)[0]
        else:
            p = sft.sft_params_default(N, K, N // M, "general", "mixed")
            p.seed = 77
            x = siggen.noisy_signal(N, K, sp["seed"], 30, mag=(1, 10))[0]
        params.append(p)
        xs.append(x)
    return params, xs


def _single(torch, p, x, cap):
    from paper_1407_8315_gb300 import sft
    h = sft.sft_plan_create(p, 1)
    try:
        xt = torch.from_numpy(x).cuda()[None, :]
        fn = sft.sft_general if p.mode == sft.SFT_GENERAL else sft.sft_exact
        out = fn(h, xt, cap)
        torch.cuda.synchronize()
        return [t.cpu().numpy()[0] for t in out]
    finally:
        sft.sft_plan_destroy(h)


def _outs(torch, n, cap):
    from paper_1407_8315_gb300 import sft
    return [sft.Result(torch.empty(cap, dtype=torch.int64, device="cuda"),
                       torch.empty(cap, dtype=torch.complex128, device="cuda"),
                       torch.empty(1, dtype=torch.int64, device="cuda"),
                       torch.empty(1, dtype=torch.int32, device="cuda"),
                       torch.empty(1, dtype=torch.int32, device="cuda")) for _ in range(n)]


def _check(torch, params, xs, outs, cap, exact_bitwise=True):
    """The batch against one plan call per signal: counts, flags and
    supports equal; values equal bit for bit for the exactly sparse signals
    (the persistent kernel repeats the launch sequence's arithmetic), and to
    1e-12 for the others (the autotuner may pick another FFT radix for a
    shape class, which changes the last bits)."""
    from paper_1407_8315_gb300 import sft
    for i, (p, x) in enumerate(zip(params, xs)):
        ri, rv, rc, ru, ro = _single(torch, p, x, cap)
        o = outs[i]
        n = int(o.count.item())
        assert n == int(rc), i
        assert int(o.unresolved.item()) == int(ru) and int(o.overflow.item()) == int(ro)
        np.testing.assert_array_equal(o.idx[:n].cpu().numpy(), ri[:n])
        if exact_bitwise and p.mode == sft.SFT_EXACT_ITER:
            np.testing.assert_array_equal(o.val[:n].cpu().numpy(), rv[:n])
        elif n:
            np.testing.assert_allclose(o.val[:n].cpu().numpy(), rv[:n], rtol=1e-12, atol=0)


def _check_oracle(orc, params, xs, outs):
    """Each signal of the batch against the FP64 oracle of its own kind."""
    from paper_1407_8315_gb300 import sft
    worst = 0.0
    for i, (p, x) in enumerate(zip(params, xs)):
        o = outs[i]
        M = p.N // p.d
        cap = o.idx.shape[0]
        if p.mode == sft.SFT_GENERAL:
            oi, ov, _ = orc.general(x, M, p.K, a_max=p.a_max, r=p.n_cs_shifts, seed=p.seed,
                                    cap=cap)
            ou = 0
        else:
            om = orc.ITER if p.mode == sft.SFT_EXACT_ITER else orc.FIXED
            oi, ov, ou = orc.exact(x, M, p.a_max, om, max_iters=p.max_iters, cap=cap,
                                   zero_tol=p.zero_tol, root_tol=p.root_tol, res_tol=p.res_tol)
        n = int(o.count.item())
        gi, gv = o.idx[:n].cpu().numpy(), o.val[:n].cpu().numpy()
        order = np.argsort(gi, kind="stable")
        gi, gv = gi[order], gv[order]
        assert int(o.overflow.item()) == 0, i
        np.testing.assert_array_equal(gi, oi, err_msg=f"signal {i}: supports differ")
        assert int(o.unresolved.item()) == ou, (i, int(o.unresolved.item()), ou)
        if n:
            worst = max(worst, float((np.abs(gv - ov) / np.abs(ov)).max()))
    assert worst <= MIXED_VAL_TOL, worst
    return worst


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_oracle_and_single_signal_calls(gpu, orc, use_graph):
    torch = gpu
    from paper_1407_8315_gb300 import sft
    cap = 2048
    params, xs = _make(24, 5)
    batch = sft.Batch(use_graph=use_graph, autotune=True)
    xt = [torch.from_numpy(x).cuda() for x in xs]
    outs = _outs(torch, len(xs), cap)
    batch.run(params, xt, outs)
    torch.cuda.synchronize()
    info = batch.info()
    n_exact = sum(p.mode == sft.SFT_EXACT_ITER for p in params)
    assert info["groups"] >= 4 and info["tuned"] >= 1
    # every exactly sparse signal of this batch fits the persistent kernel
    pinfo = batch.persistent_info()
    assert pinfo["signals"] == n_exact and pinfo["ctas"] >= 1
    if use_graph:
        assert info["graph_nodes"] > info["groups"]
    _check_oracle(orc, params, xs, outs)
    _check(torch, params, xs, outs, cap)
    # same composition, new data: the graph is replayed with fresh tables
    params2, xs2 = _make(24, 5)
    rng = np.random.default_rng(1)
    xs2 = [(x * np.complex64(np.exp(1j * rng.uniform(0, 6.28)))).astype(np.complex64) for x in xs2]
    for t, x in zip(xt, xs2):
        t.copy_(torch.from_numpy(x))
    outs2 = _outs(torch, len(xs), cap)
    batch.run(params2, xt, outs2)
    torch.cuda.synchronize()
    assert batch.info()["graph_nodes"] == info["graph_nodes"]
    _check_oracle(orc, params2, xs2, outs2)
    _check(torch, params2, xs2, outs2, cap)
    batch.close()


@pytest.mark.parametrize("ctas", [1, 3, 0])
def test_persistent_kernel_at_any_cta_count(gpu, orc, ctas):
    """The persistent kernel drains its queue with any number of CTAs (one
    CTA takes every signal in turn; three share them; 0 lets the autotuner
    choose), and gives the same results as the batch without it."""
    torch = gpu
    from paper_1407_8315_gb300 import sft
    cap = 2048
    params, xs = _make(16, 8)
    xt = [torch.from_numpy(x).cuda() for x in xs]
    ref = _outs(torch, len(xs), cap)
    b0 = sft.Batch(persistent=False)
    b0.run(params, xt, ref)
    got = _outs(torch, len(xs), cap)
    b1 = sft.Batch(persistent=True, persistent_ctas=ctas)
    b1.run(params, xt, got)
    b1.run(params, xt, got)  # replay
    torch.cuda.synchronize()
    assert b0.persistent_info()["signals"] == 0
    info = b1.persistent_info()
    assert info["signals"] == sum(p.mode == sft.SFT_EXACT_ITER for p in params)
    if ctas:
        assert info["ctas"] == min(ctas, info["signals"])
    for i, p in enumerate(params):
        n = int(ref[i].count.item())
        assert int(got[i].count.item()) == n
        assert int(got[i].unresolved.item()) == int(ref[i].unresolved.item())
        np.testing.assert_array_equal(got[i].idx[:n].cpu().numpy(), ref[i].idx[:n].cpu().numpy())
    _check_oracle(orc, params, xs, got)
    b0.close()
    b1.close()


def test_batch_rejects_bad_signal(gpu):
    torch = gpu
    from paper_1407_8315_gb300 import sft
    params, xs = _make(4, 9)
    params[2].a_max = 9
    batch = sft.Batch()
    xt = [torch.from_numpy(x).cuda() for x in xs]
    with pytest.raises(sft.SftError) as ei:
        batch.run(params, xt, _outs(torch, 4, 2048))
    assert "signal 2" in str(ei.value)
    batch.close()
