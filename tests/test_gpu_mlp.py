"""The learned support proposal on the GPU, through the C ABI: its features
and forward/backward kernels against the FP64 reference (oracle/mlp.py),
training by the library's own kernels, the judged Algorithm 2 against the
reference's judged Algorithm 2, and what the trained network gains over the
method without it."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import siggen
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


def _shifts(orc, seed, d, a_max, r):
    return np.concatenate([np.arange(2 * a_max), orc.cs_shifts(seed, d, r)]).astype(np.int64)


def test_features_match_the_oracle(gpu, orc):
    torch = gpu
    from paper_1407_8315_gb300 import Mlp, Plan
    N, K, d, seed = 1 << 16, 24, 32, 5
    M = N // d
    plan = Plan(N, K, d, "general", "mixed", max_signals=2, seed=seed)
    net = Mlp(plan)
    xs = np.stack([siggen.noisy_signal(N, K, 70 + i, 20, mag=(1, 10))[0] for i in range(2)])
    feat, rows, n = net.features(plan, torch.from_numpy(xs).cuda(), 4096)
    feat, rows = feat.cpu().numpy(), rows.cpu().numpy()
    sh = _shifts(orc, seed, d, 3, 9)
    for b in range(2):
        _, _, ak = orc.general(xs[b], M, K, a_max=3, seed=seed)
        mine = rows[rows[:, 0] == b]
        assert sorted(mine[:, 1].tolist()) == np.nonzero(ak)[0].tolist()
        np.testing.assert_array_equal(mine[:, 2], ak[mine[:, 1]])
        Y = np.stack([orc.syndrome(xs[b], d, int(s)) for s in sh])
        for j in np.nonzero(rows[:, 0] == b)[0]:
            k = int(rows[j, 1])
            want = omlp.features(Y[:, k], k, sh, N)
            np.testing.assert_allclose(feat[j], want, atol=2e-6)
    assert n == rows.shape[0]


def _random_params(net, rng, scale=1.0):
    P = omlp.init_params(net.n_in, 128, net.n_out, rng)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(size=P[k].shape) * 0.1
    flat = omlp.pack(P, net.n_in, 128, net.n_out).astype(np.float32) * scale
    return flat, omlp.unpack(flat.astype(np.float64), net.n_in, 128, net.n_out)


@pytest.mark.parametrize("rows", [1, 77, 200])
def test_forward_and_gradient_match_the_oracle(gpu, rows):
    """FP16 weights, FP32 accumulation on the GPU against the FP64 network
    with the same FP16-rounded weights: logits to 1e-5, loss to 1e-5 and
    every parameter block's gradient to 1e-3 (normwise, relative)."""
    torch = gpu
    from paper_1407_8315_gb300 import Mlp, Plan
    plan = Plan(1 << 16, 16, 128, "general", "mixed", seed=1)
    net = Mlp(plan, seed=3)
    rng = np.random.default_rng(rows)
    flat, P = _random_params(net, rng)
    net.params = flat
    np.testing.assert_array_equal(net.params, flat)
    F = rng.normal(size=(rows, net.n_in)).astype(np.float32)
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    cls = rng.integers(0, net.n_cls, rows).astype(np.int32)
    sups = [rng.choice(net.n_sup, size=int(rng.integers(0, 4)), replace=False) for _ in range(rows)]
    supb = np.zeros((rows, net.n_sup))
    for i, ts in enumerate(sups):
        supb[i, ts] = 1
    Ft = torch.from_numpy(F).cuda()
    z = net.forward(Ft).cpu().numpy()
    zo, _ = omlp.forward(P, F.astype(np.float64))
    assert np.abs(z - zo).max() <= 1e-5 * max(1.0, np.abs(zo).max())
    from paper_1407_8315_gb300 import sft
    g, loss = net.grad(Ft, torch.from_numpy(cls).cuda(),
                       torch.from_numpy(sft.support_bits(sups, net.n_sup)).cuda())
    lo, go = omlp.loss_and_grad(P, F.astype(np.float64), cls, supb, net.n_sup)
    assert abs(float(loss.item()) - lo) <= 1e-5 * abs(lo)
    G = omlp.unpack(g.cpu().numpy().astype(np.float64), net.n_in, 128, net.n_out)
    for k in go:
        err = np.linalg.norm(G[k] - go[k]) / max(np.linalg.norm(go[k]), 1e-30)
        assert err <= 1e-3, (k, err)


def _single_alias_rows(rng, n, N, M, shifts):
    d = N // M
    F, cls, sups = [], [], []
    for _ in range(n):
        k, t = int(rng.integers(M)), int(rng.integers(d))
        p = rng.uniform(1, 10) * np.exp(2j * np.pi * rng.uniform())
        Y = p * np.exp(2j * np.pi * (((k + t * M) * shifts) % N) / N)
        Y = Y + 0.05 * p * (rng.normal(size=Y.size) + 1j * rng.normal(size=Y.size))
        F.append(omlp.features(Y, k, shifts, N))
        cls.append(1)
        sups.append([t])
    return np.array(F, np.float32), np.array(cls, np.int32), sups


def test_training_on_the_gpu_learns(gpu, orc):
    """The library's own kernels (forward, backward, Adam) train the network
    on single-alias bins: the loss falls and the true t ranks first on
    held-out rows."""
    torch = gpu
    from paper_1407_8315_gb300 import Mlp, Plan, sft
    N, d = 1 << 16, 32
    M = N // d
    plan = Plan(N, 16, d, "general", "mixed", seed=2)
    net = Mlp(plan, seed=9)
    sh = _shifts(orc, 2, d, 3, 9)
    rng = np.random.default_rng(4)
    F, cls, sups = _single_alias_rows(rng, 6000, N, M, sh)
    losses = net.train(torch.from_numpy(F).cuda(), torch.from_numpy(cls).cuda(),
                       torch.from_numpy(sft.support_bits(sups, d)).cuda(), epochs=15, batch=256,
                       seed=1)
    assert losses[-1] < 0.5 * losses[0], losses
    Ft, _, supt = _single_alias_rows(rng, 500, N, M, sh)
    z = net.forward(torch.from_numpy(Ft).cuda()).cpu().numpy()
    acc = np.mean(np.argmax(z[:, :d], 1) == np.array([s[0] for s in supt]))
    assert acc > 0.95, acc


def _noisy_rows(orc, N, K, d, seed_shift, snr, seeds):
    """Oracle-side training rows (features of the bins the oracle votes,
    labels from the planted spectrum)."""
    M = N // d
    sh = _shifts(orc, seed_shift, d, 3, 9)
    F, cls, sups = [], [], []
    for sd in seeds:
        x, s, _, _ = siggen.noisy_signal(N, K, sd, snr, mag=(1, 10))
        _, _, ak = orc.general(x, M, K, a_max=3, seed=seed_shift)
        Y = np.stack([orc.syndrome(x, d, int(v)) for v in sh])
        for k in np.nonzero(ak)[0].tolist():
            ts = [int(v // M) for v in s if v % M == k]
            F.append(omlp.features(Y[:, k], k, sh, N))
            cls.append(min(len(ts), 4))
            sups.append(ts)
    return np.array(F), np.array(cls), sups


def test_judged_general_matches_the_oracle(gpu, orc):
    """Weights trained on the CPU by the FP64 reference, the same weights on
    the GPU: sft_general with the network attached returns the reference's
    judged result on every bin whose proposal and judgement are not within
    rounding of a tie."""
    torch = gpu
    from paper_1407_8315_gb300 import Mlp, Plan
    N, K, d, seed = 1 << 16, 16, 128, 1
    M = N // d
    F, cls, sups = _noisy_rows(orc, N, K, d, seed, 10, range(5000, 5150))
    sup = np.zeros((len(sups), d))
    for i, ts in enumerate(sups):
        sup[i, ts] = 1
    P = omlp.init_params(F.shape[1], 128, d + 5, np.random.default_rng(0))
    P = omlp.train_adam(P, F, cls, sup, d, epochs=12, batch=128, lr=2e-3, seed=1)
    flat = omlp.pack(P, F.shape[1], 128, d + 5).astype(np.float32)
    P32 = omlp.unpack(flat.astype(np.float64), F.shape[1], 128, d + 5)
    plan = Plan(N, K, d, "general", "mixed", max_signals=3, seed=seed)
    net = Mlp(plan)
    net.params = flat
    plan.attach_mlp(net)
    xs = np.stack([siggen.noisy_signal(N, K, 90000 + i, 10, mag=(1, 10))[0] for i in range(3)])
    out = plan.general(torch.from_numpy(xs).cuda(), 4 * K)
    torch.cuda.synchronize()
    gi_all, gv_all, gc = out.idx.cpu().numpy(), out.val.cpu().numpy(), out.count.cpu().numpy()
    taken = checked = 0
    for b in range(3):
        oi, ov, ak, info = omlp.general_mlp(orc, xs[b], M, K, lambda F_, bins: omlp.forward(P32, F_)[0],
                                           seed=seed)
        gi, gv = gi_all[b, :gc[b]], gv_all[b, :gc[b]]
        o = np.argsort(gi)
        gi, gv = gi[o], gv[o]
        for k, inf in info.items():
            near_tie = inf["gap"] < 1e-3 or (
                np.isfinite(inf["rm"]) and abs(inf["rm"] - (1 - omlp.JUDGE_MARGIN) * inf["rp"])
                <= 1e-6 * inf["rp"])
            if near_tie:
                continue
            checked += 1
            taken += inf["take"]
            gsel = gi % M == k
            osel = oi % M == k
            np.testing.assert_array_equal(gi[gsel], oi[osel], err_msg=f"signal {b} bin {k}")
            if osel.any():
                rel = np.abs(gv[gsel] - ov[osel]) / np.abs(ov[osel])
                assert rel.max() < 1e-4, (b, k, rel.max())
    assert checked >= 30 and taken >= 5, (checked, taken)


def _snr(X, idx, val):
    Xo = np.zeros_like(X)
    Xo[idx] = val
    return 10 * np.log10(np.vdot(Xo, Xo).real / np.vdot(X - Xo, X - Xo).real)


def test_trained_network_gains_over_the_plain_method(gpu):
    """Where the paper's method degrades (N/K = 2^12, d = 128, beyond its
    d = N/(32K)), the network trained on the GPU from features the GPU path
    itself computes lifts SNR_out: >= 3 dB at 10 dB input, >= 1 dB at 20 dB
    (held-out signals; the judge keeps the plain solution wherever the
    network's is not better)."""
    torch = gpu
    from paper_1407_8315_gb300 import Mlp, Plan, sft
    N, K, d, seed = 1 << 18, 64, 128, 11
    M = N // d
    B = 100
    plan = Plan(N, K, d, "general", "mixed", max_signals=B, seed=seed)
    net = Mlp(plan, seed=1)

    def gen(seeds, snrs):
        with ThreadPoolExecutor(16) as ex:
            return list(ex.map(lambda a: siggen.noisy_signal(N, K, a[0], a[1], mag=(1, 10))[:2],
                               zip(seeds, snrs)))

    feats, clss, sups = [], [], []
    for chunk in range(12):
        seeds = list(range(5000 + chunk * B, 5000 + (chunk + 1) * B))
        sig = gen(seeds, [[10, 15, 20, 30][i % 4] for i in range(B)])
        x = torch.from_numpy(np.stack([s[0] for s in sig])).cuda()
        f, rows, _ = net.features(plan, x, B * 512)
        rows = rows.cpu().numpy()
        for b, k in zip(rows[:, 0], rows[:, 1]):
            ts = [int(v // M) for v in sig[b][1] if v % M == k]
            clss.append(min(len(ts), 4))
            sups.append(ts)
        feats.append(f)
    F = torch.cat(feats)
    losses = net.train(F, torch.tensor(clss, dtype=torch.int32, device="cuda"),
                       torch.from_numpy(sft.support_bits(sups, d)).cuda(), epochs=25, batch=1024,
                       seed=2)
    assert losses[-1] < losses[0]
    for snr, need in ((10, 3.0), (20, 1.0)):
        sig = gen(list(range(900000, 900008)), [snr] * 8)
        xs = np.stack([s[0] for s in sig])
        x = torch.from_numpy(xs).cuda()
        plan.attach_mlp(None)
        p = plan.general(x, 4 * K)
        plan.attach_mlp(net)
        m = plan.general(x, 4 * K)
        torch.cuda.synchronize()
        gain = []
        for b in range(8):
            X = np.fft.fft(xs[b].astype(np.complex128))
            sp = _snr(X, p.idx[b, :p.count[b]].cpu().numpy(), p.val[b, :p.count[b]].cpu().numpy())
            sm = _snr(X, m.idx[b, :m.count[b]].cpu().numpy(), m.val[b, :m.count[b]].cpu().numpy())
            gain.append(sm - sp)
        assert np.mean(gain) >= need, (snr, gain)
