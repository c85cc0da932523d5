"""Unknown K (Sec. II-E) on the GPU, through sft_exact_auto: every signal of
a batch with very different K stops at the same M as the oracle's
bottom-up loop, with the oracle's support bit-exactly."""
import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


@pytest.mark.parametrize("mode", ["iter", "fixed"])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_auto_matches_the_oracle(gpu, orc, mode, prec):
    torch = gpu
    from paper_1407_8315_gb300 import sft
    N = 1 << 16
    Ks = [3, 40, 300, 1000, 17, 0]
    dt = np.complex64 if prec == "mixed" else np.complex128
    xs = np.stack([siggen.exact_signal(N, K, 100 + i, mag=(1, 10), dtype=dt)[0] if K else
                   np.zeros(N, dt) for i, K in enumerate(Ks)])
    p = sft.sft_params_default(N, 1, 1, mode, prec)
    out, m = sft.sft_exact_auto(p, torch.from_numpy(xs).cuda(), 4096)
    torch.cuda.synchronize()
    idx, val, cnt = out.idx.cpu().numpy(), out.val.cpu().numpy(), out.count.cpu().numpy()
    un = out.unresolved.cpu().numpy()
    tol = 1e-4 if prec == "mixed" else 1e-10
    om = orc.ITER if mode == "iter" else orc.FIXED
    for b, K in enumerate(Ks):
        oi, ov, ou, oM = orc.exact_auto(xs[b], 4, om)
        assert m[b] == oM and un[b] == ou, (b, K, m[b], oM)
        gi, gv = idx[b, :cnt[b]], val[b, :cnt[b]]
        o = np.argsort(gi, kind="stable")
        np.testing.assert_array_equal(gi[o], oi)
        if K:
            assert len(oi) == K
            assert (np.abs(gv[o] - ov) / np.abs(ov)).max() <= tol


def test_auto_rejects_bad_arguments(gpu):
    torch = gpu
    from paper_1407_8315_gb300 import sft
    x = torch.zeros((1, 1 << 12), dtype=torch.complex64, device="cuda")
    p = sft.sft_params_default(1 << 12, 1, 1, "general", "mixed")
    with pytest.raises(sft.SftError):
        sft.sft_exact_auto(p, x, 64)
    p = sft.sft_params_default(1 << 12, 1, 1, "iter", "mixed")
    with pytest.raises(sft.SftError):
        sft.sft_exact_auto(p, x, 64, M_start=3)
    with pytest.raises(sft.SftError):
        sft.sft_exact_auto(p, x, 64, M_start=64, M_max=32)
