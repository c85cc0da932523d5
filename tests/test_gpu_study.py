"""GPU parity of the collision-count study (Sec. II-C, Fig. 2) against the
oracle: the histogram of per-bin alias counts, bit-exact, including the
edge cases (no sets, one bin, counts past the last cell)."""
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


@pytest.mark.parametrize("N,K,M,sets,cells", [
    (1 << 12, 256, 256, 300, 9),
    (1 << 20, 4096, 1 << 15, 40, 9),
    (1 << 16, 1 << 14, 1 << 10, 20, 33),   # 16 per bin on average: clipped cells
    (1 << 10, 37, 1, 5, 9),                # one bin holds every location
])
def test_alias_histogram_matches_oracle(gpu, orc, N, K, M, sets, cells):
    from paper_1407_8315_gb300 import sft
    rng = np.random.default_rng(N + K)
    S = np.stack([siggen.sparse_support(N, K, rng) for _ in range(sets)])
    h = sft.alias_histogram(gpu.from_numpy(S).cuda(), M, cells)
    gpu.cuda.synchronize()
    np.testing.assert_array_equal(h.cpu().numpy(), orc.alias_histogram(S, M, cells))


def test_alias_histogram_edges(gpu):
    from paper_1407_8315_gb300 import sft
    empty = gpu.zeros((0, 8), dtype=gpu.int64, device="cuda")
    assert sft.alias_histogram(empty, 64, 5).cpu().tolist() == [0] * 5
    no_locations = gpu.zeros((3, 0), dtype=gpu.int64, device="cuda")
    assert sft.alias_histogram(no_locations, 64, 5).cpu().tolist() == [3 * 64, 0, 0, 0, 0]
    big = gpu.zeros((1, 8), dtype=gpu.int64, device="cuda")
    with pytest.raises(sft.SftError):
        sft.alias_histogram(big, 1 << 16, 5)
    with pytest.raises(sft.SftError):
        sft.alias_histogram(big, 48, 5)
