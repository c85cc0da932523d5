"""The device arithmetic the FP64 decoders build on, against correctly
rounded references computed on the host (numpy): the bit-move seeded
Newton reciprocal within one ulp of 1/x, the bit-move float-to-double
widening exact, the complex square root within a few ulps of the
principal root."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_8315_gb300 as pkg
    pkg.build()
    return torch


def _run(torch, x, which, n):
    from paper_1407_8315_gb300 import sft
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    od = torch.empty_like(xd)
    sft.sft_device_math_check(xd.data_ptr(), n, od.data_ptr(), which,
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return od.cpu().numpy()


def _ulps(a, b):
    """|a - b| in units in the last place of b."""
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_reciprocal_within_one_ulp(gpu):
    rng = np.random.default_rng(7)
    x = rng.uniform(1.0, 2.0, 200000) * np.exp2(rng.integers(-140, 140, 200000))
    x *= np.where(rng.random(200000) < 0.5, -1.0, 1.0)
    # the seed's range edges, powers of two, and the division fallback
    edges = np.array([2.0 ** -123, 2.0 ** -123 * 1.5, 2.0 ** 124 * 0.999, 2.0 ** 124, 2.0 ** 200,
                      2.0 ** -300, 1.0, -1.0, 3.0, 1.0 / 3.0, np.nextafter(1.0, 2.0)])
    x = np.concatenate([x, edges, -edges])
    r = _run(gpu, x, 0, x.size)
    ref = 1.0 / x
    assert _ulps(r, ref).max() <= 1.0


def test_float_widening_is_exact(gpu):
    rng = np.random.default_rng(8)
    f = (rng.standard_normal(100000) * np.exp2(rng.integers(-140, 120, 100000))).astype(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -1e-45, 1.17549435e-38, 3.4028235e38],
                       dtype=np.float32)
    f = np.concatenate([f, special])
    out = _run(gpu, f.astype(np.float64), 1, f.size)
    np.testing.assert_array_equal(out, f.astype(np.float64))
    assert np.array_equal(np.signbit(out), np.signbit(f))
    nan = _run(gpu, np.array([np.nan]), 1, 1)
    assert np.isnan(nan[0])


def test_complex_square_root_is_the_principal_root(gpu):
    rng = np.random.default_rng(9)
    n = 100000
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.exp2(rng.integers(-60, 60, n))
    # (the magnitudes the decoders see: |z|^2 a normal double)
    z = np.concatenate([z, [4.0 + 0j, -4.0 + 0j, 1j, -1j, 0j, -3.0 + 1e-9j, -3.0 - 1e-9j]])
    pairs = np.stack([z.real, z.imag], axis=1).ravel()
    out = _run(gpu, pairs, 2, z.size).reshape(-1, 2)
    got = out[:, 0] + 1j * out[:, 1]
    ref = np.sqrt(z)
    scale = np.maximum(np.abs(ref), 1e-300)
    assert (np.abs(got - ref) / scale).max() <= 4 * np.finfo(np.float64).eps
    assert (got.real >= 0).all()
