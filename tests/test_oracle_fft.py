"""Pins of the oracle's FFT and syndromes (Eq. (1)-(2)) against what the
mathematics fixes: the DFT's definition, closed forms of single tones, the
alias-sum identity of Eq. (2) computed straight from a planted spectrum, and
the fold identity used between levels of Algorithm 1."""
import numpy as np
import pytest

import siggen


def _rand(n, seed):
    r = np.random.default_rng(seed)
    return r.normal(size=n) + 1j * r.normal(size=n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024])
def test_fft_matches_brute_dft(orc, n):
    a = _rand(n, n)
    ref = orc.dft_brute(a)
    got = orc.fft(a)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    # library FFT as a second, independent reference
    assert np.abs(got - np.fft.fft(a)).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_fft_inverse_roundtrip(orc):
    a = _rand(512, 3)
    back = orc.fft(orc.fft(a, -1), +1) / 512
    assert np.abs(back - a).max() < 1e-13


def test_brute_dft_closed_forms(orc):
    n = 32
    for s0 in (0, 1, 7, 31):
        tone = np.exp(2j * np.pi * s0 * np.arange(n) / n)
        X = orc.dft_brute(tone)
        want = np.zeros(n, complex)
        want[s0] = n
        assert np.abs(X - want).max() < 1e-12
    delta = np.zeros(n, complex)
    delta[0] = 1
    assert np.abs(orc.dft_brute(delta) - 1).max() < 1e-15


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.fft(np.ones(12))


def _alias_sum(N, supp, vals, d, l):
    """Right-hand side of Eq. (2), X the unnormalised DFT and x its inverse
    with 1/N: sum over the aliases of bin k of
    X[k + jM] * omega^{(k + jM) l}, written straight from the planted X."""
    M = N // d
    Y = np.zeros(M, complex)
    for s, v in zip(supp, vals):
        Y[s % M] += v * np.exp(2j * np.pi * ((s * l) % N) / N)
    return Y


@pytest.mark.parametrize("N,K,d", [(64, 5, 4), (1024, 40, 16), (4096, 100, 64), (1 << 14, 300, 8)])
def test_syndrome_is_alias_sum(orc, N, K, d):
    x, supp, vals = siggen.exact_signal(N, K, seed=N + K, mag=(1, 10))
    for l in (0, 1, 2, 3, 5, d - 1, d, d + 3):
        Y = orc.syndrome(x, d, l)
        want = _alias_sum(N, supp, vals, d, l)
        assert np.abs(Y - want).max() < 1e-9 * np.abs(vals).max(), (d, l)


def test_syndrome_d1_is_plain_dft(orc):
    x = _rand(256, 9)
    assert np.abs(orc.syndrome(x, 1, 0) - np.fft.fft(x)).max() < 1e-11


def test_fold_identity(orc):
    """Y_{2d,l}[k] = Y_{d,l}[k] + Y_{d,l}[k + M/2]: the identity that lets
    Algorithm 1 keep earlier shifts when d doubles."""
    N = 1 << 12
    x, _, _ = siggen.exact_signal(N, 60, seed=1, mag=(1, 10))
    for d in (4, 16, 64):
        M = N // d
        for l in (0, 1, 5):
            Yd = orc.syndrome(x, d, l)
            Y2d = orc.syndrome(x, 2 * d, l)
            assert np.abs(Y2d - (Yd[: M // 2] + Yd[M // 2:])).max() < 1e-10


def test_syndrome_single_alias_ratio(orc):
    """a = 1 (Sec. II-A): m_1 / m_0 = e^{i 2 pi s0 / N} and |m_0| = |m_1|."""
    N, d = 1 << 10, 32
    s0, v = 517, 2.5 - 1.0j
    x = siggen.tone_signal(N, [s0], [v])
    m0 = orc.syndrome(x, d, 0)[s0 % (N // d)]
    m1 = orc.syndrome(x, d, 1)[s0 % (N // d)]
    assert abs(m0 - v) < 1e-12
    assert abs(m1 / m0 - np.exp(2j * np.pi * s0 / N)) < 1e-13
