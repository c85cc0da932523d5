"""Pins of the oracle's generally K-sparse path (Sec. III, Algorithm 2):
the random-shift generator, the Hankel singular values (Eq. (26)), Subspace
Pursuit (Dai and Dai 2009), the noiseless case where Algorithm 2 must return
the planted spectrum, Theorem 5's guarantee on the vote, and the SNR trend of
Tables III-V (SNR_out reaches SNR_in once N/K <= 2^9)."""
import itertools

import numpy as np
import pytest

import siggen


def test_splitmix64_reference_outputs(orc):
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the reference
    implementation's first outputs for seed 1234567."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [orc.splitmix64(1234567, i) for i in range(5)] == want


def test_cs_shifts_distinct_in_range_and_uniform(orc):
    d, r = 32, 9
    counts = np.zeros(d)
    for seed in range(2000):
        n = orc.cs_shifts(seed, d, r)
        assert len(set(n.tolist())) == r and n.min() >= 0 and n.max() < d
        counts[n] += 1
    # each shift is drawn with probability r/d: chi-square over 32 cells
    exp = 2000 * r / d
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 70  # 31 degrees of freedom; P(chi2 > 70) ~ 1e-4
    assert (orc.cs_shifts(5, d, d) >= 0).all()
    with pytest.raises(ValueError):
        orc.cs_shifts(5, 8, 9)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_hankel_singular_values_against_numpy(orc, n):
    r = np.random.default_rng(n)
    for _ in range(30):
        m = r.normal(size=2 * n - 1) + 1j * r.normal(size=2 * n - 1)
        H = np.array([[m[i + j] for j in range(n)] for i in range(n)])
        np.testing.assert_allclose(orc.hankel_svals(m, n), np.linalg.svd(H, compute_uv=False),
                                   rtol=1e-12, atol=1e-13)


def test_hankel_rank_equals_alias_count(orc):
    """Eq. (27): M = sum_j p_j z_j z_j^T, so with c < a_m aliases exactly c
    singular values are non-zero."""
    N, M, am = 1 << 12, 64, 4
    r = np.random.default_rng(2)
    for c in (1, 2, 3):
        t = r.choice(N // M, size=c, replace=False)
        z = np.exp(2j * np.pi * (5 + t * M) / N)
        p = r.uniform(1, 10, c) * np.exp(2j * np.pi * r.uniform(size=c))
        m = np.array([(p * z ** i).sum() for i in range(2 * am - 1)])
        sv = orc.hankel_svals(m, am)
        assert (sv[:c] > 1e-3).all() and (sv[c:] < 1e-10 * sv[0]).all()


def test_subspace_pursuit_exact_sparse(orc):
    """With a well-conditioned Gaussian sensing matrix SP returns the planted
    ks-sparse vector exactly."""
    r = np.random.default_rng(7)
    for trial in range(50):
        rows, cols, ks = 9, 6, 1 + trial % 3
        Phi = r.normal(size=(rows, cols)) + 1j * r.normal(size=(rows, cols))
        b = np.zeros(cols, complex)
        b[r.choice(cols, ks, replace=False)] = r.normal(size=ks) + 1j * r.normal(size=ks) + 2
        got = orc.subspace_pursuit(Phi, Phi @ b, ks)
        np.testing.assert_allclose(got, b, atol=1e-10)


def test_subspace_pursuit_matches_brute_force_best_subset(orc):
    """On small noisy problems SP's support is the least-squares-best ks-subset
    whenever that optimum is clear (its residual beats the runner-up by 2x)."""
    r = np.random.default_rng(11)
    checked = 0
    for trial in range(200):
        rows, cols, ks = 9, 6, 2
        Phi = r.normal(size=(rows, cols)) + 1j * r.normal(size=(rows, cols))
        b = np.zeros(cols, complex)
        b[r.choice(cols, ks, replace=False)] = 3 + r.normal(size=ks)
        y = Phi @ b + 0.05 * (r.normal(size=rows) + 1j * r.normal(size=rows))
        res = []
        for T in itertools.combinations(range(cols), ks):
            A = Phi[:, T]
            xT = np.linalg.lstsq(A, y, rcond=None)[0]
            res.append((np.linalg.norm(y - A @ xT), T))
        res.sort()
        if res[1][0] < 2 * res[0][0]:
            continue
        got = orc.subspace_pursuit(Phi, y, ks)
        assert tuple(np.nonzero(got)[0]) == res[0][1]
        checked += 1
    assert checked > 150


def test_general_noiseless_returns_planted_spectrum(orc):
    """Without noise and with every bin holding <= a_m terms, the K largest
    singular values are exactly the non-zero ones, a_k is each bin's count,
    the candidate pass keeps the true locations and SP the true values."""
    for seed in range(4):
        N, K = 1 << 16, 128
        M = N // 16
        x, s, v = siggen.exact_signal(N, K, seed, mag=(1, 10))
        counts = np.bincount(s % M, minlength=M)
        if counts.max() > 3:
            continue
        idx, val, ak = orc.general(x, M, K, a_max=3, seed=seed)
        np.testing.assert_array_equal(ak, counts)
        np.testing.assert_array_equal(idx, s)
        assert np.abs(val - v).max() < 1e-9 * np.abs(v).max()


def test_theorem5_vote_is_exact(orc):
    """Theorem 5: if every bin holds at most one significant term and
    eps_min > 2 d q_max, the vote finds the number of significant terms of
    every bin.  Spectrum: K unit-or-larger terms in distinct bins plus
    insignificant terms of magnitude <= q_max at every other location."""
    N, M = 1 << 14, 1 << 10
    d = N // M
    r = np.random.default_rng(3)
    K = 200
    bins = r.choice(M, K, replace=False)
    s = bins + M * r.integers(0, d, K)
    eps_min = 1.0
    q_max = eps_min / (2.5 * d)
    X = q_max * r.uniform(0.2, 1.0, N) * np.exp(2j * np.pi * r.uniform(size=N))
    X[s] = r.uniform(eps_min, 5, K) * np.exp(2j * np.pi * r.uniform(size=K))
    x = np.fft.ifft(X)
    _, _, ak = orc.general(x, M, K, a_max=3, seed=9)
    want = np.zeros(M, np.uint8)
    want[bins] = 1
    np.testing.assert_array_equal(ak, want)


def _snr_out(X, idx, val):
    """SNR(x_out) = 10 log10(MSE(x_out) / MSE(x - x_out)) (Eq. (37))."""
    xo = np.zeros(X.size, complex)
    xo[idx] = val
    return 10 * np.log10(np.vdot(xo, xo).real / np.vdot(X - xo, X - xo).real)


@pytest.mark.parametrize("snr", [30, 20, 10])
def test_snr_out_reaches_snr_in_below_n_over_k_2_9(orc, snr):
    """Tables III-V: with d = N/(32K) and a_m = 3 the output SNR equals the
    input SNR whenever N/K <= 2^9 (Sec. III-F).  Checked at N = 2^18,
    K = 2^9 over three seeds (mean within 0.3 dB)."""
    N, K = 1 << 18, 1 << 9
    M = N // (N // (32 * K))
    outs = []
    for seed in range(3):
        x, _, _, _ = siggen.noisy_signal(N, K, 100 + seed, snr, mag=(1, 10))
        X = np.fft.fft(x.astype(np.complex128))
        idx, val, _ = orc.general(x, M, K, a_max=3, seed=seed)
        outs.append(_snr_out(X, idx, val))
    assert abs(np.mean(outs) - snr) < 0.3, outs


def test_snr_out_drops_above_n_over_k_2_9(orc):
    """Tables III-V: at 10 dB the output SNR falls well below the input once
    N/K grows past 2^9 (2^12 here), averaged over seeds."""
    N, K = 1 << 18, 1 << 6
    M = N // (N // (32 * K))
    outs = []
    for seed in range(4):
        x, _, _, _ = siggen.noisy_signal(N, K, 200 + seed, 10, mag=(1, 10))
        X = np.fft.fft(x.astype(np.complex128))
        idx, val, _ = orc.general(x, M, K, a_max=3, seed=seed)
        outs.append(_snr_out(X, idx, val))
    assert np.mean(outs) < 8.5, outs


# ---------------------------------------------- the CS model without pruning
def test_unpruned_matches_per_bin_subspace_pursuit(orc):
    """Sec. III-B without pruning, rebuilt independently in numpy: per bin k
    the sensing matrix Phi[j][t] = omega^{(k + tM) n_j} (Eq. (18)) over all d
    candidates, y_j = d * FFT_M(x[n d + n_j])[k], Subspace Pursuit at
    sparsity a_m, every non-zero coefficient placed at k + tM."""
    N, M, am = 1 << 10, 32, 2
    d, r = N // M, 3 * am
    x, _, _, _ = siggen.noisy_signal(N, 12, 4, 20, mag=(1, 10))
    x = x.astype(np.complex128)
    ns = orc.cs_shifts(9, d, r)
    Y = np.stack([d * np.fft.fft(x[(np.arange(M) * d + n) % N]) for n in ns])
    want = {}
    for k in range(M):
        s = k + np.arange(d) * M
        Phi = np.exp(2j * np.pi * np.outer(ns, s) / N)
        b = orc.subspace_pursuit(Phi, Y[:, k], am)
        for t in np.nonzero(b)[0]:
            want[int(s[t])] = b[t]
    idx, val, ak = orc.general(x, M, 0, a_max=am, seed=9, cap=M * am, prune=False)
    assert (ak == am).all()
    assert sorted(want) == sorted(idx.tolist())
    got = dict(zip(idx.tolist(), val))
    err = max(abs(got[s] - v) / abs(v) for s, v in want.items())
    assert err < 1e-9, err


def test_unpruned_noiseless_recovers_planted_spectrum(orc):
    """Without noise, bins holding at most a_m terms and r = 3 a_m random
    shifts over d = 16 candidates: SP at sparsity a_m fits every bin
    exactly, so the coefficients above rounding are the planted spectrum
    (the other a_m - a selected coefficients are zero up to rounding)."""
    checked = 0
    for seed in range(6):
        N, K, M, am = 1 << 14, 96, 1 << 10, 3
        x, s, v = siggen.exact_signal(N, K, seed, mag=(1, 10))
        if np.bincount(s % M, minlength=M).max() > am:
            continue
        idx, val, _ = orc.general(x, M, K, a_max=am, seed=seed, cap=M * am, prune=False)
        big = np.abs(val) > 1e-8 * np.abs(v).max()
        np.testing.assert_array_equal(idx[big], s)
        assert np.abs(val[big] - v).max() < 1e-9 * np.abs(v).max()
        checked += 1
    assert checked >= 3


def test_unpruned_reaches_snr_in_at_small_n_over_k(orc):
    """Tables III-V: without pruning the output SNR also reaches the input
    SNR at N/K = 2^8 (28.7 dB at 30 dB there): at least 28.5 dB.  Here
    d = 8 candidates per bin, so r = 8 shifts (3 a_m = 9 exceeds d)."""
    N, K = 1 << 16, 1 << 8
    M = 32 * K
    outs = []
    for seed in range(3):
        x, _, _, _ = siggen.noisy_signal(N, K, 300 + seed, 30, mag=(1, 10))
        X = np.fft.fft(x.astype(np.complex128))
        idx, val, _ = orc.general(x, M, K, a_max=3, r=8, seed=seed, cap=3 * M, prune=False)
        outs.append(_snr_out(X, idx, val))
    assert np.mean(outs) > 28.5, outs
