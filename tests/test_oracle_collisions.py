"""Pins of the collision-count study (Sec. II-C: Lemma 2, Fig. 2): the
oracle's histogram of per-bin alias counts against the hypergeometric law,
exhaustively on a tiny case and statistically on sampled supports, and
Lemma 2's bound on the probability that some bin exceeds a_m."""
import itertools
from math import comb

import numpy as np

import siggen


def test_exhaustive_histogram_is_hypergeometric(orc):
    """Over all C(N, K) support sets the count of bins holding exactly a
    locations is C(N, K) * M * C(d, a) C(N - d, K - a) / C(N, K) -- integers,
    compared exactly."""
    N, K, M = 12, 4, 4
    d = N // M
    sets = np.array(list(itertools.combinations(range(N), K)), dtype=np.int64)
    hist = orc.alias_histogram(sets, M, n_cells=K + 2)
    want = [M * comb(d, a) * comb(N - d, K - a) if a <= K else 0 for a in range(K + 2)]
    assert hist.tolist() == want
    assert hist.sum() == comb(N, K) * M


def test_sampled_histogram_matches_the_law(orc):
    """2000 sampled sets at N = 2^12, K = 256, M = 256 (N+ = M/K = 1): cell
    frequencies within a chi-square bound of the hypergeometric law."""
    N, K, M, sets = 1 << 12, 256, 256, 2000
    rng = np.random.default_rng(5)
    S = np.stack([siggen.sparse_support(N, K, rng) for _ in range(sets)])
    hist = orc.alias_histogram(S, M, n_cells=6)
    p = [orc.alias_count_pmf(N, K, M, a) for a in range(5)]
    p.append(1.0 - sum(p))
    exp = np.array(p) * sets * M
    keep = exp > 20
    chi2 = (((hist - exp) ** 2 / exp)[keep]).sum()
    assert chi2 < 25, (hist, exp)  # <= 5 degrees of freedom; P(chi2 > 25) ~ 1e-4


def test_lemma2_bound_holds(orc):
    """Lemma 2: Pr(some bin holds more than a_m) <= (N/d) (d e K / (N (a_m + 1)))^(a_m + 1).
    At N = 2^14, M = 2^10, K = 64 and a_m = 2 the bound is 0.076; the
    sampled frequency over 3000 sets stays below it."""
    N, M, K, am = 1 << 14, 1 << 10, 64, 2
    d = N // M
    bound = (N / d) * (d * np.e * K / (N * (am + 1))) ** (am + 1)
    rng = np.random.default_rng(9)
    bad = 0
    for _ in range(3000):
        s = siggen.sparse_support(N, K, rng)
        if np.bincount(s % M, minlength=M).max() > am:
            bad += 1
    assert bad / 3000 <= bound, (bad, bound)
    assert orc.alias_histogram(np.arange(0, 64, dtype=np.int64)[None, :] * M, M, 4)[-1] == 1
