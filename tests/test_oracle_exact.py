"""Pins of the whole exactly-K-sparse oracle (Algorithm 1 and the
non-iterative variant of Fig. 1(b)).

* The worked example of Fig. 1 (fixture under tests/golden/).
* A support-only simulation of the decision rule: with exact arithmetic a
  bin decodes iff its (residual) alias count equals the a being decoded, so
  the recovered set follows from the planted support alone.  The oracle must
  reproduce it exactly, and the recovered values must equal the planted ones.
* Lemma 2 (failure probability of the non-iterative method) and Theorem 2
  (at most tau*K bins fail) as statistical bounds.
"""
import os
from collections import Counter

import numpy as np
import pytest

import siggen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_fixture(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


def test_fig1_worked_example(orc):
    g = _read_fixture("fig1_worked_example.txt")
    N, d0 = g["N"][0], g["d0"][0]
    supp = g["support"]
    x = siggen.tone_signal(N, supp, [1.0, 2.0j, -3.0 + 0.5j])
    M0 = N // d0
    idx, _, un = orc.exact(x, M0, a_max=2, mode=orc.ITER, max_iters=1)
    assert idx.tolist() == g["iter_level0_solved"]
    assert un == g["iter_level0_unresolved_bins"][0]
    idx, val, un = orc.exact(x, M0, a_max=2, mode=orc.ITER, max_iters=2)
    assert idx.tolist() == g["iter_level1_solved"] and un == 0
    assert np.abs(val - np.array([1.0, 2.0j, -3.0 + 0.5j])).max() < 1e-12
    idx, _, un = orc.exact(x, M0, a_max=1, mode=orc.FIXED)
    assert idx.tolist() == g["fixed_a1_solved"] and un == 1
    idx, _, un = orc.exact(x, M0, a_max=2, mode=orc.FIXED)
    assert idx.tolist() == g["fixed_a2_solved"] and un == 0


def simulate_fixed(supp, M, a_max):
    """Decision rule of the non-iterative method: a bin with c <= a_m aliases
    is solved, one with c > a_m is not (Sec. II-B)."""
    cnt = Counter((supp % M).tolist())
    rec = sorted(int(s) for s in supp if cnt[int(s) % M] <= a_max)
    return rec, sum(1 for c in cnt.values() if c > a_max)


def simulate_iter(supp, M0, iters):
    """Decision rule of Algorithm 1: level l (M = M0 / 2^l bins) solves the
    bins whose residual alias count is exactly l + 1."""
    remaining = set(int(s) for s in supp)
    rec = []
    M = M0
    for l in range(iters):
        if l:
            M //= 2
        groups = {}
        for s in remaining:
            groups.setdefault(s % M, []).append(s)
        for members in groups.values():
            if len(members) == l + 1:
                rec += members
                remaining -= set(members)
    unres = len({s % M for s in remaining})
    return sorted(rec), unres


CASES = [  # (N, K, M0, seeds)
    (1 << 16, 64, 256, range(0, 40)),        # the plain-FP64 configuration
    (1 << 16, 512, 1024, range(0, 20)),      # K / M = 1/2 as at 2^22
    (1 << 18, 2048, 4096, range(0, 6)),
]


@pytest.mark.parametrize("N,K,M0,seeds", CASES)
@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_exact_matches_support_simulation(orc, N, K, M0, seeds, mode):
    for seed in seeds:
        x, supp, vals = siggen.exact_signal(N, K, seed, mag=(1, 10))
        if mode == "iter":
            want, want_unres = simulate_iter(supp, M0, 4)
            idx, val, un = orc.exact(x, M0, 4, orc.ITER)
        else:
            want, want_unres = simulate_fixed(supp, M0, 4)
            idx, val, un = orc.exact(x, M0, 4, orc.FIXED)
        assert idx.tolist() == want, (seed, len(idx), len(want))
        assert un == want_unres, seed
        j = np.searchsorted(supp, idx)
        assert np.abs(val - vals[j]).max() < 1e-8 * np.abs(vals).max(), seed


def test_unit_magnitude_config_recovers_everything(orc):
    """N = 2^16, K = 64, M = 256, |X| = 1: every planted value comes back."""
    x, supp, vals = siggen.exact_signal(1 << 16, 64, 123, mag=(1, 1))
    for mode in (orc.ITER, orc.FIXED):
        idx, val, un = orc.exact(x, 256, 4, mode)
        want = simulate_iter(supp, 256, 4)[0] if mode == orc.ITER else simulate_fixed(supp, 256, 4)[0]
        assert idx.tolist() == want
        j = np.searchsorted(supp, idx)
        assert np.abs(val - vals[j]).max() < 1e-10


def test_lemma2_failure_bound(orc):
    """Lemma 2: Pr(some bin has a > a_m) <= (N/d) (d e K / (N (a_m + 1)))^(a_m+1);
    at N = 2^16, K = 64, d = 256, a_m = 4 the bound is 0.0119.  Over 200 seeds
    the non-iterative method may fail on a handful at most."""
    N, K, M, am = 1 << 16, 64, 256, 4
    d = N // M
    bound = (N / d) * (d * np.e * K / (N * (am + 1))) ** (am + 1)
    assert abs(bound - 0.0119) < 1e-3
    fails = 0
    for seed in range(200):
        x, supp, _ = siggen.exact_signal(N, K, 10_000 + seed)
        _, _, un = orc.exact(x, M, am, orc.FIXED)
        fails += un > 0
    assert fails <= 8  # P(Binomial(200, 0.0119) > 8) < 1e-3


def test_theorem2_tau_bound(orc):
    """Theorem 2 with d = N/(mu K): at most tau*K bins fail except with
    probability (d^a K^a e^(a+2) / (tau N^a (a+1)^(a+1)))^(tau K) -- about
    0.16^205 at N = 2^22, K = 4096, mu = 2, tau = 0.05.  Checked on a smaller
    signal with the same K / M and mu (N = 2^18, K = 1024, M = 2048)."""
    N, K, M = 1 << 18, 1024, 2048
    tau = 0.05
    for seed in range(5):
        x, supp, _ = siggen.exact_signal(N, K, 777 + seed, mag=(1, 10))
        for mode in (orc.FIXED, orc.ITER):
            idx, _, un = orc.exact(x, M, 4, mode)
            assert un < tau * K
            assert np.isin(idx, supp).all()


def test_complex64_input_has_no_false_frequencies(orc):
    """A complex64 signal is exactly sparse only to its rounding; the oracle
    upcasts it and, with tolerances above that floor, reports no location
    outside the planted support."""
    for seed in range(3):
        x, supp, vals = siggen.exact_signal(1 << 20, 1024, seed, mag=(1, 10), dtype=np.complex64)
        for mode in (orc.ITER, orc.FIXED):
            idx, val, un = orc.exact(x, 2048, 4, mode)
            assert np.isin(idx, supp).all()
            assert len(idx) > 0.95 * 1024
            j = np.searchsorted(supp, idx)
            assert np.median(np.abs(val - vals[j]) / np.abs(vals[j])) < 1e-5


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_up_to_eight_aliases_matches_support_simulation(orc, mode):
    """a_m = 8 (Berlekamp-Massey locator and candidate search above four
    aliases, Sec. II-B): at K / M0 = 1 the non-iterative method solves every
    bin holding at most 8 frequencies and Algorithm 1 runs 8 levels; both
    recover exactly the set the decision rule predicts, with the planted
    values."""
    N, K, M0 = 1 << 18, 1024, 1024
    for seed in range(3):
        x, supp, vals = siggen.exact_signal(N, K, 40 + seed, mag=(1, 10))
        if mode == "iter":
            want, want_unres = simulate_iter(supp, M0, 8)
            idx, val, un = orc.exact(x, M0, 8, orc.ITER, cap=8 * M0)
        else:
            want, want_unres = simulate_fixed(supp, M0, 8)
            idx, val, un = orc.exact(x, M0, 8, orc.FIXED, cap=8 * M0)
        assert idx.tolist() == want, (seed, len(idx), len(want))
        assert un == want_unres, seed
        j = np.searchsorted(supp, idx)
        assert np.abs(val - vals[j]).max() < 1e-8 * np.abs(vals).max(), seed


def test_bad_parameters_rejected(orc):
    x = np.zeros(1000, complex)  # N not a power of two
    with pytest.raises(ValueError):
        orc.exact(x, 8)
    x = np.zeros(1024, complex)
    with pytest.raises(ValueError):
        orc.exact(x, 12)
    with pytest.raises(ValueError):
        orc.exact(x, 16, a_max=9)


def test_empty_signal(orc):
    x = np.zeros(1 << 12, complex)
    idx, val, un = orc.exact(x, 64)
    assert idx.size == 0 and un == 0


@pytest.mark.parametrize("mode", ["iter", "fixed"])
def test_unknown_k_stops_where_the_decision_rule_first_solves_every_bin(orc, mode):
    """Sec. II-E: starting at d = N (M = 1) and halving d, the bottom-up
    strategy stops at the first M whose run leaves no bin unsolved.  The
    support-only simulation of the decision rule predicts that M and the
    recovered set exactly; at that M the whole planted spectrum is
    returned."""
    for N, K, seeds in [(1 << 12, 5, range(8)), (1 << 14, 40, range(6)), (1 << 16, 300, range(3))]:
        for seed in seeds:
            x, supp, vals = siggen.exact_signal(N, K, seed, mag=(1, 10))
            M = 1
            while True:
                iters = min(4, int(np.log2(M)) + 1)
                want, un = (simulate_iter(supp, M, iters) if mode == "iter"
                            else simulate_fixed(supp, M, 4))
                if un == 0:
                    break
                M *= 2
            idx, val, un, M_got = orc.exact_auto(x, 4, orc.ITER if mode == "iter" else orc.FIXED)
            assert M_got == M and un == 0, (N, K, seed, M_got, M)
            assert idx.tolist() == sorted(supp.tolist())
            assert np.abs(val - vals[np.argsort(supp)]).max() < 1e-8 * np.abs(vals).max()
            # no earlier M solves every bin
            assert M == 1 or (simulate_iter(supp, M // 2, min(4, int(np.log2(M // 2)) + 1))[1]
                              if mode == "iter" else simulate_fixed(supp, M // 2, 4)[1]) > 0


def test_unknown_k_costs_at_most_twice_the_known_k_run(orc):
    """Sec. II-E's cost claim in transform sizes: the runs at M = 1, 2, ...,
    M* sum to sum_j 2^j log 2^j <= 2 M* log M* (FFT work of the final run)."""
    x, supp, _ = siggen.exact_signal(1 << 16, 300, 1, mag=(1, 10))
    _, _, _, Ms = orc.exact_auto(x, 4, orc.FIXED)
    total = sum((1 << j) * max(j, 1) for j in range(int(np.log2(Ms)) + 1))
    assert total <= 2 * Ms * max(int(np.log2(Ms)), 1)
