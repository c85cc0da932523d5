"""Pins of the oracle's per-bin syndrome decoder (Sec. II-B, Alg. 1 SynDec):
planted bins with a = 1..4 aliases whose syndromes are written straight from
Eq. (3), the analytical a = 2 solution of the Appendix (with the sign of m_3
in c_1 restored), root finding against numpy, and rejection of bins holding
more aliases than decoded."""
import numpy as np
import pytest


def _planted_bin(N, M, k, a, seed, n_m):
    r = np.random.default_rng(seed)
    d = N // M
    t = np.sort(r.choice(d, size=a, replace=False))
    s = k + t * M
    p = r.uniform(1, 10, size=a) * np.exp(2j * np.pi * r.uniform(size=a))
    z = np.exp(2j * np.pi * s / N)
    m = np.array([(p * z ** i).sum() for i in range(n_m)])  # Eq. (3)
    return s, p, m


@pytest.mark.parametrize("a", [1, 2, 3, 4])
@pytest.mark.parametrize("n_extra", [0, 1, 4])
def test_decode_planted(orc, a, n_extra):
    N, M = 1 << 16, 256
    n_m = 2 * a + n_extra
    for trial in range(25):
        k = (37 * trial + 11) % M
        s, p, m = _planted_bin(N, M, k, a, 1000 * a + trial, n_m)
        ok, s_out, p_out = orc.decode(a, m, k, M, N, 1e-9, 0.1, 1e-9)
        assert ok, (a, trial)
        np.testing.assert_array_equal(s_out, s)
        assert np.abs(p_out - p).max() < 1e-8 * np.abs(p).max()


@pytest.mark.parametrize("a", [1, 2, 3])
def test_decode_rejects_more_aliases_than_decoded(orc, a):
    """A bin with a + 1 aliases cannot pass validation when decoded with a
    (Sec. II-B: with a > a_m the syndromes carry too little information)."""
    N, M = 1 << 16, 256
    for trial in range(40):
        k = (13 * trial + 5) % M
        _, _, m = _planted_bin(N, M, k, a + 1, 77 * a + trial, 2 * a)
        ok, _, _ = orc.decode(a, m, k, M, N, 1e-9, 0.1, 1e-9)
        assert not ok, (a, trial)


def test_decode_zero_bin_fails(orc):
    ok, _, _ = orc.decode(2, np.zeros(4), 3, 256, 1 << 16, 1e-9, 0.1, 1e-9)
    assert not ok


def test_decode_wrong_bin_index_fails(orc):
    """The decoded locations must lie in S_k (location check of SynDec, Algorithm 1)."""
    N, M = 1 << 16, 256
    s, p, m = _planted_bin(N, M, 17, 2, 5, 4)
    ok, _, _ = orc.decode(2, m, 18, M, N, 1e-9, 0.1, 1e-9)
    assert not ok


def test_appendix_a2_closed_form(orc):
    """Appendix, a = 2: c_d = |m0 m1; m1 m2|, c0 = |-m2 m1; -m3 m2| / c_d,
    c1 = |m0 -m2; m1 -m3| / c_d (the printed +m3 in c1 is a typo: with it the
    polynomial does not vanish at the planted roots), z = roots of
    z^2 + c1 z + c0, p0 = |m0 1; m1 z1| / (z1 - z0), p1 = m0 - p0."""
    N, M = 1 << 16, 256
    for trial in range(20):
        k = 3 + trial
        s, p, m = _planted_bin(N, M, k, 2, 500 + trial, 4)
        m0, m1, m2, m3 = m
        cd = m0 * m2 - m1 * m1
        c0 = (-m2 * m2 + m1 * m3) / cd
        c1 = (-m0 * m3 + m2 * m1) / cd
        disc = np.sqrt(c1 * c1 - 4 * c0)
        z0, z1 = (-c1 - disc) / 2, (-c1 + disc) / 2
        p0 = (m0 * z1 - m1) / (z1 - z0)
        p1 = m0 - p0
        zt = np.exp(2j * np.pi * s / N)
        # closed form reproduces the planted aliases (in some order)
        pairs = sorted(zip([z0, z1], [p0, p1]), key=lambda e: np.angle(e[0] / zt[0]) ** 2)
        assert abs(pairs[0][0] - zt[0]) < 1e-9 and abs(pairs[1][0] - zt[1]) < 1e-9
        assert abs(pairs[0][1] - p[0]) < 1e-8 and abs(pairs[1][1] - p[1]) < 1e-8
        # the oracle's decoder agrees
        ok, s_out, p_out = orc.decode(2, m, k, M, N, 1e-9, 0.1, 1e-9)
        assert ok
        np.testing.assert_array_equal(s_out, s)
        assert np.abs(p_out - p).max() < 1e-8
        # the printed sign does not solve Eq. (5)
        c1_printed = (m0 * m3 + m2 * m1) / cd
        assert abs(zt[0] ** 2 + c1_printed * zt[0] + c0) > 1e-3


@pytest.mark.parametrize("a", [1, 2, 3, 4])
def test_poly_roots_against_numpy(orc, a):
    r = np.random.default_rng(a)
    for trial in range(50):
        if trial % 2:
            roots = np.exp(2j * np.pi * r.uniform(size=a))       # unit circle
        else:
            roots = r.normal(size=a) + 1j * r.normal(size=a)     # general
        coeffs = np.poly(roots)              # highest power first, monic
        c = coeffs[::-1][:-1]                # c_0 .. c_{a-1}
        z = orc.poly_roots(c)
        for rt in roots:
            assert np.min(np.abs(z - rt)) < 1e-9 * max(1, np.abs(roots).max())
        P = np.polyval(coeffs, z)
        assert np.abs(P).max() < 1e-9 * max(1, np.abs(coeffs).max())


def test_poly_roots_biquadratic(orc):
    """q = 0 in Ferrari's reduction: z^4 - 1 has roots 1, -1, i, -i."""
    z = orc.poly_roots([-1, 0, 0, 0])
    for rt in (1, -1, 1j, -1j):
        assert np.min(np.abs(z - rt)) < 1e-12


# ---------------------------------------------- more than four aliases
@pytest.mark.parametrize("a", [1, 3, 5, 6, 7, 8])
def test_bm_locator_is_the_root_polynomial(orc, a):
    """Berlekamp-Massey on the 2a syndromes of a planted a-alias bin returns
    the locator whose roots are the planted z_j = omega^{s_j}: its
    coefficients are those of prod_j (z - z_j) (numpy.poly)."""
    N, M = 1 << 20, 1024
    for trial in range(10):
        s, p, m = _planted_bin(N, M, (91 * trial) % M, a, 500 * a + trial, 2 * a)
        c = orc.bm_locator(m, a)
        assert c is not None
        want = np.poly(np.exp(2j * np.pi * s / N))[::-1][:a]  # c_0 .. c_{a-1}
        assert np.abs(c - want).max() < 1e-6 * max(1.0, np.abs(want).max()), (a, trial)


@pytest.mark.parametrize("a", [5, 6, 7, 8])
@pytest.mark.parametrize("n_extra", [0, 2])
def test_decode_above_four_planted(orc, a, n_extra):
    """a > 4: Berlekamp-Massey locator, candidate search over the d members
    of S_k, least-squares values: the planted bin comes back exactly (with
    up to 16 syndromes, the most a bin holds at a_m = 8)."""
    N, M = 1 << 20, 1024
    for trial in range(12):
        k = (53 * trial + 7) % M
        s, p, m = _planted_bin(N, M, k, a, 900 * a + trial, min(16, 2 * a + n_extra))
        ok, s_out, p_out = orc.decode(a, m, k, M, N, 1e-9, 0.1, 1e-9)
        assert ok, (a, trial)
        np.testing.assert_array_equal(s_out, s)
        assert np.abs(p_out - p).max() < 1e-8 * np.abs(p).max()


@pytest.mark.parametrize("a", [5, 7])
def test_decode_above_four_rejects_more_aliases(orc, a):
    """A bin with a + 1 aliases fails validation when decoded with a (its
    2a syndromes carry too little information).  (A bin with fewer aliases
    never reaches the a-alias decoder: FIXED tries a = 1, 2, ... in turn and
    ITER's residual counts after level l are 0 or at least l + 2.)"""
    N, M = 1 << 20, 1024
    for trial in range(12):
        k = (29 * trial + 3) % M
        _, _, m_more = _planted_bin(N, M, k, a + 1, 31 * a + trial, 2 * a)
        assert not orc.decode(a, m_more, k, M, N, 1e-9, 0.1, 1e-9)[0], (a, trial)
