"""Seeded synthetic signals for the sparse FFT.

This module only *makes inputs*.  It holds none of the transform's own
arithmetic (no downsampling, no syndrome, no decoding); it is shared by the
CPU oracle tests, the GPU parity tests and the benchmark so that both sides
see byte-identical inputs.

Conventions (the unnormalised DFT, see the problem statement of Sec. II-A):

    X[s] = sum_n x[n] exp(-2 pi i s n / N),     x = IDFT(X) with 1/N.

Signal recipes follow the paper's experiments:

* exactly K-sparse (Sec. II-F): draw a K-sparse spectrum, then take the
  inverse FFT.  Positions are uniform without replacement; magnitudes are
  either 1 or uniform on [lo, hi]; phases are uniform on [0, 2 pi).
* generally K-sparse (Sec. III-F): the K significant terms as above plus
  i.i.d. complex Gaussian noise on every time sample.  White time noise is a
  white spectrum (Parseval), so SNR = 10 log10(||x_sig||^2 / ||noise||^2),
  the same quantity as SNR(x_s) of Eq. (37).
"""
from __future__ import annotations

import numpy as np

__all__ = ["sparse_support", "sparse_spectrum", "exact_signal", "noisy_signal",
           "tone_signal", "batch_exact", "hetero_batch_spec"]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed) & 0xFFFFFFFFFFFFFFFF, 0x5F1F]))


def sparse_support(N: int, K: int, rng: np.random.Generator) -> np.ndarray:
    """K distinct positions uniform in [0, N), sorted ascending (int64)."""
    if K > N:
        raise ValueError("K > N")
    if K == 0:
        return np.zeros(0, dtype=np.int64)
    if K * 4 >= N:  # dense case: a permutation is cheap enough
        return np.sort(rng.permutation(N)[:K]).astype(np.int64)
    pool = np.unique(rng.integers(0, N, size=int(K * 1.25) + 16, dtype=np.int64))
    while pool.size < K:
        more = rng.integers(0, N, size=K, dtype=np.int64)
        pool = np.unique(np.concatenate([pool, more]))
    pick = rng.choice(pool.size, size=K, replace=False)
    return np.sort(pool[pick]).astype(np.int64)


def sparse_spectrum(N: int, K: int, seed: int, mag=(1.0, 1.0)):
    """Return (support, values) of a K-sparse spectrum.

    mag=(1, 1) gives unit magnitudes; mag=(lo, hi) gives |X| ~ U[lo, hi].
    Phases are U[0, 2 pi).
    """
    rng = _rng(seed)
    supp = sparse_support(N, K, rng)
    lo, hi = float(mag[0]), float(mag[1])
    m = np.full(K, lo) if hi == lo else rng.uniform(lo, hi, size=K)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=K)
    vals = (m * np.exp(1j * ph)).astype(np.complex128)
    return supp, vals


def _idft_sparse(N: int, supp: np.ndarray, vals: np.ndarray) -> np.ndarray:
    X = np.zeros(N, dtype=np.complex128)
    X[supp] = vals
    return np.fft.ifft(X)


def exact_signal(N: int, K: int, seed: int, mag=(1.0, 1.0), dtype=np.complex128):
    """Exactly K-sparse time signal: x = IDFT(X).  Returns (x, support, values).

    With dtype=complex64 the FP64 signal is rounded once to complex64; the
    oracle then upcasts that same complex64 array, so both sides see one input.
    """
    supp, vals = sparse_spectrum(N, K, seed, mag)
    x = _idft_sparse(N, supp, vals).astype(dtype)
    return x, supp, vals


def noisy_signal(N: int, K: int, seed: int, snr_db: float, mag=(1.0, 10.0),
                 dtype=np.complex64):
    """Generally K-sparse signal: K significant tones plus white complex noise.

    Noise variance per sample: sigma^2 = (||x_sig||^2 / N) * 10^(-snr/10).
    Returns (x, support, values, x_sig) with x_sig the noiseless part (FP64).
    """
    supp, vals = sparse_spectrum(N, K, seed, mag)
    x_sig = _idft_sparse(N, supp, vals)
    rng = _rng(seed ^ 0x6E6F697365)  # independent stream for the noise
    p_sig = float(np.vdot(x_sig, x_sig).real) / N
    sigma2 = p_sig * 10.0 ** (-float(snr_db) / 10.0)
    s = np.sqrt(sigma2 / 2.0)
    noise = rng.normal(0.0, s, size=N) + 1j * rng.normal(0.0, s, size=N)
    x = (x_sig + noise).astype(dtype)
    return x, supp, vals, x_sig


def tone_signal(N: int, supp, vals, dtype=np.complex128) -> np.ndarray:
    """Time signal of an explicitly given sparse spectrum (for hand-built cases)."""
    supp = np.asarray(supp, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.complex128)
    return _idft_sparse(N, supp, vals).astype(dtype)


def batch_exact(N: int, K: int, seeds, mag=(1.0, 10.0), dtype=np.complex64, out=None):
    """Stack exact_signal() for several seeds into one [B, N] array.

    `out` may be a preallocated (e.g. pinned) [B, N] array of the same dtype.
    Returns (x[B, N], supports list, values list).
    """
    seeds = list(seeds)
    if out is None:
        out = np.empty((len(seeds), N), dtype=dtype)
    supps, valss = [], []
    for i, sd in enumerate(seeds):
        x, s, v = exact_signal(N, K, sd, mag, dtype)
        out[i] = x
        supps.append(s)
        valss.append(v)
    return out, supps, valss


def _next_pow2(v: int) -> int:
    return 1 << max(0, int(v - 1).bit_length())


def hetero_batch_spec(n_signals: int, seed: int):
    """Sizes for a heterogeneous batch: N = 2^u, u ~ U{12..20};
    K = round(2^v), v ~ U[3, 10], capped at N/64; even entries exactly sparse,
    odd entries noisy at 30 dB.  Bins: exact entries M = min(N, pow2 >= 4K);
    noisy entries M = min(N/16, pow2 >= 32K), so that d = N/M >= 16 leaves room
    for the 2a_m = 6 consecutive and r = 9 random shifts of the general path.
    Returns a list of dicts (N, K, M, kind, seed)."""
    rng = _rng(seed ^ 0xBA7C4)
    out = []
    for i in range(n_signals):
        u = int(rng.integers(12, 21))
        N = 1 << u
        K = int(round(2.0 ** rng.uniform(3.0, 10.0)))
        K = max(1, min(K, N // 64))
        kind = "exact" if i % 2 == 0 else "noisy"
        if kind == "exact":
            M = min(N, _next_pow2(4 * K))
        else:
            M = min(N // 16, _next_pow2(32 * K))
        out.append({"N": N, "K": K, "M": M, "kind": kind,
                    "seed": int(seed) * 100003 + i})
    return out
