"""Plain FP64 CPU oracle of sFFT-DT -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it.  The C source (``sfft_oracle.c``) follows Algorithm 1
and Sec. II-B of the paper step by step; this module only builds it with gcc
and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["sfft_oracle.c"]
_lock = threading.Lock()
_lib = None

ITER, FIXED = 0, 1

# Validation tolerances, keyed to the precision of the *input*: a complex128
# signal is exactly sparse to ~1e-16, a complex64 one only to its rounding
# (~1e-7 relative), and the thresholds sit between that floor and O(1).
# root_tol is only a sanity bound (the root must lie near the unit circle):
# for adjacent aliases the Hankel system has condition ~1e4-1e5 and the root
# moves by ~1e-3 while its nearest candidate stays right; the residual test
# (res_tol, in data units) is the discriminating check.
TOL_FP64 = dict(zero_tol=1e-10, root_tol=0.1, res_tol=1e-9)
TOL_MIXED = dict(zero_tol=1e-6, root_tol=0.1, res_tol=1e-6)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "sfft_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # no contraction into fused multiply-adds: the same rounding on every
    # host (gcc fuses by default where the target has FMA, e.g. aarch64)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-o",
           tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(C.Structure):
    _fields_ = [("N", C.c_int64), ("M0", C.c_int64), ("a_max", C.c_int32),
                ("max_iters", C.c_int32), ("mode", C.c_int32), ("pad_", C.c_int32),
                ("zero_tol", C.c_double), ("root_tol", C.c_double), ("res_tol", C.c_double)]


class _GParams(C.Structure):
    _fields_ = [("N", C.c_int64), ("K", C.c_int64), ("M", C.c_int64), ("a_max", C.c_int32),
                ("r", C.c_int32), ("seed", C.c_uint64), ("keep", C.c_int32),
                ("sp_iters", C.c_int32), ("prune", C.c_int32), ("pad_", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            lib.orc_fft.argtypes = [C.c_int64, P(C.c_double), C.c_int]
            lib.orc_dft_brute.argtypes = [C.c_int64, P(C.c_double), P(C.c_double), C.c_int]
            lib.orc_syndrome.argtypes = [P(C.c_double), C.c_int64, C.c_int64, C.c_int64,
                                         P(C.c_double)]
            lib.orc_poly_roots.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            lib.orc_bm_locator.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            lib.orc_decode.argtypes = [C.c_int, P(C.c_double), C.c_int, C.c_int64, C.c_int64,
                                       C.c_int64, C.c_double, C.c_double, C.c_double,
                                       P(C.c_int64), P(C.c_double)]
            lib.orc_exact.argtypes = [P(C.c_double), P(_Params), C.c_int64, P(C.c_int64),
                                      P(C.c_double), P(C.c_int64)]
            lib.orc_exact.restype = C.c_int64
            lib.orc_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
            lib.orc_splitmix64.restype = C.c_uint64
            lib.orc_cs_shifts.argtypes = [C.c_uint64, C.c_int64, C.c_int, P(C.c_int64)]
            lib.orc_hankel_svals.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            lib.orc_subspace_pursuit.argtypes = [C.c_int, C.c_int, P(C.c_double), P(C.c_double),
                                                 C.c_int, C.c_int, P(C.c_double)]
            lib.orc_general.argtypes = [P(C.c_double), P(_GParams), C.c_int64, P(C.c_int64),
                                        P(C.c_double), P(C.c_ubyte)]
            lib.orc_general.restype = C.c_int64
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def fft(a, sign: int = -1) -> np.ndarray:
    """Unnormalised radix-2 FFT (sign -1 forward, +1 inverse)."""
    a = _c128(a).copy()
    if _load().orc_fft(a.size, _dp(a), int(sign)) != 0:
        raise ValueError("length must be a power of two")
    return a


def dft_brute(a, sign: int = -1) -> np.ndarray:
    a = _c128(a)
    out = np.empty_like(a)
    _load().orc_dft_brute(a.size, _dp(a), _dp(out), int(sign))
    return out


def syndrome(x, d: int, shift: int) -> np.ndarray:
    """Y_{d,shift} = d * FFT_{N/d}(x[n d + shift])  (Eq. (2))."""
    x = _c128(x)
    N = x.size
    Y = np.empty(N // d, dtype=np.complex128)
    if _load().orc_syndrome(_dp(x), N, int(d), int(shift), _dp(Y)) != 0:
        raise ValueError("bad sizes")
    return Y


def poly_roots(c) -> np.ndarray:
    """Roots of z^a + c[a-1] z^{a-1} + ... + c[0], 1 <= a <= 4."""
    c = _c128(c)
    z = np.empty(c.size, dtype=np.complex128)
    if _load().orc_poly_roots(c.size, _dp(c), _dp(z)) != 0:
        raise ValueError("degree must be 1..4")
    return z


def decode(a: int, m, k: int, M: int, N: int, theta: float, root_tol: float, res_tol: float):
    """SynDec of one bin: returns (ok, s[a], p[a])."""
    m = _c128(m)
    s = np.zeros(8, dtype=np.int64)
    p = np.zeros(8, dtype=np.complex128)
    ok = _load().orc_decode(int(a), _dp(m), m.size, int(k), int(M), int(N), float(theta),
                            float(root_tol), float(res_tol),
                            s.ctypes.data_as(C.POINTER(C.c_int64)), _dp(p))
    return bool(ok), s[:a].copy(), p[:a].copy()


def bm_locator(m, a: int):
    """Berlekamp-Massey locator for a aliases from m_0..m_{2a-1}: returns c
    (c_0..c_{a-1} of P(z) = z^a + sum c_j z^j) or None when the shortest
    recurrence is not of length a."""
    m = _c128(m)
    c = np.zeros(8, dtype=np.complex128)
    ok = _load().orc_bm_locator(int(a), _dp(m), _dp(c))
    return c[:a].copy() if ok else None


def exact(x, M0: int, a_max: int = 4, mode: int = ITER, max_iters: int | None = None,
          zero_tol: float | None = None, root_tol: float | None = None,
          res_tol: float | None = None, cap: int | None = None):
    """Whole exactly-K-sparse sFFT-DT.  x of any complex dtype is upcast to
    complex128.  Default tolerances are TOL_MIXED for complex64 input and
    TOL_FP64 otherwise.  Returns (idx int64 sorted, val complex128, unresolved)."""
    x_in = np.asarray(x)
    tol = TOL_MIXED if x_in.dtype == np.complex64 else TOL_FP64
    x = _c128(x_in)
    N = x.size
    prm = _Params(N=N, M0=int(M0), a_max=int(a_max),
                  max_iters=int(a_max if max_iters is None else max_iters), mode=int(mode),
                  pad_=0,
                  zero_tol=float(tol["zero_tol"] if zero_tol is None else zero_tol),
                  root_tol=float(tol["root_tol"] if root_tol is None else root_tol),
                  res_tol=float(tol["res_tol"] if res_tol is None else res_tol))
    if cap is None:
        cap = int(M0) * int(a_max)
    idx = np.zeros(cap, dtype=np.int64)
    val = np.zeros(cap, dtype=np.complex128)
    unres = C.c_int64(0)
    n = _load().orc_exact(_dp(x), C.byref(prm), int(cap),
                          idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(val), C.byref(unres))
    if n < 0:
        raise ValueError("bad parameters")
    n = min(int(n), cap)
    return idx[:n].copy(), val[:n].copy(), int(unres.value)


def exact_auto(x, a_max: int = 4, mode: int = ITER, M_start: int = 1, M_max: int | None = None,
               zero_tol: float | None = None, root_tol: float | None = None,
               res_tol: float | None = None):
    """Unknown K (Sec. II-E, the bottom-up strategy): run the exact transform
    with d = N / M_start and halve d (double M) until a run leaves no bin
    unsolved, or M reaches M_max (default N).  ITER runs
    min(a_max, log2(M) + 1) levels.  Returns (idx, val, unresolved, M) of the
    last run."""
    x = np.asarray(x)
    N = x.size
    M_max = N if M_max is None else int(M_max)
    M = int(M_start)
    while True:
        iters = min(int(a_max), int(np.log2(M)) + 1) if mode == ITER else int(a_max)
        idx, val, un = exact(x, M, a_max, mode, max_iters=iters, zero_tol=zero_tol,
                             root_tol=root_tol, res_tol=res_tol, cap=4 * M * int(a_max))
        if un == 0 or M >= M_max:
            return idx, val, un, M
        M *= 2


# --------------------------------------------- generally K-sparse (Alg. 2)
def splitmix64(seed: int, i: int) -> int:
    """Output i of the SplitMix64 stream of `seed`."""
    return int(_load().orc_splitmix64(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), i))


def cs_shifts(seed: int, d: int, r: int) -> np.ndarray:
    """The r distinct random shifts n_l in [0, d) drawn from `seed`."""
    out = np.zeros(r, dtype=np.int64)
    if _load().orc_cs_shifts(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(d), int(r),
                             out.ctypes.data_as(C.POINTER(C.c_int64))) != 0:
        raise ValueError("need 0 <= r <= d")
    return out


def hankel_svals(m, n: int) -> np.ndarray:
    """Singular values (descending) of the n x n Hankel matrix H_ij = m_{i+j}."""
    m = _c128(m)
    if m.size < 2 * n - 1:
        raise ValueError("need 2n - 1 syndromes")
    sv = np.zeros(n)
    _load().orc_hankel_svals(int(n), _dp(m), sv.ctypes.data_as(C.POINTER(C.c_double)))
    return sv


def subspace_pursuit(Phi, y, ks: int, iters: int = 8) -> np.ndarray:
    Phi = _c128(Phi)
    y = _c128(y)
    rows, cols = Phi.shape
    b = np.zeros(cols, dtype=np.complex128)
    n = _load().orc_subspace_pursuit(rows, cols, _dp(Phi), _dp(y), int(ks), int(iters), _dp(b))
    if n < 0:
        raise ValueError("subspace pursuit failed")
    return b


def general(x, M: int, K: int, a_max: int = 3, r: int | None = None, seed: int = 0,
            keep: int = 2, sp_iters: int = 8, cap: int | None = None, prune: bool = True):
    """Algorithm 2 on x (upcast to complex128).  Returns (idx, val, a_k).
    prune=False: the CS model of Sec. III-B without the pruning strategy
    (every bin by SP at sparsity a_m over all d candidates; K unused)."""
    x = _c128(x)
    N = x.size
    r = 3 * a_max if r is None else r
    prm = _GParams(N=N, K=int(K), M=int(M), a_max=int(a_max), r=int(r),
                   seed=int(seed) & 0xFFFFFFFFFFFFFFFF, keep=int(keep), sp_iters=int(sp_iters),
                   prune=1 if prune else 0)
    cap = int(K) * 2 + 16 if cap is None else int(cap)
    idx = np.zeros(cap, dtype=np.int64)
    val = np.zeros(cap, dtype=np.complex128)
    ak = np.zeros(M, dtype=np.uint8)
    n = _load().orc_general(_dp(x), C.byref(prm), cap, idx.ctypes.data_as(C.POINTER(C.c_int64)),
                            _dp(val), ak.ctypes.data_as(C.POINTER(C.c_ubyte)))
    if n < 0:
        raise ValueError("bad parameters")
    n = min(int(n), cap)
    return idx[:n].copy(), val[:n].copy(), ak


def alias_histogram(supports, M: int, n_cells: int = 9) -> np.ndarray:
    """Collision counts of Sec. II-C (Lemma 2, Fig. 2): for each support set
    (a row of `supports`), the number of bins k < M that hold exactly a of
    its locations, k = s mod M; summed over the sets.  hist[a] for
    a < n_cells - 1; the last cell counts n_cells - 1 or more."""
    S = np.asarray(supports, dtype=np.int64)
    if S.ndim == 1:
        S = S[None, :]
    hist = np.zeros(n_cells, dtype=np.int64)
    for row in S:
        counts = np.bincount(row % M, minlength=M)
        hist += np.bincount(np.minimum(counts, n_cells - 1), minlength=n_cells)
    return hist


def alias_count_pmf(N: int, K: int, M: int, a: int) -> float:
    """P(a bin holds exactly a locations) for K distinct locations drawn
    uniformly from [0, N) and a bin of d = N/M candidates: hypergeometric,
    C(d, a) C(N - d, K - a) / C(N, K)."""
    from math import comb
    d = N // M
    if a < 0 or a > d or a > K:
        return 0.0
    return comb(d, a) * comb(N - d, K - a) / comb(N, K)
