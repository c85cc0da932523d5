/*
 * sfft_oracle.h -- plain FP64 CPU oracle of sFFT-DT (Hsieh, Lu, Pei).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the GPU library.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call it; the library never links or calls it, and it shares no code,
 * header, table or constant with the GPU path.
 *
 * Conventions (reading of Sec. II-A and Eq. (1)-(2)):
 *   X[s] = sum_n x[n] e^{-2 pi i s n/N}   (unnormalised DFT)
 *   omega = e^{+2 pi i / N}
 *   Y_{d,l}[k] = d * FFT_M(x[n d + l])[k] = sum_{j<d} X[k + jM] omega^{(k+jM) l}
 * so the syndromes m_l of bin k are moments sum_j p_j z_j^l with p_j = X[s_j]
 * and z_j = omega^{s_j} (Eq. (3)).
 */
#ifndef SFFT_ORACLE_H
#define SFFT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Complex arrays are interleaved (re, im) doubles. */

/* In-place radix-2 FFT, unnormalised; sign = -1 forward, +1 inverse.
 * n must be a power of two.  Returns 0, or -1 on bad n. */
int orc_fft(int64_t n, double* a, int sign);

/* O(n^2) DFT straight from the definition (for pinning orc_fft). */
int orc_dft_brute(int64_t n, const double* in, double* out, int sign);

/* Syndrome spectrum of one shift (Eq. (2); the syndrome step of Algorithm 1):
 *   Y[k] = d * sum_{n<M} x[n d + shift] e^{-2 pi i k n / M},  M = N/d.
 * Returns 0, or -1 on bad sizes. */
int orc_syndrome(const double* x, int64_t N, int64_t d, int64_t shift, double* Y);

/* Roots of z^a + c[a-1] z^{a-1} + ... + c[0] for 1 <= a <= 4 by the
 * analytical solutions (quadratic, Cardano, Ferrari).  Returns 0 / -1. */
int orc_poly_roots(int a, const double* c, double* z);

/* Berlekamp-Massey locator for a aliases from m_0..m_{2a-1} (Step (i) for
 * a > 4): writes c[a] with sum_j c_j m_{i+j} = -m_{a+i} and returns 1 when
 * the shortest recurrence has length exactly a, else 0. */
int orc_bm_locator(int a, const double* m, double* c);

/* SynDec of one bin (Sec. II-B steps (i)-(iii); SynDec of Algorithm 1).
 *   a      number of aliases assumed (1..8): a <= 4 by the Hankel solve and
 *          the analytical roots snapped to S_k; a > 4 by the
 *          Berlekamp-Massey locator and the a smallest |P| over the d
 *          candidates of S_k (each at most root_tol (1 + sum |c_j|))
 *   m      n_m syndromes m_0..m_{n_m-1} of bin k (2a <= n_m <= 16)
 *   k, M, N  bin index, number of bins, signal length
 *   theta  zero threshold; root_tol, res_tol  validation tolerances
 * On success writes s_out[a] (ascending) and p_out[a] and returns 1;
 * returns 0 when the bin does not decode with a aliases. */
int orc_decode(int a, const double* m, int n_m, int64_t k, int64_t M, int64_t N,
               double theta, double root_tol, double res_tol,
               int64_t* s_out, double* p_out);

enum { ORC_ITER = 0, ORC_FIXED = 1 };

typedef struct {
  int64_t N;          /* signal length (power of two)                        */
  int64_t M0;         /* number of bins at the first level, d0 = N / M0       */
  int32_t a_max;      /* largest alias count decoded (1..8)                  */
  int32_t max_iters;  /* ITER: number of levels (<= a_max)                    */
  int32_t mode;       /* ORC_ITER (Algorithm 1) or ORC_FIXED (non-iterative)  */
  int32_t pad_;
  double zero_tol;    /* theta = zero_tol * max_k |Y_{d0,0}[k]|               */
  double root_tol;    /* |z_j - omega^{s_j}| bound                            */
  double res_tol;     /* ||m - Z p||_inf <= res_tol * ||m||_inf               */
} orc_exact_params;

/* Whole exactly-K-sparse transform.  Writes up to cap (s, X[s]) pairs sorted
 * by s into idx / val, the number of unresolved bins into *unresolved, and
 * returns the number of recovered frequencies (or -1 on bad parameters). */
int64_t orc_exact(const double* x, const orc_exact_params* p, int64_t cap,
                  int64_t* idx, double* val, int64_t* unresolved);

#ifdef __cplusplus
}
#endif
#endif

#ifndef SFFT_ORACLE_GENERAL_H
#define SFFT_ORACLE_GENERAL_H
#ifdef __cplusplus
extern "C" {
#endif

/* ---- generally K-sparse signals (Sec. III, Algorithm 2) ---------------- */

/* SplitMix64 (Steele, Lea, Flood 2014): output i of the stream seeded with
 * `seed` (counter-based: state = seed + (i+1) * 0x9E3779B97F4A7C15). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i);

/* r distinct shifts uniform in [0, d) (reading of Sec. III-A: "uniformly
 * drawn", without replacement so no measurement repeats): partial
 * Fisher-Yates on 0..d-1 driven by the SplitMix64 stream of `seed`,
 * draw i swapping position i with i + (u_i mod (d - i)).  Returns 0 / -1. */
int orc_cs_shifts(uint64_t seed, int64_t d, int r, int64_t* out);

/* Singular values (descending) of the n x n complex Hankel matrix
 * H_ij = m_{i+j} (Eq. (26)), by one-sided Jacobi in FP64. */
int orc_hankel_svals(int n, const double* m, double* sv);

/* Subspace Pursuit (Dai and Dai 2009) for y = Phi b with sparsity ks:
 * Phi is rows x cols (row-major, complex; rows <= 32, cols <= 2^16,
 * ks <= 8), at most `iters` iterations.  Writes b (cols complex values, ks
 * of them non-zero) and returns the number of non-zeros (or -1). */
int orc_subspace_pursuit(int rows, int cols, const double* Phi, const double* y, int ks,
                         int iters, double* b);

typedef struct {
  int64_t N;        /* signal length                                        */
  int64_t K;        /* number of significant frequencies kept               */
  int64_t M;        /* bins, d = N / M                                      */
  int32_t a_max;    /* a_m: syndromes 0..2a_m-1, Hankel a_m x a_m           */
  int32_t r;        /* random shifts for the CS measurements (3 a_m)        */
  uint64_t seed;    /* draws the random shifts                              */
  int32_t keep;     /* candidates kept per significant term (2: O(a) = 2a)  */
  int32_t sp_iters; /* Subspace Pursuit iteration cap                       */
  int32_t prune;    /* 1: Algorithm 2 with the pruning strategy (Sec. III-C);
                       0: the CS model of Sec. III-B without it -- every bin
                       solved by SP at sparsity a_m over all d candidates   */
  int32_t pad_;
} orc_general_params;

/* Algorithm 2.  Writes the recovered (s, X[s]) in ascending s (at most cap)
 * and, if a_k is not NULL, the vote a_k of every bin (M bytes; a_m for
 * every bin without pruning).  Returns the number of entries or -1. */
int64_t orc_general(const double* x, const orc_general_params* p, int64_t cap, int64_t* idx,
                    double* val, unsigned char* a_k);

#ifdef __cplusplus
}
#endif
#endif
