/*
 * sfft_oracle.c -- plain FP64 CPU oracle of sFFT-DT for exactly K-sparse
 * signals (Sec. II, Algorithm 1).  TEST INFRASTRUCTURE ONLY: called by the
 * tests, the smoke check and the benchmark's CPU baseline, never by the
 * library.  Slow on purpose: every step is written the way the paper states
 * it, with no blocking, fusion or reordering.
 */
#include "sfft_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

/* omega^e with omega = e^{2 pi i / N}; the exponent is reduced mod N in
 * integers first so that e * l never loses precision. */
static cplx omega_pow(int64_t N, int64_t e) {
  int64_t r = e % N;
  if (r < 0) r += N;
  double t = (double)r / (double)N; /* exact for power-of-two N */
  return cos(TWO_PI * t) + I * sin(TWO_PI * t);
}

/* ------------------------------------------------------------------ FFT */

int orc_fft(int64_t n, double* data, int sign) {
  if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
  cplx* a = (cplx*)data;
  /* bit-reversal permutation */
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      cplx t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  /* iterative radix-2 butterflies; each twiddle from its own cos/sin */
  for (int64_t len = 2; len <= n; len <<= 1) {
    int64_t half = len >> 1;
    for (int64_t j = 0; j < half; ++j) {
      double t = (double)j / (double)len;
      cplx w = cos(TWO_PI * t) + I * (sign * sin(TWO_PI * t));
      for (int64_t i = 0; i < n; i += len) {
        cplx u = a[i + j];
        cplx v = a[i + j + half] * w;
        a[i + j] = u + v;
        a[i + j + half] = u - v;
      }
    }
  }
  return 0;
}

int orc_dft_brute(int64_t n, const double* in, double* out, int sign) {
  if (n <= 0 || (sign != 1 && sign != -1)) return -1;
  const cplx* x = (const cplx*)in;
  cplx* X = (cplx*)out;
  for (int64_t k = 0; k < n; ++k) {
    cplx acc = 0;
    for (int64_t j = 0; j < n; ++j) {
      int64_t e = (k * j) % n;
      double t = (double)e / (double)n;
      acc += x[j] * (cos(TWO_PI * t) + I * (sign * sin(TWO_PI * t)));
    }
    X[k] = acc;
  }
  return 0;
}

/* ------------------------------------------------------------ syndromes */

/* Eq. (2) with X the unnormalised DFT (x its inverse with 1/N):
 * Y_{d,l} = d * FFT_M(x_{d,l}),  x_{d,l}[n] = x[n d + l]. */
int orc_syndrome(const double* xin, int64_t N, int64_t d, int64_t shift, double* Yout) {
  if (!is_pow2(N) || d <= 0 || N % d != 0 || shift < 0) return -1;
  int64_t M = N / d;
  if (!is_pow2(M)) return -1;
  const cplx* x = (const cplx*)xin;
  cplx* Y = (cplx*)Yout;
  for (int64_t n = 0; n < M; ++n) Y[n] = x[(n * d + shift) % N];
  orc_fft(M, (double*)Y, -1);
  for (int64_t k = 0; k < M; ++k) Y[k] *= (double)d;
  return 0;
}

/* ------------------------------------------------- small linear algebra */

/* Gaussian elimination with partial pivoting on an n x n complex system
 * A x = b (A row-major, destroyed).  Fails when a pivot is zero or below
 * 1e-14 of the largest entry of A. */
static int solve_lin(int n, cplx* A, cplx* b, cplx* x) {
  double amax = 0;
  for (int i = 0; i < n * n; ++i) amax = fmax(amax, cabs(A[i]));
  if (!(amax > 0)) return 0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (cabs(A[r * n + col]) > cabs(A[piv * n + col])) piv = r;
    if (!(cabs(A[piv * n + col]) > 1e-14 * amax)) return 0;
    if (piv != col) {
      for (int c = 0; c < n; ++c) {
        cplx t = A[col * n + c];
        A[col * n + c] = A[piv * n + c];
        A[piv * n + c] = t;
      }
      cplx t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
    for (int r = col + 1; r < n; ++r) {
      cplx f = A[r * n + col] / A[col * n + col];
      for (int c = col; c < n; ++c) A[r * n + c] -= f * A[col * n + c];
      b[r] -= f * b[col];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    cplx acc = b[r];
    for (int c = r + 1; c < n; ++c) acc -= A[r * n + c] * x[c];
    x[r] = acc / A[r * n + r];
  }
  return 1;
}

/* ------------------------------------------------------- polynomial roots */

static cplx cbrt_c(cplx v) {
  if (v == 0) return 0;
  return cpow(v, 1.0 / 3.0);
}

/* Roots of the monic quadratic z^2 + b z + c, in the cancellation-free form
 * q = -(b + sgn * sqrt(b^2 - 4c)) / 2,  z1 = q,  z2 = c / q. */
static void roots2(cplx b, cplx c, cplx* z) {
  cplx sq = csqrt(b * b - 4.0 * c);
  cplx qp = b + sq, qm = b - sq;
  cplx q = -0.5 * (cabs(qp) >= cabs(qm) ? qp : qm);
  if (q == 0) {
    z[0] = z[1] = 0;
    return;
  }
  z[0] = q;
  z[1] = c / q;
}

/* Monic cubic z^3 + c2 z^2 + c1 z + c0 by Cardano: z = y - c2/3 gives the
 * depressed cubic y^3 + p y + q = 0; y = u + v with u^3 = -q/2 + sqrt(D),
 * D = (q/2)^2 + (p/3)^3 and u v = -p/3.  The three roots take u through its
 * three cube-root branches. */
static void roots3(cplx c2, cplx c1, cplx c0, cplx* z) {
  cplx sh = c2 / 3.0;
  cplx p = c1 - c2 * c2 / 3.0;
  cplx q = 2.0 * c2 * c2 * c2 / 27.0 - c2 * c1 / 3.0 + c0;
  cplx sD = csqrt(q * q / 4.0 + p * p * p / 27.0);
  cplx w1 = -q / 2.0 + sD, w2 = -q / 2.0 - sD;
  cplx u = cbrt_c(cabs(w1) >= cabs(w2) ? w1 : w2);
  const cplx e3 = -0.5 + I * 0.86602540378443864676372317075294; /* e^{2 pi i/3} */
  cplx br[3] = {1.0, e3, conj(e3)};
  for (int j = 0; j < 3; ++j) {
    cplx uj = u * br[j];
    cplx vj = (uj == 0) ? 0 : -p / (3.0 * uj);
    z[j] = uj + vj - sh;
  }
}

/* Monic quartic z^4 + c3 z^3 + c2 z^2 + c1 z + c0 by Ferrari: z = y - c3/4
 * gives y^4 + p y^2 + q y + r.  With m a root of the resolvent cubic
 * 8 m^3 + 8 p m^2 + (2 p^2 - 8 r) m - q^2 = 0 the quartic factors as
 * (y^2 - s y + p/2 + m + q/(2s)) (y^2 + s y + p/2 + m - q/(2s)), s^2 = 2m.
 * When every resolvent root is zero (q = 0) the quartic is biquadratic. */
static void roots4(cplx c3, cplx c2, cplx c1, cplx c0, cplx* z) {
  cplx sh = c3 / 4.0;
  cplx p = c2 - 3.0 * c3 * c3 / 8.0;
  cplx q = c3 * c3 * c3 / 8.0 - c3 * c2 / 2.0 + c1;
  cplx r = -3.0 * c3 * c3 * c3 * c3 / 256.0 + c3 * c3 * c2 / 16.0 - c3 * c1 / 4.0 + c0;
  cplx mr[3];
  roots3(p, (2.0 * p * p - 8.0 * r) / 8.0, -q * q / 8.0, mr);
  int best = 0;
  for (int j = 1; j < 3; ++j)
    if (cabs(mr[j]) > cabs(mr[best])) best = j;
  cplx m = mr[best];
  cplx y[4];
  if (cabs(m) == 0) {
    cplx w[2];
    roots2(p, r, w);
    y[0] = csqrt(w[0]);
    y[1] = -y[0];
    y[2] = csqrt(w[1]);
    y[3] = -y[2];
  } else {
    cplx s = csqrt(2.0 * m);
    roots2(-s, p / 2.0 + m + q / (2.0 * s), y);
    roots2(s, p / 2.0 + m - q / (2.0 * s), y + 2);
  }
  for (int j = 0; j < 4; ++j) z[j] = y[j] - sh;
}

int orc_poly_roots(int a, const double* cin, double* zout) {
  const cplx* c = (const cplx*)cin;
  cplx* z = (cplx*)zout;
  switch (a) {
    case 1: z[0] = -c[0]; return 0;
    case 2: roots2(c[1], c[0], z); return 0;
    case 3: roots3(c[2], c[1], c[0], z); return 0;
    case 4: roots4(c[3], c[2], c[1], c[0], z); return 0;
    default: return -1;
  }
}

/* ---------------------------------------------------------------- SynDec */

/* Step (i) for a > 4 (Sec. II-B cites Berlekamp-Massey for it): the
 * shortest linear recurrence m_n + sum_{i=1}^{L} C_i m_{n-i} = 0 (n >= L)
 * that generates m_0..m_{2a-1}, built one syndrome at a time (Massey,
 * "Shift-register synthesis and BCH decoding", 1969).  A discrepancy counts
 * as zero only when it is exactly zero.  The locator exists when L = a;
 * then Eq. (4)-(5) hold with c_j = C_{a-j}. */
int orc_bm_locator(int a, const double* min, double* cout) {
  const cplx* m = (const cplx*)min;
  cplx* c = (cplx*)cout;
  if (a < 1 || a > 8) return 0;
  cplx C[17] = {0}, Bp[17] = {0}, T[17];
  C[0] = 1;
  Bp[0] = 1;
  int L = 0, shift = 1;
  cplx bd = 1;
  for (int n = 0; n < 2 * a; ++n) {
    cplx delta = m[n];
    for (int i = 1; i <= L; ++i) delta += C[i] * m[n - i];
    if (delta == 0) {
      ++shift;
      continue;
    }
    const cplx f = delta / bd;
    if (2 * L <= n) {
      memcpy(T, C, sizeof T);
      for (int i = 0; i + shift <= 16; ++i) C[i + shift] -= f * Bp[i];
      L = n + 1 - L;
      memcpy(Bp, T, sizeof T);
      bd = delta;
      shift = 1;
    } else {
      for (int i = 0; i + shift <= 16; ++i) C[i + shift] -= f * Bp[i];
      ++shift;
    }
  }
  if (L != a) return 0;
  for (int j = 0; j < a; ++j) c[j] = C[a - j];
  return 1;
}

int orc_decode(int a, const double* min, int n_m, int64_t k, int64_t M, int64_t N,
               double theta, double root_tol, double res_tol,
               int64_t* s_out, double* p_out) {
  if (a < 1 || a > 8 || n_m < 2 * a || n_m > 16 || M <= 0 || N % M != 0) return 0;
  const cplx* m = (const cplx*)min;
  int64_t d = N / M;
  if (d < a) return 0;
  int64_t s[8];
  cplx c[8];

  if (a <= 4) {
    /* Step (i), Eq. (4)-(5): the a x a Hankel system
     *   sum_j c_j m_{i+j} = -m_{a+i},  i = 0..a-1. */
    cplx H[16], rhs[4];
    for (int i = 0; i < a; ++i) {
      for (int j = 0; j < a; ++j) H[i * a + j] = m[i + j];
      rhs[i] = -m[a + i];
    }
    if (!solve_lin(a, H, rhs, c)) return 0;

    /* Step (ii): the roots z_j of P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0. */
    cplx z[4];
    orc_poly_roots(a, (const double*)c, (double*)z);

    /* Algorithm 1, location check of SynDec.  s_j = ln(z_j) N / (i 2 pi) taken as the member of
     * S_k = {k + tM} nearest to it; the root belongs to U_k only if z_j lies
     * within root_tol of omega^{s_j}. */
    for (int j = 0; j < a; ++j) {
      if (!(cabs(z[j]) > 0) || !isfinite(creal(z[j])) || !isfinite(cimag(z[j]))) return 0;
      double pos = carg(z[j]) / TWO_PI * (double)N; /* real-valued location */
      double tf = nearbyint((pos - (double)k) / (double)M);
      int64_t t = (int64_t)tf % d;
      if (t < 0) t += d;
      s[j] = k + t * M;
      if (!(cabs(z[j] - omega_pow(N, s[j])) <= root_tol)) return 0;
    }
  } else {
    /* a > 4: Berlekamp-Massey locator, and as no closed form gives the
     * roots, the candidate search of Step (ii): |P(omega^{k+tM})| at every
     * t < d, the a smallest kept (ties: smaller t).  They must be roots up
     * to root_tol (1 + sum |c_j|). */
    if (!orc_bm_locator(a, (const double*)m, (double*)c)) return 0;
    double bound = 1;
    for (int j = 0; j < a; ++j) bound += cabs(c[j]);
    bound *= root_tol;
    double bv[8];
    int64_t bt[8];
    int have = 0;
    for (int64_t t = 0; t < d; ++t) {
      cplx z = omega_pow(N, k + t * M), P = 1;
      for (int j = a - 1; j >= 0; --j) P = P * z + c[j];
      const double v = cabs(P);
      if (have < a || v < bv[a - 1]) {
        int pos = have < a ? have : a - 1;
        while (pos > 0 && bv[pos - 1] > v) {
          bv[pos] = bv[pos - 1];
          bt[pos] = bt[pos - 1];
          --pos;
        }
        bv[pos] = v;
        bt[pos] = t;
        if (have < a) ++have;
      }
    }
    if (!(bv[a - 1] <= bound)) return 0;
    for (int j = 0; j < a; ++j) s[j] = k + bt[j] * M;
  }
  /* sort ascending and require distinct locations */
  for (int i = 1; i < a; ++i)
    for (int j = i; j > 0 && s[j - 1] > s[j]; --j) {
      int64_t t = s[j];
      s[j] = s[j - 1];
      s[j - 1] = t;
    }
  for (int j = 1; j < a; ++j)
    if (s[j] == s[j - 1]) return 0;

  /* Step (iii): substitute the z_j = omega^{s_j} into all available
   * equations of Eq. (3), m_i = sum_j p_j z_j^i (i < n_m), and solve them in
   * the least-squares sense through the normal equations (Z^H Z) p = Z^H m. */
  cplx G[64], g[8], p[8];
  for (int u = 0; u < a; ++u) {
    g[u] = 0;
    for (int v = 0; v < a; ++v) G[u * a + v] = 0;
  }
  for (int i = 0; i < n_m; ++i) {
    cplx zi[8];
    for (int j = 0; j < a; ++j) zi[j] = omega_pow(N, s[j] * (int64_t)i);
    for (int u = 0; u < a; ++u) {
      g[u] += conj(zi[u]) * m[i];
      for (int v = 0; v < a; ++v) G[u * a + v] += conj(zi[u]) * zi[v];
    }
  }
  if (!solve_lin(a, G, g, p)) return 0;

  /* Validation: every value non-zero and the equations of Eq. (3) met. */
  double mmax = 0, rmax = 0;
  for (int j = 0; j < a; ++j)
    if (!(cabs(p[j]) > theta)) return 0;
  for (int i = 0; i < n_m; ++i) {
    cplx fit = 0;
    for (int j = 0; j < a; ++j) fit += p[j] * omega_pow(N, s[j] * (int64_t)i);
    mmax = fmax(mmax, cabs(m[i]));
    rmax = fmax(rmax, cabs(m[i] - fit));
  }
  if (!(rmax <= res_tol * mmax)) return 0;

  for (int j = 0; j < a; ++j) {
    s_out[j] = s[j];
    p_out[2 * j] = creal(p[j]);
    p_out[2 * j + 1] = cimag(p[j]);
  }
  return 1;
}

/* ------------------------------------------------------------- transform */

typedef struct {
  int64_t s;
  cplx v;
} entry;

static int cmp_entry(const void* A, const void* B) {
  int64_t a = ((const entry*)A)->s, b = ((const entry*)B)->s;
  return (a > b) - (a < b);
}

static int push(entry** S, int64_t* n, int64_t* capS, int64_t s, cplx v) {
  if (*n == *capS) {
    int64_t nc = *capS ? 2 * *capS : 1024;
    entry* t = (entry*)realloc(*S, (size_t)nc * sizeof(entry));
    if (!t) return 0;
    *S = t;
    *capS = nc;
  }
  (*S)[*n].s = s;
  (*S)[*n].v = v;
  ++*n;
  return 1;
}

int64_t orc_exact(const double* xin, const orc_exact_params* prm, int64_t cap,
                  int64_t* idx, double* val, int64_t* unresolved) {
  const int64_t N = prm->N, M0 = prm->M0;
  const int am = prm->a_max;
  if (!is_pow2(N) || !is_pow2(M0) || M0 > N || am < 1 || am > 8) return -1;
  const int64_t d0 = N / M0;
  const int iters = prm->mode == ORC_ITER ? prm->max_iters : 1;
  if (prm->mode == ORC_ITER && (iters < 1 || iters > am)) return -1;
  if (prm->mode == ORC_ITER && (M0 >> (iters - 1)) < 1) return -1;
  (void)d0; /* shifts >= d wrap circularly: Eq. (2) holds for any shift */

  const int nsh = 2 * am; /* syndromes ever held */
  cplx* held = (cplx*)calloc((size_t)nsh * (size_t)M0, sizeof(cplx));
  unsigned char* T = (unsigned char*)calloc((size_t)M0, 1);
  entry* S = NULL;
  int64_t nS = 0, capS = 0;
  double theta = 0;
  int64_t nT = 0;
  if (!held || !T) {
    free(held);
    free(T);
    return -1;
  }
#define HELD(j, k) held[(size_t)(j) * (size_t)M0 + (size_t)(k)]

  if (prm->mode == ORC_FIXED) {
    /* Non-iterative sFFT-DT (Fig. 1(b)): all 2 a_m syndromes at d0, every
     * active bin decoded once with the smallest a <= a_m that validates. */
    for (int j = 0; j < nsh; ++j) orc_syndrome(xin, N, d0, j, (double*)&HELD(j, 0));
    double ymax = 0;
    for (int64_t k = 0; k < M0; ++k) ymax = fmax(ymax, cabs(HELD(0, k)));
    theta = prm->zero_tol * ymax;
    for (int64_t k = 0; k < M0; ++k) {
      int active = 0;
      cplx m[16];
      for (int j = 0; j < nsh; ++j) {
        m[j] = HELD(j, k);
        if (cabs(m[j]) > theta) active = 1;
      }
      if (!active) continue;
      int ok = 0;
      for (int a = 1; a <= am && !ok; ++a) {
        int64_t s[8];
        cplx p[8];
        if (orc_decode(a, (const double*)m, nsh, k, M0, N, theta, prm->root_tol,
                       prm->res_tol, s, (double*)p)) {
          for (int j = 0; j < a; ++j) push(&S, &nS, &capS, s[j], p[j]);
          ok = 1;
        }
      }
      if (!ok) ++nT;
    }
  } else {
    /* Iterative sFFT-DT, Algorithm 1.  Level l works at d = 2^l d0 with
     * M = M0 / 2^l bins and decodes a = l + 1 aliases from 2l + 2 syndromes.
     * The syndromes of shifts < 2l held from earlier levels are folded,
     * Y_{2d,j}[k] = Y_{d,j}[k] + Y_{d,j}[k + M/2] (reading of Algorithm 1's level step). */
    int64_t M = M0, d = d0;
    for (int l = 0; l < iters; ++l) {
      if (l > 0) {
        /* next level: d = 2d, and T is taken modulo N/d (T holds bins) */
        M >>= 1;
        d <<= 1;
        for (int j = 0; j < 2 * l; ++j)
          for (int64_t k = 0; k < M; ++k) HELD(j, k) += HELD(j, k + M);
        for (int64_t k = 0; k < M; ++k) T[k] = (unsigned char)(T[k] | T[k + M]);
      }
      /* Algorithm 1: the two new shifts 2l, 2l+1 at the current d */
      orc_syndrome(xin, N, d, 2 * l, (double*)&HELD(2 * l, 0));
      orc_syndrome(xin, N, d, 2 * l + 1, (double*)&HELD(2 * l + 1, 0));
      /* SubFreq: remove every frequency solved so far */
      for (int64_t e = 0; e < nS; ++e) {
        int64_t kd = S[e].s % M;
        HELD(2 * l, kd) -= S[e].v * omega_pow(N, S[e].s * (int64_t)(2 * l));
        HELD(2 * l + 1, kd) -= S[e].v * omega_pow(N, S[e].s * (int64_t)(2 * l + 1));
      }
      if (l == 0) {
        double ymax = 0;
        for (int64_t k = 0; k < M; ++k) ymax = fmax(ymax, cabs(HELD(0, k)));
        theta = prm->zero_tol * ymax;
      }
      /* activity test and SynDec of every active bin */
      const int a = l + 1, nm = 2 * l + 2;
      for (int64_t k = 0; k < M; ++k) {
        if (!(T[k] || cabs(HELD(2 * l, k)) > theta || cabs(HELD(2 * l + 1, k)) > theta)) continue;
        cplx m[16];
        for (int j = 0; j < nm; ++j) m[j] = HELD(j, k);
        int64_t s[8];
        cplx p[8];
        if (orc_decode(a, (const double*)m, nm, k, M, N, theta, prm->root_tol, prm->res_tol, s,
                       (double*)p)) {
          /* SynDec success: S = S u s, x^[s_j] = p_j; the solved terms leave
           * every syndrome held for this bin */
          for (int i = 0; i < a; ++i) {
            push(&S, &nS, &capS, s[i], p[i]);
            for (int j = 0; j < nm; ++j) HELD(j, k) -= p[i] * omega_pow(N, s[i] * (int64_t)j);
          }
          T[k] = 0;
        } else {
          T[k] = 1; /* SynDec failure: the bin joins T */
        }
      }
    }
    for (int64_t k = 0; k < M; ++k) nT += T[k];
  }
#undef HELD

  qsort(S, (size_t)nS, sizeof(entry), cmp_entry);
  int64_t nout = nS < cap ? nS : cap;
  for (int64_t e = 0; e < nout; ++e) {
    idx[e] = S[e].s;
    val[2 * e] = creal(S[e].v);
    val[2 * e + 1] = cimag(S[e].v);
  }
  if (unresolved) *unresolved = nT;
  free(S);
  free(held);
  free(T);
  return nS;
}

/* ===================================================================== */
/*            generally K-sparse signals: Sec. III, Algorithm 2           */
/* ===================================================================== */

uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int orc_cs_shifts(uint64_t seed, int64_t d, int r, int64_t* out) {
  if (d < 1 || r < 0 || r > d) return -1;
  int64_t* a = (int64_t*)malloc((size_t)d * sizeof(int64_t));
  if (!a) return -1;
  for (int64_t i = 0; i < d; ++i) a[i] = i;
  for (int i = 0; i < r; ++i) {
    int64_t j = i + (int64_t)(orc_splitmix64(seed, (uint64_t)i) % (uint64_t)(d - i));
    int64_t t = a[i];
    a[i] = a[j];
    a[j] = t;
    out[i] = a[i];
  }
  free(a);
  return 0;
}

/* One-sided Jacobi: rotate pairs of columns of A until every pair is
 * orthogonal; the singular values are then the column norms. */
int orc_hankel_svals(int n, const double* min, double* sv) {
  if (n < 1 || n > 8) return -1;
  const cplx* m = (const cplx*)min;
  cplx A[64];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = m[i + j];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0, beta = 0;
        cplx gamma = 0;
        for (int i = 0; i < n; ++i) {
          alpha += creal(conj(A[i * n + p]) * A[i * n + p]);
          beta += creal(conj(A[i * n + q]) * A[i * n + q]);
          gamma += conj(A[i * n + p]) * A[i * n + q];
        }
        double g = cabs(gamma);
        if (!(g > 0) || !(alpha > 0) || !(beta > 0)) continue;
        off = fmax(off, g / sqrt(alpha * beta));
        if (!(g > 1e-15 * sqrt(alpha * beta))) continue;
        /* make the inner product real: a_q <- e^{-i phi} a_q, then a real
         * rotation with cot(2 theta) = (beta - alpha) / (2 |gamma|) */
        cplx ph = gamma / g;
        double zeta = (beta - alpha) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < n; ++i) {
          cplx ap = A[i * n + p], aq = A[i * n + q] * conj(ph);
          A[i * n + p] = c * ap - s * aq;
          A[i * n + q] = s * ap + c * aq;
        }
      }
    if (off <= 1e-15) break;
  }
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < n; ++i) s2 += creal(conj(A[i * n + j]) * A[i * n + j]);
    sv[j] = sqrt(s2);
  }
  for (int i = 1; i < n; ++i) /* descending */
    for (int j = i; j > 0 && sv[j - 1] < sv[j]; --j) {
      double t = sv[j];
      sv[j] = sv[j - 1];
      sv[j - 1] = t;
    }
  return 0;
}

/* indices of the ks largest values (ties: smaller index first), returned in
 * ascending index order; taken is n bytes of scratch */
static int top_ks(int n, const double* v, const unsigned char* allowed, int ks, int* out,
                  unsigned char* taken) {
  memset(taken, 0, (size_t)n);
  int cnt = 0;
  for (int r = 0; r < ks; ++r) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if ((!allowed || allowed[i]) && !taken[i] && (best < 0 || v[i] > v[best])) best = i;
    if (best < 0) break;
    taken[best] = 1;
    ++cnt;
  }
  int w = 0;
  for (int i = 0; i < n; ++i)
    if (taken[i]) out[w++] = i;
  return cnt;
}

/* least squares on the columns T of Phi (normal equations); fills the
 * coefficients and the residual y - Phi_T x; returns |res|^2 or -1 */
static double ls_on(int rows, int cols, const cplx* Phi, const cplx* y, const int* T, int nT,
                    cplx* x, cplx* res) {
  cplx G[64], g[8];
  for (int u = 0; u < nT; ++u) {
    g[u] = 0;
    for (int v = 0; v < nT; ++v) G[u * nT + v] = 0;
    for (int i = 0; i < rows; ++i) {
      g[u] += conj(Phi[i * cols + T[u]]) * y[i];
      for (int v = 0; v < nT; ++v) G[u * nT + v] += conj(Phi[i * cols + T[u]]) * Phi[i * cols + T[v]];
    }
  }
  if (!solve_lin(nT, G, g, x)) return -1;
  double rn = 0;
  for (int i = 0; i < rows; ++i) {
    cplx f = 0;
    for (int u = 0; u < nT; ++u) f += Phi[i * cols + T[u]] * x[u];
    res[i] = y[i] - f;
    rn += creal(conj(res[i]) * res[i]);
  }
  return rn;
}

int orc_subspace_pursuit(int rows, int cols, const double* Phin, const double* yn, int ks,
                         int iters, double* bout) {
  const cplx* Phi = (const cplx*)Phin;
  const cplx* y = (const cplx*)yn;
  cplx* b = (cplx*)bout;
  if (rows < 1 || rows > 32 || cols < 1 || cols > (1 << 16) || ks > 4) return -1;
  for (int j = 0; j < cols; ++j) b[j] = 0;
  if (ks > cols) ks = cols;
  if (ks <= 0) return 0;
  /* per-column scratch: correlations / magnitudes, membership flags */
  double* corr = (double*)malloc((size_t)cols * sizeof(double));
  unsigned char* flags = (unsigned char*)malloc((size_t)cols * 3);
  if (!corr || !flags) {
    free(corr);
    free(flags);
    return -1;
  }
  unsigned char *taken = flags, *in2 = flags + cols, *allow = flags + 2 * cols;
  cplx res[32], x[8], xn[8], resn[32];
  int T[8], nT;
  /* initialisation: the ks columns most correlated with y */
  for (int j = 0; j < cols; ++j) {
    cplx c = 0;
    for (int i = 0; i < rows; ++i) c += conj(Phi[(size_t)i * cols + j]) * y[i];
    corr[j] = cabs(c);
  }
  nT = top_ks(cols, corr, NULL, ks, T, taken);
  double rn = ls_on(rows, cols, Phi, y, T, nT, x, res);
  if (rn < 0) {
    free(corr);
    free(flags);
    return -1;
  }
  for (int it = 0; it < iters; ++it) {
    /* expand by the ks columns most correlated with the residual */
    for (int j = 0; j < cols; ++j) {
      cplx c = 0;
      for (int i = 0; i < rows; ++i) c += conj(Phi[(size_t)i * cols + j]) * res[i];
      corr[j] = cabs(c);
    }
    int add[8];
    int na = top_ks(cols, corr, NULL, ks, add, taken);
    memset(in2, 0, (size_t)cols);
    for (int u = 0; u < nT; ++u) in2[T[u]] = 1;
    for (int u = 0; u < na; ++u) in2[add[u]] = 1;
    int T2[16], n2 = 0;
    for (int j = 0; j < cols; ++j)
      if (in2[j]) T2[n2++] = j;
    /* least squares on the union, keep the ks largest coefficients */
    cplx x2[16], r2[32];
    if (ls_on(rows, cols, Phi, y, T2, n2, x2, r2) < 0) break;
    memset(allow, 0, (size_t)cols);
    for (int u = 0; u < n2; ++u) {
      corr[T2[u]] = cabs(x2[u]);
      allow[T2[u]] = 1;
    }
    int Tn[8];
    int nn = top_ks(cols, corr, allow, ks, Tn, taken);
    double rnn = ls_on(rows, cols, Phi, y, Tn, nn, xn, resn);
    if (rnn < 0 || rnn >= rn) break; /* no improvement: keep the previous support */
    nT = nn;
    for (int u = 0; u < nT; ++u) {
      T[u] = Tn[u];
      x[u] = xn[u];
    }
    for (int i = 0; i < rows; ++i) res[i] = resn[i];
    rn = rnn;
  }
  for (int u = 0; u < nT; ++u) b[T[u]] = x[u];
  free(corr);
  free(flags);
  return nT;
}

typedef struct {
  double v;
  int64_t i;
} keyed;

static int cmp_desc(const void* A, const void* B) {
  const keyed* a = (const keyed*)A;
  const keyed* b = (const keyed*)B;
  if (a->v > b->v) return -1;
  if (a->v < b->v) return 1;
  return (a->i > b->i) - (a->i < b->i);
}

int64_t orc_general(const double* xin, const orc_general_params* p, int64_t cap, int64_t* idx,
                    double* val, unsigned char* a_k_out) {
  const int64_t N = p->N, M = p->M, K = p->K;
  const int am = p->a_max, r = p->r;
  if (!is_pow2(N) || !is_pow2(M) || M > N || am < 1 || am > 4 || r < 1 || r > 32 ||
      p->keep < 1 || K < 0)
    return -1;
  const int64_t d = N / M;
  if (r > d || (!p->prune && d > (1 << 16))) return -1;
  int64_t ns[32];
  if (orc_cs_shifts(p->seed, d, r, ns) != 0) return -1;
  const int nc = 2 * am;
  cplx* Yc = (cplx*)malloc((size_t)nc * (size_t)M * sizeof(cplx));
  cplx* Ys = (cplx*)malloc((size_t)r * (size_t)M * sizeof(cplx));
  keyed* sv = (keyed*)malloc((size_t)M * (size_t)am * sizeof(keyed));
  unsigned char* ak = (unsigned char*)calloc((size_t)M, 1);
  entry* S = NULL;
  int64_t nS = 0, capS = 0;
  if (!Yc || !Ys || !sv || !ak) {
    free(Yc);
    free(Ys);
    free(sv);
    free(ak);
    return -1;
  }
  /* Algorithm 2, Part 1: consecutive shifts 0..2a_m-1 and the r random
   * shifts, each d * FFT_M */
  if (p->prune)
    for (int j = 0; j < nc; ++j) orc_syndrome(xin, N, d, j, (double*)&Yc[(size_t)j * M]);
  for (int l = 0; l < r; ++l) orc_syndrome(xin, N, d, ns[l], (double*)&Ys[(size_t)l * M]);
  if (!p->prune) {
    /* Sec. III-B without the pruning strategy: every bin's CS model
     * y = Phi b over all d candidates (Eq. (18)), solved by SP at sparsity
     * a_m; every non-zero coefficient is output */
    cplx* Phi = (cplx*)malloc((size_t)r * (size_t)d * sizeof(cplx));
    cplx* b = (cplx*)malloc((size_t)d * sizeof(cplx));
    int ok = Phi && b;
    for (int64_t k = 0; ok && k < M; ++k) {
      cplx y[32];
      for (int j = 0; j < r; ++j) {
        y[j] = Ys[(size_t)j * M + k];
        for (int64_t t = 0; t < d; ++t) Phi[(size_t)j * d + t] = omega_pow(N, (k + t * M) * ns[j]);
      }
      /* a singular first least-squares problem leaves the bin empty */
      int nz = orc_subspace_pursuit(r, (int)d, (const double*)Phi, (const double*)y, am,
                                    p->sp_iters, (double*)b);
      for (int64_t t = 0; nz > 0 && t < d; ++t)
        if (b[t] != 0) push(&S, &nS, &capS, k + t * M, b[t]);
      ak[k] = (unsigned char)am;
    }
    free(Phi);
    free(b);
    if (!ok) {
      free(S);
      free(Yc);
      free(Ys);
      free(sv);
      free(ak);
      return -1;
    }
    goto output;
  }
  /* Algorithm 2, Part 2: singular values of every bin's a_m x a_m Hankel
   * matrix (m_0 .. m_{2a_m-2}, Eq. (26)); the K largest vote */
  for (int64_t k = 0; k < M; ++k) {
    cplx m[8];
    double s[4];
    for (int j = 0; j < 2 * am - 1; ++j) m[j] = Yc[(size_t)j * M + k];
    orc_hankel_svals(am, (const double*)m, s);
    for (int i = 0; i < am; ++i) {
      sv[k * am + i].v = s[i];
      sv[k * am + i].i = k * am + i;
    }
  }
  qsort(sv, (size_t)(M * am), sizeof(keyed), cmp_desc);
  const int64_t nvote = K < M * am ? K : M * am;
  for (int64_t e = 0; e < nvote; ++e) ak[sv[e].i / am] += 1;
  /* Algorithm 2, Parts 3-4: pruning Steps 2-3 and Subspace Pursuit */
  for (int64_t k = 0; k < M; ++k) {
    const int a = ak[k];
    if (a == 0) continue;
    cplx m[8];
    for (int j = 0; j < 2 * a; ++j) m[j] = Yc[(size_t)j * M + k];
    /* (a): the a x a Hankel system with the observed syndromes */
    cplx H[16], rhs[4], c[4];
    for (int i = 0; i < a; ++i) {
      for (int j = 0; j < a; ++j) H[i * a + j] = m[i + j];
      rhs[i] = -m[a + i];
    }
    if (!solve_lin(a, H, rhs, c)) continue;
    /* (b)-(c): |P~(z)| at every candidate z = omega^{k + tM} of U_k; keep
     * the min(d, keep * a) smallest (ties: smaller t) */
    int64_t nkeep = (int64_t)p->keep * a < d ? (int64_t)p->keep * a : d;
    if (nkeep > 32) nkeep = 32;
    double* pv = (double*)malloc((size_t)d * sizeof(double));
    unsigned char* tk = (unsigned char*)calloc((size_t)d, 1);
    /* P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0 by Horner */
    for (int64_t t = 0; t < d; ++t) {
      cplx z = omega_pow(N, k + t * M), P = 1;
      for (int j = a - 1; j >= 0; --j) P = P * z + c[j];
      pv[t] = cabs(P);
    }
    int64_t kept[32];
    int nk = 0;
    for (int64_t rr = 0; rr < nkeep; ++rr) {
      int64_t best = -1;
      for (int64_t t = 0; t < d; ++t)
        if (!tk[t] && (best < 0 || pv[t] < pv[best])) best = t;
      tk[best] = 1;
    }
    for (int64_t t = 0; t < d; ++t)
      if (tk[t]) kept[nk++] = t;
    free(pv);
    free(tk);
    /* Step 3: Phi_p[j][u] = omega^{(k + kept_u M) n_j}, y_j = Y_{n_j}[k] */
    cplx Phi[32 * 32], y[32], b[32];
    for (int j = 0; j < r; ++j) {
      y[j] = Ys[(size_t)j * M + k];
      for (int u = 0; u < nk; ++u) Phi[j * nk + u] = omega_pow(N, (k + kept[u] * M) * ns[j]);
    }
    int nz = orc_subspace_pursuit(r, nk, (const double*)Phi, (const double*)y, a, p->sp_iters,
                                  (double*)b);
    if (nz <= 0) continue;
    for (int u = 0; u < nk; ++u)
      if (b[u] != 0) push(&S, &nS, &capS, k + kept[u] * M, b[u]);
  }
output:
  qsort(S, (size_t)nS, sizeof(entry), cmp_entry);
  const int64_t nout = nS < cap ? nS : cap;
  for (int64_t e = 0; e < nout; ++e) {
    idx[e] = S[e].s;
    val[2 * e] = creal(S[e].v);
    val[2 * e + 1] = cimag(S[e].v);
  }
  if (a_k_out) memcpy(a_k_out, ak, (size_t)M);
  free(S);
  free(Yc);
  free(Ys);
  free(sv);
  free(ak);
  return nS;
}
