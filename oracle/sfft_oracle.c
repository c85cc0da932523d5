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

/* Eq. (2) with R1: Y_{d,l} = d * FFT_M(x_{d,l}),  x_{d,l}[n] = x[n d + l]. */
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

int orc_decode(int a, const double* min, int n_m, int64_t k, int64_t M, int64_t N,
               double theta, double root_tol, double res_tol,
               int64_t* s_out, double* p_out) {
  if (a < 1 || a > 4 || n_m < 2 * a || M <= 0 || N % M != 0) return 0;
  const cplx* m = (const cplx*)min;
  int64_t d = N / M;

  /* Step (i), Eq. (4)-(5): the a x a Hankel system
   *   sum_j c_j m_{i+j} = -m_{a+i},  i = 0..a-1. */
  cplx H[16], rhs[4], c[4];
  for (int i = 0; i < a; ++i) {
    for (int j = 0; j < a; ++j) H[i * a + j] = m[i + j];
    rhs[i] = -m[a + i];
  }
  if (!solve_lin(a, H, rhs, c)) return 0;

  /* Step (ii): the roots z_j of P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0. */
  cplx z[4];
  orc_poly_roots(a, (const double*)c, (double*)z);

  /* Alg. 1 lines 29-30.  s_j = ln(z_j) N / (i 2 pi) taken as the member of
   * S_k = {k + tM} nearest to it; the root belongs to U_k only if z_j lies
   * within root_tol of omega^{s_j}. */
  int64_t s[4];
  for (int j = 0; j < a; ++j) {
    if (!(cabs(z[j]) > 0) || !isfinite(creal(z[j])) || !isfinite(cimag(z[j]))) return 0;
    double pos = carg(z[j]) / TWO_PI * (double)N; /* real-valued location */
    double tf = nearbyint((pos - (double)k) / (double)M);
    int64_t t = (int64_t)tf % d;
    if (t < 0) t += d;
    s[j] = k + t * M;
    if (!(cabs(z[j] - omega_pow(N, s[j])) <= root_tol)) return 0;
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
  cplx G[16], g[4], p[4];
  for (int u = 0; u < a; ++u) {
    g[u] = 0;
    for (int v = 0; v < a; ++v) G[u * a + v] = 0;
  }
  for (int i = 0; i < n_m; ++i) {
    cplx zi[4];
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
  if (!is_pow2(N) || !is_pow2(M0) || M0 > N || am < 1 || am > 4) return -1;
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
      cplx m[8];
      for (int j = 0; j < nsh; ++j) {
        m[j] = HELD(j, k);
        if (cabs(m[j]) > theta) active = 1;
      }
      if (!active) continue;
      int ok = 0;
      for (int a = 1; a <= am && !ok; ++a) {
        int64_t s[4];
        cplx p[4];
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
     * Y_{2d,j}[k] = Y_{d,j}[k] + Y_{d,j}[k + M/2] (reading of line 10). */
    int64_t M = M0, d = d0;
    for (int l = 0; l < iters; ++l) {
      if (l > 0) {
        /* line 14: d = 2d; line 15: T taken modulo N/d (T holds bins) */
        M >>= 1;
        d <<= 1;
        for (int j = 0; j < 2 * l; ++j)
          for (int64_t k = 0; k < M; ++k) HELD(j, k) += HELD(j, k + M);
        for (int64_t k = 0; k < M; ++k) T[k] = (unsigned char)(T[k] | T[k + M]);
      }
      /* lines 03-06: the two new shifts 2l, 2l+1 at the current d */
      orc_syndrome(xin, N, d, 2 * l, (double*)&HELD(2 * l, 0));
      orc_syndrome(xin, N, d, 2 * l + 1, (double*)&HELD(2 * l + 1, 0));
      /* line 07, SubFreq (lines 17-22): remove every frequency solved so far */
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
      /* lines 08-13 */
      const int a = l + 1, nm = 2 * l + 2;
      for (int64_t k = 0; k < M; ++k) {
        if (!(T[k] || cabs(HELD(2 * l, k)) > theta || cabs(HELD(2 * l + 1, k)) > theta)) continue;
        cplx m[8];
        for (int j = 0; j < nm; ++j) m[j] = HELD(j, k);
        int64_t s[4];
        cplx p[4];
        if (orc_decode(a, (const double*)m, nm, k, M, N, theta, prm->root_tol, prm->res_tol, s,
                       (double*)p)) {
          /* lines 31-32: S = S u s, x^[s_j] = p_j; the solved terms leave
           * every syndrome held for this bin */
          for (int i = 0; i < a; ++i) {
            push(&S, &nS, &capS, s[i], p[i]);
            for (int j = 0; j < nm; ++j) HELD(j, k) -= p[i] * omega_pow(N, s[i] * (int64_t)j);
          }
          T[k] = 0;
        } else {
          T[k] = 1; /* line 34 */
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
