// sft_decode.cuh -- per-bin syndrome decoding in FP64 (Sec. II-B, the SynDec
// function of Algorithm 1), one thread per (active) bin.
//
// Given n_m >= 2a syndromes m_i = sum_j p_j z_j^i of bin k (Eq. (3)):
//  (i)   solve the a x a Hankel system sum_j c_j m_{i+j} = -m_{a+i}
//        (Eq. (4)-(5)) by Gaussian elimination with partial pivoting;
//  (ii)  take the roots of P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0 by the
//        analytical solutions for a <= 4 (quadratic, Cardano, Ferrari);
//        each root gives the location s_j = ln(z_j) N / (i 2 pi), taken as
//        the member k + tM of S_k nearest to it (location check of SynDec, Algorithm 1);
//  (iii) solve all n_m equations of Eq. (3) for the values p_j in the least
//        squares sense (normal equations).
// Accept iff every root lies within root_tol of omega^{s_j}, the s_j are
// distinct, every |p_j| > theta and ||m - Z p||_inf <= res_tol ||m||_inf.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the FP64
// work per bin is kept lean: magnitudes are compared squared (no hypot),
// complex quotients use one reciprocal, the candidate index of a root comes
// from an FP32 angle unless that angle lies near the midpoint of two
// candidates (then the FP64 formula decides, as in the oracle), and cube
// roots are an FP32 estimate polished by FP64 Newton steps (any cube root
// gives the same three roots of the cubic).
#pragma once

#include "sft_common.cuh"

namespace sft {

// Squared magnitudes (non-negative doubles) order like their bit patterns
// as integers, NaN above +inf: their maxima and comparisons run on the
// integer pipes instead of occupying GB300's scarce FP64 unit.
__device__ __forceinline__ long long ordbits(double v) { return __double_as_longlong(v); }
// z == 0 (either sign of zero in both parts), on the bit patterns
__device__ __forceinline__ bool is_zero_c(cdbl z) {
  return ((__double_as_longlong(z.x) | __double_as_longlong(z.y)) << 1) == 0;
}

// 1/x: an FP32 seed refined by two Newton steps r <- r + r (1 - x r) (each
// doubles the correct bits: ~2^-22 -> 2^-44 -> below an FP64 ulp); an
// exact FP64 division when |x| lies outside [2^-123, 2^124).  The seed's
// operand is x truncated to float and its result widened back, both by
// moving bits (sign, exponent rebiased by 896, top 23 significand bits) on
// the integer pipes: a conversion instruction, like the range test on a
// double, would occupy GB300's scarce FP64 unit.
__device__ __forceinline__ double rcp_d(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t ex = (uint32_t)(u >> 52) & 0x7FFu;
  if (ex < 900u || ex >= 1147u) return 1.0 / x;
  const uint32_t fb = ((uint32_t)(u >> 63) << 31) | ((ex - 896u) << 23) |
                      (uint32_t)((u >> 29) & 0x7FFFFFu);
  double r = f2d_exact(__frcp_rn(__uint_as_float(fb)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ cdbl crcp(cdbl b) {
  const double inv = rcp_d(norm2(b));
  return cdbl{b.x * inv, -b.y * inv};
}
__device__ __forceinline__ cdbl csqrt_fast(cdbl v) {
  const double r = sqrt(norm2(v));
  if (r == 0.0) return cdbl{0.0, 0.0};
  if (v.x >= 0.0) {
    const double t = sqrt(0.5 * (r + v.x));
    return cdbl{t, v.y * (0.5 * rcp_d(t))};
  }
  const double t = sqrt(0.5 * (r - v.x));
  return cdbl{fabs(v.y) * (0.5 * rcp_d(t)), copysign(t, v.y)};
}
// a cube root of v: FP32 polar estimate (relative error ~1e-6), one FP64
// Newton step u <- (2u + v / u^2) / 3 (quadratic: ~1e-12).  The roots it
// yields only choose candidates (an angle against margins of 1e-3 of a
// candidate spacing) and pass the 0.1 root tolerance; the values come from
// the candidates themselves.
__device__ __forceinline__ cdbl ccbrt_any(cdbl v) {
  if (is_zero_c(v)) return cdbl{0.0, 0.0};
  const float rf = cbrtf((float)sqrt(norm2(v)));
  const float th = atan2f((float)v.y, (float)v.x) * (1.0f / 3.0f);
  float sf, cf;
  sincosf(th, &sf, &cf);
  cdbl u{(double)(rf * cf), (double)(rf * sf)};
  const cdbl u2 = u * u;
  u = (u * 2.0 + v * crcp(u2)) * (1.0 / 3.0);
  return u;
}

// Gaussian elimination with partial pivoting on an n x n system (n <= 4).
// A is row-major and destroyed.  Fails on a pivot below 1e-14 of max |A|.
template <int n>
__device__ __forceinline__ bool solve_small(cdbl* A, cdbl* b, cdbl* x) {
  long long amax_b = 0;
#pragma unroll
  for (int i = 0; i < n * n; ++i) amax_b = max(amax_b, ordbits(norm2(A[i])));
  const double amax2 = __longlong_as_double(amax_b);
  if (!(amax2 > 0.0)) return false;
  cdbl inv[n];
#pragma unroll
  for (int col = 0; col < n; ++col) {
    int piv = col;
    long long best_b = ordbits(norm2(A[col * n + col]));
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      const long long v = ordbits(norm2(A[r * n + col]));
      if (v > best_b) {
        best_b = v;
        piv = r;
      }
    }
    const double best = __longlong_as_double(best_b);
    if (!(best > 1e-28 * amax2)) return false;
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      if (r == piv) {
#pragma unroll
        for (int c = 0; c < n; ++c) {
          const cdbl t = A[col * n + c];
          A[col * n + c] = A[r * n + c];
          A[r * n + c] = t;
        }
        const cdbl t = b[col];
        b[col] = b[r];
        b[r] = t;
      }
    }
    // 1 / pivot = conj(pivot) / |pivot|^2, |pivot|^2 being `best`
    inv[col] = conjd(A[col * n + col]) * rcp_d(best);
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      const cdbl f = A[r * n + col] * inv[col];
#pragma unroll
      for (int c = col + 1; c < n; ++c) A[r * n + c] = A[r * n + c] - f * A[col * n + c];
      b[r] = b[r] - f * b[col];
    }
  }
#pragma unroll
  for (int r = n - 1; r >= 0; --r) {
    cdbl acc = b[r];
#pragma unroll
    for (int c = r + 1; c < n; ++c) acc = acc - A[r * n + c] * x[c];
    x[r] = acc * inv[r];
  }
  return true;
}

// z^2 + b z + c = 0 in the cancellation-free form q = -(b + sgn sqrt(D))/2,
// roots q and c/q.
__device__ __forceinline__ void quad_roots(cdbl b, cdbl c, cdbl* z) {
  const cdbl sq = csqrt_fast(b * b - c * 4.0);
  const cdbl qp = b + sq, qm = b - sq;
  const cdbl q = (ordbits(norm2(qp)) >= ordbits(norm2(qm)) ? qp : qm) * -0.5;
  if (is_zero_c(q)) {
    z[0] = z[1] = mk(0.0, 0.0);
    return;
  }
  z[0] = q;
  z[1] = c * crcp(q);
}

// z^3 + c2 z^2 + c1 z + c0 = 0: shift z = y - c2/3 to y^3 + p y + q = 0;
// y = u + v, u^3 = -q/2 +- sqrt((q/2)^2 + (p/3)^3) (the larger), u v = -p/3,
// u over its three cube-root branches.
__device__ __forceinline__ void cubic_roots(cdbl c2, cdbl c1, cdbl c0, cdbl* z) {
  const cdbl sh = c2 * (1.0 / 3.0);
  const cdbl p = c1 - c2 * c2 * (1.0 / 3.0);
  const cdbl q = c2 * c2 * c2 * (2.0 / 27.0) - c2 * c1 * (1.0 / 3.0) + c0;
  const cdbl sD = csqrt_fast(q * q * 0.25 + p * p * p * (1.0 / 27.0));
  const cdbl w1 = q * -0.5 + sD, w2 = q * -0.5 - sD;
  const cdbl u = ccbrt_any(ordbits(norm2(w1)) >= ordbits(norm2(w2)) ? w1 : w2);
  const cdbl br[3] = {mk(1.0, 0.0), mk(-0.5, 0.86602540378443864676),
                      mk(-0.5, -0.86602540378443864676)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const cdbl uj = u * br[j];
    const cdbl vj = is_zero_c(uj) ? mk(0.0, 0.0) : (-p) * crcp(uj * 3.0);
    z[j] = uj + vj - sh;
  }
}

// z^4 + c3 z^3 + c2 z^2 + c1 z + c0 = 0: shift z = y - c3/4 to
// y^4 + p y^2 + q y + r; m = largest root of 8m^3 + 8p m^2 + (2p^2 - 8r) m - q^2;
// with s^2 = 2m the quartic splits into y^2 -+ s y + p/2 + m +- q/(2s).
__device__ __forceinline__ void quartic_roots(cdbl c3, cdbl c2, cdbl c1, cdbl c0, cdbl* z) {
  const cdbl sh = c3 * 0.25;
  const cdbl c3s = c3 * c3;
  const cdbl p = c2 - c3s * (3.0 / 8.0);
  const cdbl q = c3s * c3 * (1.0 / 8.0) - c3 * c2 * 0.5 + c1;
  const cdbl r = c3s * c3s * (-3.0 / 256.0) + c3s * c2 * (1.0 / 16.0) - c3 * c1 * 0.25 + c0;
  cdbl mr[3];
  cubic_roots(p, (p * p * 2.0 - r * 8.0) * (1.0 / 8.0), q * q * (-1.0 / 8.0), mr);
  int best = 0;
  if (ordbits(norm2(mr[1])) > ordbits(norm2(mr[best]))) best = 1;
  if (ordbits(norm2(mr[2])) > ordbits(norm2(mr[best]))) best = 2;
  const cdbl m = mr[best];
  cdbl y[4];
  if (is_zero_c(m)) {
    cdbl w[2];
    quad_roots(p, r, w);
    y[0] = csqrt_fast(w[0]);
    y[1] = -y[0];
    y[2] = csqrt_fast(w[1]);
    y[3] = -y[2];
  } else {
    const cdbl s = csqrt_fast(m * 2.0);
    const cdbl qs = q * crcp(s * 2.0);
    quad_roots(-s, p * 0.5 + m + qs, y);
    quad_roots(s, p * 0.5 + m - qs, y + 2);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = y[j] - sh;
}

struct BinGeom {
  int64_t N, M, d;  // signal length, bins at this level, N / M
  OmegaTab om;
};

// k / M in FP32 for a power of two M (< 2^30) and 0 <= k < M: k times the
// exact reciprocal 2^-log2(M), formed from the exponent bits -- the same
// value as the FP32 quotient, without a division
__device__ __forceinline__ float k_over_M(int64_t k, int64_t M) {
  return (float)(int)k * __int_as_float((127 - (__ffsll(M) - 1)) << 23);
}
// the candidate index t in [0, d) from its rounded value (d a power of two,
// so the mask is the modulo for negative values too)
__device__ __forceinline__ int64_t cand_of(int t, int64_t d) { return (int64_t)(t & (int)(d - 1)); }

// Thresholds, squared: theta^2, root_tol^2, res_tol^2.
struct Tol2 {
  double theta2, root2, res2;
};
// The same thresholds rounded to float, for the float-float decoders (their
// decisions keep margins far wider than the rounding).
struct Tol2f {
  float theta2, root2, res2;
};

// Location of root z: the member k + tM of S_k nearest to it, i.e.
// t = round((arg(z) N / (2 pi) - k) / M) mod d.  The FP32 estimate is exact
// unless it falls within its error bound of a midpoint; then the oracle's
// FP64 formula decides.
__device__ __forceinline__ int64_t snap_root(cdbl z, int64_t k, const BinGeom& g) {
  const float inv2pi = 0.15915494309189533577f;
  const float ang = atan2f((float)z.y, (float)z.x);
  const float df = (float)(int)g.d;
  const float q = fmaf(ang, df * inv2pi, -k_over_M(k, g.M));
  const float fr = q - rintf(q);
  const float margin = fmaxf(1e-3f, 8e-7f * df);
  int t;
  if (fabsf(fabsf(fr) - 0.5f) < margin) {
    const double pos = atan2(z.y, z.x) * 0.15915494309189533577 * (double)g.N;
    t = (int)rint((pos - (double)k) / (double)g.M);
  } else {
    t = __float2int_rn(q);
  }
  return k + cand_of(t, g.d) * g.M;
}

// snap_root for a root given in FP32 (z = m1 / m0 rounded): the FP64 root
// is formed only when the FP32 angle lies near a candidate midpoint.
__device__ __forceinline__ int64_t snap_root_f(float zx, float zy, int64_t k, const BinGeom& g,
                                               cdbl m0, cdbl m1) {
  const float inv2pi = 0.15915494309189533577f;
  const float ang = atan2f(zy, zx);
  const float df = (float)(int)g.d;
  const float q = fmaf(ang, df * inv2pi, -k_over_M(k, g.M));
  const float fr = q - rintf(q);
  const float margin = fmaxf(1e-3f, 8e-7f * df);
  if (fabsf(fabsf(fr) - 0.5f) < margin) return snap_root(m1 * crcp(m0), k, g);
  return k + cand_of(__float2int_rn(q), g.d) * g.M;
}

// Validation (iii) in float-float on the FP32 pipes (mixed path): the
// residual r_i = m_i - sum_j p_j omega^{s_j i} over all nm equations from the
// float-float syndromes `raw`, the values p rounded to float-float and the
// float-float omega tables.  Its error (~1e-13 |m|) is far below res_tol, so
// it accepts exactly the bins the FP64 residual accepts.  Returns -1 when the
// squared magnitudes leave the float range (the caller then uses FP64),
// else whether max |r_i|^2 <= res_tol^2 max |m_i|^2; on acceptance writes
// the residual to res_out (if not null).
template <int a, int nm>
__device__ __forceinline__ int ff_residual_ok(const float4* raw, const int64_t* s, const cdbl* p,
                                              const OmegaTabFF& omff, double res2, float4* res_out) {
  FF::V pf[a], wf[a], wp[a];
#pragma unroll
  for (int j = 0; j < a; ++j) {
    pf[j] = FF::from4(Store<FF>::from_d(p[j]));
    wf[j] = omega_ff(omff, s[j]);
    wp[j] = FF::V{1.0f, 0.0f, 0.0f, 0.0f};
  }
  float mmax2 = 0.0f, rmax2 = 0.0f;
  FF::V r[nm];
#pragma unroll
  for (int i = 0; i < nm; ++i) {
    const FF::V mi = FF::from4(raw[i]);
    FF::V fit = FF::mulv(pf[0], wp[0]);
#pragma unroll
    for (int j = 1; j < a; ++j) fit = FF::add(fit, FF::mulv(pf[j], wp[j]));
    r[i] = FF::sub(mi, fit);
    if (i + 1 < nm) {
#pragma unroll
      for (int j = 0; j < a; ++j) wp[j] = FF::mulv(wp[j], wf[j]);
    }
    // magnitudes from hi + lo: after the cancellation in r the pair is not
    // normalised (its hi part alone can overstate it by many ulps)
    const float mx = __fadd_rn(mi.rh, mi.rl), my = __fadd_rn(mi.ih, mi.il);
    const float rx = __fadd_rn(r[i].rh, r[i].rl), ry = __fadd_rn(r[i].ih, r[i].il);
    mmax2 = fmaxf(mmax2, mx * mx + my * my);
    rmax2 = fmaxf(rmax2, rx * rx + ry * ry);
  }
  if (!(mmax2 < 1e36f) || !(rmax2 < 1e36f)) return -1;
  if (!(f2d_exact(rmax2) <= res2 * f2d_exact(mmax2))) return 0;
  if (res_out != nullptr) {
#pragma unroll
    for (int i = 0; i < nm; ++i) res_out[i] = FF::to4(r[i]);
  }
  return 1;
}

// The one-alias decode of the mixed path entirely in float-float on the
// FP32 pipes, from the syndromes `raw` (Sec. II-A: z = m_1 / m_0, snapped to
// S_k; p = (1/nm) sum_i conj(w^i) m_i; the residual test).  It takes the
// FP64 decoder's decisions: every FP32 quantity that decides is formed as
// the FP64 decoder forms it (the float rounding of the float-float value is
// the float rounding of its FP64 value), and wherever a float-float result
// lies within its error bound of a threshold (a candidate midpoint, the
// root_tol bound, theta, the residual bound) or leaves the float range it
// returns -1 and the caller runs the FP64 decoder.  Returns 1 on success
// (s, the value p_ff and the residual res_out filled), 0 on failure.
__device__ __forceinline__ float ff_re(const FF::V& v) { return __fadd_rn(v.rh, v.rl); }
__device__ __forceinline__ float ff_im(const FF::V& v) { return __fadd_rn(v.ih, v.il); }
__device__ __forceinline__ float ff_norm(const FF::V& v) {
  const float x = ff_re(v), y = ff_im(v);
  return x * x + y * y;
}
// x <= lim decided in FP32 unless within 1e-5 of lim (relative): -1 there.
// x carries FP32 rounding of its FP64 counterpart and lim is rounded once
// to float, both ~1e-7 relative, far inside the 1e-5 margin, so outside it
// the decision is the FP64 one.  One conversion is the only FP64-pipe
// instruction.
__device__ __forceinline__ int ff_le_f(float x, float lf) {
  if (!(x < 1e36f) || !(lf < 1e36f)) return -1;
  if (fabsf(x - lf) <= 1e-5f * lf) return -1;
  return x <= lf ? 1 : 0;
}
__device__ __forceinline__ int ff_le(float x, double lim) { return ff_le_f(x, (float)lim); }

template <int nm>
__device__ __forceinline__ int decode_a1_ff(const float4* raw, int64_t k, const BinGeom& g,
                                            const Tol2f& tol, const OmegaTabFF& omff, int64_t* s,
                                            float4* p_ff, float4* res_out) {
  const FF::V m0 = FF::from4(raw[0]), m1 = FF::from4(raw[1]);
  const float m0x = ff_re(m0), m0y = ff_im(m0), m1x = ff_re(m1), m1y = ff_im(m1);
  if (m0x == 0.0f && m0y == 0.0f) return 0;
  const float den = m0x * m0x + m0y * m0y;
  if (!(den > 1e-30f && den < 1e30f)) return -1;
  const float inv = __frcp_rn(den);
  const float zx = (m1x * m0x + m1y * m0y) * inv, zy = (m1y * m0x - m1x * m0y) * inv;
  if (zx == 0.0f && zy == 0.0f) return 0;
  // the nearest candidate from the FP32 angle (as snap_root_f)
  const float ang = atan2f(zy, zx);
  const float df = (float)(int)g.d;
  const float q = fmaf(ang, df * 0.15915494309189533577f, -k_over_M(k, g.M));
  const float fr = q - rintf(q);
  if (fabsf(fabsf(fr) - 0.5f) < fmaxf(1e-3f, 8e-7f * df)) return -1;
  s[0] = k + cand_of(__float2int_rn(q), g.d) * g.M;
  const FF::V w = omega_ff(omff, s[0]);
  const float dx = zx - ff_re(w), dy = zy - ff_im(w);
  const float dz = dx * dx + dy * dy, r2 = tol.root2;
  if (fabsf(dz - r2) <= 1e-4f * r2) return -1;
  if (!(dz <= r2)) return 0;
  // least squares over the nm equations: p = (1/nm) sum_i conj(w^i) m_i
  FF::V acc = m0, wp = w;
#pragma unroll
  for (int i = 1; i < nm; ++i) {
    const FF::V mi = FF::from4(raw[i]);
    acc = FF::add(acc, FF::mul4(mi, wp.rh, wp.rl, -wp.ih, -wp.il));
    if (i + 1 < nm) wp = FF::mulv(wp, w);
  }
  constexpr float inv_nm = 1.0f / (float)nm;  // a power of two: exact
  const FF::V p{acc.rh * inv_nm, acc.rl * inv_nm, acc.ih * inv_nm, acc.il * inv_nm};
  const int small = ff_le_f(ff_norm(p), tol.theta2);
  if (small != 0) return small < 0 ? -1 : 0;
  // residual r_i = m_i - p w^i over all equations
  float mmax2 = 0.0f, rmax2 = 0.0f;
  FF::V r[nm];
  FF::V pw = p;
#pragma unroll
  for (int i = 0; i < nm; ++i) {
    const FF::V mi = FF::from4(raw[i]);
    r[i] = FF::sub(mi, pw);
    if (i + 1 < nm) pw = FF::mulv(pw, w);
    mmax2 = fmaxf(mmax2, ff_norm(mi));
    rmax2 = fmaxf(rmax2, ff_norm(r[i]));
  }
  const int fits = ff_le_f(rmax2, tol.res2 * mmax2);
  if (fits <= 0) return fits;
  *p_ff = FF::to4(p);
#pragma unroll
  for (int i = 0; i < nm; ++i) res_out[i] = FF::to4(r[i]);
  return 1;
}

// ----------------------------------------------- float-float arithmetic
// Real float-float numbers (h + l, |l| <= ulp(h)/2) and the complex
// operations the two-alias decoder needs, on the FP32 pipes: products by
// FMA-based TwoProd, quotients and square roots by one float-float
// correction of the correctly rounded FP32 result (Dekker 1971; Karp and
// Markstein 1997), ~44 significant bits.
struct FR {
  float h, l;
};
__device__ __forceinline__ FR fr_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return FR{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ FR fr_add(FR a, FR b) {
  float s, e;
  FF::two_sum(a.h, b.h, s, e);
  return fr_norm(s, __fadd_rn(__fadd_rn(a.l, b.l), e));
}
__device__ __forceinline__ FR fr_sub(FR a, FR b) { return fr_add(a, FR{-b.h, -b.l}); }
__device__ __forceinline__ FR fr_mul(FR a, FR b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return fr_norm(p, e);
}
__device__ __forceinline__ FR fr_div(FR a, FR b) {
  const float q = __fdiv_rn(a.h, b.h);
  const FR r = fr_sub(a, fr_mul(FR{q, 0.0f}, b));
  return fr_norm(q, __fdiv_rn(__fadd_rn(r.h, r.l), b.h));
}
__device__ __forceinline__ FR fr_sqrt(FR a) {
  if (!(a.h > 0.0f)) return FR{0.0f, 0.0f};
  const float s = __fsqrt_rn(a.h);
  const FR r = fr_sub(a, fr_mul(FR{s, 0.0f}, FR{s, 0.0f}));
  return fr_norm(s, __fdiv_rn(__fadd_rn(r.h, r.l), 2.0f * s));
}
__device__ __forceinline__ FR re_of(const FF::V& v) { return FR{v.rh, v.rl}; }
__device__ __forceinline__ FR im_of(const FF::V& v) { return FR{v.ih, v.il}; }
__device__ __forceinline__ FF::V cmk(FR x, FR y) { return FF::V{x.h, x.l, y.h, y.l}; }
__device__ __forceinline__ FF::V cconj(const FF::V& v) { return FF::V{v.rh, v.rl, -v.ih, -v.il}; }
__device__ __forceinline__ FF::V cscale(const FF::V& v, FR s) {
  return cmk(fr_mul(re_of(v), s), fr_mul(im_of(v), s));
}
__device__ __forceinline__ FR cnorm2(const FF::V& v) {
  return fr_add(fr_mul(re_of(v), re_of(v)), fr_mul(im_of(v), im_of(v)));
}
// a / b = a conj(b) / |b|^2
__device__ __forceinline__ FF::V cdiv(const FF::V& a, const FF::V& b) {
  const FR n = cnorm2(b);
  const FF::V t = FF::mulv(a, cconj(b));
  return cmk(fr_div(re_of(t), n), fr_div(im_of(t), n));
}
// principal square root, as csqrt_fast
__device__ __forceinline__ FF::V csqrt_ff(const FF::V& v) {
  const FR r = fr_sqrt(cnorm2(v));
  if (r.h == 0.0f) return FF::V{0.0f, 0.0f, 0.0f, 0.0f};
  const FR x = re_of(v), y = im_of(v);
  const FR half{0.5f, 0.0f};
  if (x.h >= 0.0f) {
    const FR t = fr_sqrt(fr_mul(half, fr_add(r, x)));
    return cmk(t, fr_div(fr_mul(y, half), t));
  }
  const FR t = fr_sqrt(fr_mul(half, fr_sub(r, x)));
  const FR ay = y.h < 0.0f ? FR{-y.h, -y.l} : y;
  return cmk(fr_div(fr_mul(ay, half), t), y.h < 0.0f ? FR{-t.h, -t.l} : t);
}

// One Newton step on P(z) = z^a + sum_j c_j z^j from the float-float root
// z, and a bound on the remaining error of the root: |P| plus the
// float-float errors of the coefficients (1e-13 times the locator solve's
// condition estimate `cond`) and of the evaluation, all weighted by
// sum |c_j| and divided by |P'|.  A root of a cluster (small |P'|) or of an
// ill-conditioned locator gets a large bound, and the caller's decisions
// then go to the FP64 decoder whenever the bound could move them.
template <int a>
__device__ __forceinline__ float root_polish(const FF::V* c, FF::V& z, float cond) {
  FF::V P{1.0f, 0.0f, 0.0f, 0.0f}, dP{0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int j = a - 1; j >= 0; --j) {
    dP = FF::add(FF::mulv(dP, z), P);
    P = FF::add(FF::mulv(P, z), c[j]);
  }
  const float nd = ff_norm(dP);
  if (!(nd > 1e-30f && nd < 1e30f)) return INFINITY;
  z = FF::sub(z, cdiv(P, dP));
  float cs = 1.0f;
#pragma unroll
  for (int j = 0; j < a; ++j) cs += sqrtf(ff_norm(c[j]));
  // the step's size, squared, is ~|P|^2 / |P'|^2; after the step the error
  // is quadratically smaller for a simple root, but a cluster keeps it
  const float step = sqrtf(ff_norm(P) / nd);
  return fminf(step, 1.0f) * 0.5f + 1e-13f * fmaxf(cond, 1.0f) * cs / sqrtf(nd);
}

// The two-alias decode of the mixed path in float-float (Sec. II-B steps
// (i)-(iii) for a = 2): the 2 x 2 Hankel solve by Gaussian elimination with
// partial pivoting, the quadratic's roots in the cancellation-free form, the
// snap of each root to S_k, the values by the normal equations over all nm
// equations, the theta and residual tests.  As decode_a1_ff: every deciding
// quantity is compared in FP32 against its threshold, and a value within
// the float-float error's margin of it (or a degenerate pivot, root or
// normal matrix) returns -1 so that the caller runs the FP64 decoder.
// Returns 1 on success (s ascending, p_ff, res_out filled), 0 on failure.
template <int nm>
__device__ __forceinline__ int decode_a2_ff(const float4* raw, int64_t k, const BinGeom& g,
                                            const Tol2f& tol, const OmegaTabFF& omff, int64_t* s,
                                            float4* p_ff, float4* res_out) {
  FF::V m[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) m[i] = FF::from4(raw[i]);
  const float n0 = ff_norm(m[0]), n1 = ff_norm(m[1]), n2 = ff_norm(m[2]);
  const float amax2 = fmaxf(n0, fmaxf(n1, n2));
  if (!(amax2 > 1e-30f && amax2 < 1e30f)) return -1;
  // (i) sum_j c_j m_{i+j} = -m_{2+i}: pivot on the larger of |m0|, |m1|
  const bool swap = n1 > n0;
  const FF::V a0 = swap ? m[1] : m[0], a1 = swap ? m[2] : m[1];  // pivot row
  const FF::V o0 = swap ? m[0] : m[1], o1 = swap ? m[1] : m[2];  // other row
  const FF::V r0 = swap ? m[3] : m[2], r1 = swap ? m[2] : m[3];  // -rhs
  const float best = fmaxf(n0, n1);
  if (best <= 1e-24f * amax2) return -1;
  const FF::V f = cdiv(o0, a0);
  const FF::V a22 = FF::sub(o1, FF::mulv(f, a1));
  const float n22 = ff_norm(a22);
  if (n22 <= 1e-24f * amax2) return -1;
  const FF::V b2 = FF::sub(FF::mulv(f, r0), r1);  // -r1 - f (-r0)
  const FF::V c1 = cdiv(b2, a22);
  const FF::V c0 = cdiv(FF::sub(FF::V{-r0.rh, -r0.rl, -r0.ih, -r0.il}, FF::mulv(a1, c1)), a0);
  // (ii) z^2 + c1 z + c0: q = -(c1 + sqrt(D)) / 2 on the larger branch
  const FF::V D = FF::sub(FF::mulv(c1, c1), cscale(c0, FR{4.0f, 0.0f}));
  const FF::V sq = csqrt_ff(D);
  const FF::V qp = FF::add(c1, sq), qm = FF::sub(c1, sq);
  const FF::V qs = ff_norm(qp) >= ff_norm(qm) ? qp : qm;
  const FF::V q = cscale(qs, FR{-0.5f, 0.0f});
  const float nq = ff_norm(q);
  if (!(nq > 1e-30f && nq < 1e30f)) return -1;
  FF::V z[2] = {q, cdiv(c0, q)};
  FF::V w[2];
  const FF::V cc[2] = {c0, c1};
  const float cond = sqrtf(amax2 / fminf(best, n22));
  const float r2 = tol.root2;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float err = root_polish<2>(cc, z[j], cond);
    const float zx = ff_re(z[j]), zy = ff_im(z[j]);
    if (!(zx * zx + zy * zy > 1e-30f && zx * zx + zy * zy < 1e30f)) return -1;
    const float df = (float)(int)g.d;
    const float qa = fmaf(atan2f(zy, zx), df * 0.15915494309189533577f, -k_over_M(k, g.M));
    const float fr = qa - rintf(qa);
    const float err_t = 10.0f * err * df * 0.15915494309189533577f;
    if (!(err_t < 0.25f)) return -1;
    if (fabsf(fabsf(fr) - 0.5f) < fmaxf(fmaxf(1e-3f, 8e-7f * df), err_t)) return -1;
    s[j] = k + cand_of(__float2int_rn(qa), g.d) * g.M;
    w[j] = omega_ff(omff, s[j]);
    const float dx = zx - ff_re(w[j]), dy = zy - ff_im(w[j]);
    const float dz = dx * dx + dy * dy;
    if (fabsf(dz - r2) <= 1e-4f * r2) return -1;
    if (fabsf(sqrtf(dz) - sqrtf(r2)) < 10.0f * err) return -1;
    if (!(dz <= r2)) return 0;
  }
  if (s[0] == s[1]) return 0;
  if (s[0] > s[1]) {
    const int64_t ts = s[0];
    s[0] = s[1];
    s[1] = ts;
    const FF::V tw = w[0];
    w[0] = w[1];
    w[1] = tw;
  }
  // (iii) normal equations: G = [[nm, S], [conj(S), nm]], S = sum_i
  // (conj(w0) w1)^i; g_u = sum_i conj(w_u)^i m_i
  const FF::V u = FF::mulv(cconj(w[0]), w[1]);
  FF::V S{1.0f, 0.0f, 0.0f, 0.0f}, up = u;
  FF::V g0 = m[0], g1 = m[0];
  FF::V c0p = cconj(w[0]), c1p = cconj(w[1]);
  const FF::V cw0 = c0p, cw1 = c1p;
#pragma unroll
  for (int i = 1; i < nm; ++i) {
    const FF::V mi = FF::from4(raw[i]);
    S = FF::add(S, up);
    g0 = FF::add(g0, FF::mulv(mi, c0p));
    g1 = FF::add(g1, FF::mulv(mi, c1p));
    if (i + 1 < nm) {
      up = FF::mulv(up, u);
      c0p = FF::mulv(c0p, cw0);
      c1p = FF::mulv(c1p, cw1);
    }
  }
  const FR fnm{(float)nm, 0.0f};
  const FR nS = cnorm2(S);
  // nm^2 - |S|^2 = nm a22 with a22 the second pivot of the FP64 solve,
  // which fails when |a22| <= 1e-14 nm; the float-float difference carries
  // an absolute error near 1e-14 nm^2, so below 1e-12 nm^2 FP64 decides
  const FR det = fr_sub(fr_mul(fnm, fnm), nS);
  if (!(det.h > 1e-12f * (float)(nm * nm))) return -1;
  // p1 = (nm g1 - conj(S) g0) / det,  p0 = (g0 - S p1) / nm
  const FF::V num1 = FF::sub(cscale(g1, fnm), FF::mulv(cconj(S), g0));
  const FF::V p1 = cmk(fr_div(re_of(num1), det), fr_div(im_of(num1), det));
  const FF::V t0 = FF::sub(g0, FF::mulv(S, p1));
  const FF::V p0 = cmk(fr_div(re_of(t0), fnm), fr_div(im_of(t0), fnm));
  const int small0 = ff_le_f(ff_norm(p0), tol.theta2), small1 = ff_le_f(ff_norm(p1), tol.theta2);
  if (small0 < 0 || small1 < 0) return -1;
  if (small0 || small1) return 0;
  // the residual over all equations
  float mmax2 = 0.0f, rmax2 = 0.0f;
  FF::V r[nm];
  FF::V f0 = p0, f1 = p1;
#pragma unroll
  for (int i = 0; i < nm; ++i) {
    const FF::V mi = FF::from4(raw[i]);
    r[i] = FF::sub(mi, FF::add(f0, f1));
    if (i + 1 < nm) {
      f0 = FF::mulv(f0, w[0]);
      f1 = FF::mulv(f1, w[1]);
    }
    mmax2 = fmaxf(mmax2, ff_norm(mi));
    rmax2 = fmaxf(rmax2, ff_norm(r[i]));
  }
  const int fits = ff_le_f(rmax2, tol.res2 * mmax2);
  if (fits <= 0) return fits;
  p_ff[0] = FF::to4(p0);
  p_ff[1] = FF::to4(p1);
#pragma unroll
  for (int i = 0; i < nm; ++i) res_out[i] = FF::to4(r[i]);
  return 1;
}

// Decode bin k with `a` aliases from m[0..nm).  On success fills s[0..a)
// (ascending), p[0..a), replaces m[0..nm) by the residual m - Z p and
// returns true; on failure m is unchanged.
//
// On the mixed path the caller passes the float-float syndromes `raw` and
// the float-float omega tables: validation (iii) then runs in float-float
// (ff_residual_ok) and, on success, the residual goes to res_out (float-
// float) instead of m.  With raw == nullptr everything stays in FP64.
template <int a, int nm>
__device__ __forceinline__ bool decode_bin(cdbl* m, int64_t k, const BinGeom& g, const Tol2& tol,
                                           int64_t* s, cdbl* p, const float4* raw = nullptr,
                                           const OmegaTabFF* omff = nullptr,
                                           float4* res_out = nullptr) {
  static_assert(nm >= 2 * a && nm <= 16, "need 2a <= nm <= 16 syndromes");
  if constexpr (a == 1) {
    // c_0 = -m_1 / m_0, the single root z = m_1 / m_0 (Sec. II-A).  Only
    // the root's angle (to pick the candidate) and its distance to that
    // candidate (against root_tol) are used, so z is formed in FP32; FP64
    // decides where the FP32 values lie near a candidate midpoint or near
    // the root_tol bound, and when the FP32 quotient leaves the float range.
    if (m[0].x == 0.0 && m[0].y == 0.0) return false;
    const float m0x = (float)m[0].x, m0y = (float)m[0].y;
    const float m1x = (float)m[1].x, m1y = (float)m[1].y;
    const float den = m0x * m0x + m0y * m0y;
    cdbl w;
    if (den > 1e-30f && den < 1e30f) {
      const float inv = __frcp_rn(den);
      const float zx = (m1x * m0x + m1y * m0y) * inv, zy = (m1y * m0x - m1x * m0y) * inv;
      if (zx == 0.0f && zy == 0.0f) return false;
      s[0] = snap_root_f(zx, zy, k, g, m[0], m[1]);
      w = omega_pow(g.om, s[0]);
      const float dx = zx - (float)w.x, dy = zy - (float)w.y;
      const float dz = dx * dx + dy * dy, r2 = (float)tol.root2;
      if (fabsf(dz - r2) <= 1e-4f * r2) {
        const cdbl z = m[1] * crcp(m[0]);
        if (!(norm2(z - w) <= tol.root2)) return false;
      } else if (!(dz <= r2)) {
        return false;
      }
    } else {
      const cdbl z = m[1] * crcp(m[0]);
      if (!(isfinite(z.x) && isfinite(z.y)) || (z.x == 0.0 && z.y == 0.0)) return false;
      s[0] = snap_root(z, k, g);
      w = omega_pow(g.om, s[0]);
      if (!(norm2(z - w) <= tol.root2)) return false;
    }
    // least squares over all equations: Z^H Z = nm, p = (1/nm) sum conj(w^i) m_i
    if constexpr (nm == 2) {
      // p = (m0 + conj(w) m1) / 2; the residuals are r0 = (m0 - conj(w) m1)/2
      // and r1 = m1 - p w = -w r0, so |r1| = |r0|
      const cdbl t = conjd(w) * m[1];
      p[0] = (m[0] + t) * 0.5;
      if (!(norm2(p[0]) > tol.theta2)) return false;
      const cdbl r0 = (m[0] - t) * 0.5;
      const double mmax2 = fmax(norm2(m[0]), norm2(m[1]));
      if (!(norm2(r0) <= tol.res2 * mmax2)) return false;
      m[0] = r0;
      m[1] = -(w * r0);
      if (res_out != nullptr) {
        res_out[0] = Store<FF>::from_d_small(m[0]);
        res_out[1] = Store<FF>::from_d_small(m[1]);
      }
      return true;
    } else {
      cdbl acc = m[0], wp = w;
#pragma unroll
      for (int i = 1; i < nm; ++i) {
        acc = acc + conjd(wp) * m[i];
        wp = wp * w;
      }
      p[0] = acc * (1.0 / (double)nm);
      if (!(norm2(p[0]) > tol.theta2)) return false;
      if (raw != nullptr) {
        const int ok = ff_residual_ok<1, nm>(raw, s, p, *omff, tol.res2, res_out);
        if (ok >= 0) return ok == 1;
      }
      double mmax2 = 0.0, rmax2 = 0.0;
      cdbl r[nm];
      wp = mk(1.0, 0.0);
#pragma unroll
      for (int i = 0; i < nm; ++i) {
        r[i] = m[i] - p[0] * wp;
        wp = wp * w;
        mmax2 = fmax(mmax2, norm2(m[i]));
        rmax2 = fmax(rmax2, norm2(r[i]));
      }
      if (!(rmax2 <= tol.res2 * mmax2)) return false;
#pragma unroll
      for (int i = 0; i < nm; ++i) m[i] = r[i];
      if (res_out != nullptr) {
#pragma unroll
        for (int i = 0; i < nm; ++i) res_out[i] = Store<FF>::from_d_small(m[i]);
      }
      return true;
    }
  } else {
    cdbl H[a * a], rhs[a], c[a];
#pragma unroll
    for (int i = 0; i < a; ++i) {
#pragma unroll
      for (int j = 0; j < a; ++j) H[i * a + j] = m[i + j];
      rhs[i] = -m[a + i];
    }
    if (!solve_small<a>(H, rhs, c)) return false;

    cdbl z[4];
    if constexpr (a == 2) {
      quad_roots(c[1], c[0], z);
    } else if constexpr (a == 3) {
      cubic_roots(c[2], c[1], c[0], z);
    } else {
      quartic_roots(c[3], c[2], c[1], c[0], z);
    }
    cdbl w[a];
#pragma unroll
    for (int j = 0; j < a; ++j) {
      if (!(isfinite(z[j].x) && isfinite(z[j].y)) || is_zero_c(z[j])) return false;
      s[j] = snap_root(z[j], k, g);
      w[j] = omega_pow(g.om, s[j]);
      if (!(norm2(z[j] - w[j]) <= tol.root2)) return false;
    }
    // ascending locations (sorting network on (s, w) pairs), distinct
    auto cswap = [&](int u, int v) {
      if (s[u] > s[v]) {
        const int64_t ts = s[u];
        s[u] = s[v];
        s[v] = ts;
        const cdbl tw = w[u];
        w[u] = w[v];
        w[v] = tw;
      }
    };
    if constexpr (a == 2) {
      cswap(0, 1);
    } else if constexpr (a == 3) {
      cswap(0, 1);
      cswap(1, 2);
      cswap(0, 1);
    } else {
      cswap(0, 1);
      cswap(2, 3);
      cswap(0, 2);
      cswap(1, 3);
      cswap(1, 2);
    }
#pragma unroll
    for (int j = 1; j < a; ++j)
      if (s[j] == s[j - 1]) return false;

    // normal equations (Z^H Z) p = Z^H m over all nm equations, Z_ij = w_j^i.
    // Z^H Z is Hermitian with diagonal nm, and its (u, v) entry is the
    // geometric sum sum_i q^i of q = conj(w_u) w_v: a(a-1)/2 sums.  Both
    // the sums and Z^H m (sum_i conj(w_u)^i m_i) are polynomials evaluated
    // by Horner's rule: one complex multiply-add per term.
    cdbl G[a * a], gr[a], wp[a];
#pragma unroll
    for (int u = 0; u < a; ++u) {
      G[u * a + u] = mk((double)nm, 0.0);
#pragma unroll
      for (int v = u + 1; v < a; ++v) {
        const cdbl q = conjd(w[u]) * w[v];
        cdbl acc = mk(1.0 + q.x, q.y);
#pragma unroll
        for (int i = 2; i < nm; ++i) acc = cfma(acc, q, mk(1.0, 0.0));
        G[u * a + v] = acc;
        G[v * a + u] = conjd(acc);
      }
    }
#pragma unroll
    for (int u = 0; u < a; ++u) {
      const cdbl cw = conjd(w[u]);
      cdbl acc = m[nm - 1];
#pragma unroll
      for (int i = nm - 2; i >= 0; --i) acc = cfma(acc, cw, m[i]);
      gr[u] = acc;
    }
    if (!solve_small<a>(G, gr, p)) return false;
#pragma unroll
    for (int j = 0; j < a; ++j)
      if (!(norm2(p[j]) > tol.theta2)) return false;
    if (raw != nullptr) {
      const int ok = ff_residual_ok<a, nm>(raw, s, p, *omff, tol.res2, res_out);
      if (ok >= 0) return ok == 1;
    }
    double mmax2 = 0.0, rmax2 = 0.0;
    cdbl r[nm];
#pragma unroll
    for (int u = 0; u < a; ++u) wp[u] = mk(1.0, 0.0);
#pragma unroll
    for (int i = 0; i < nm; ++i) {
      cdbl fit = mk(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < a; ++j) {
        fit = fit + p[j] * wp[j];
        wp[j] = wp[j] * w[j];
      }
      r[i] = m[i] - fit;
      mmax2 = fmax(mmax2, norm2(m[i]));
      rmax2 = fmax(rmax2, norm2(r[i]));
    }
    if (!(rmax2 <= tol.res2 * mmax2)) return false;
#pragma unroll
    for (int i = 0; i < nm; ++i) m[i] = r[i];
    if (res_out != nullptr) {
#pragma unroll
      for (int i = 0; i < nm; ++i) res_out[i] = Store<FF>::from_d_small(m[i]);
    }
    return true;
  }
}

}  // namespace sft
