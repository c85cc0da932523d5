// sft_common.cuh -- value types and small helpers shared by the sm_103a
// kernels of the sparse FFT library.
//
// Two arithmetic flavours run the FFTs:
//   F64 : complex FP64 on the FP64 pipes (the plain FP64 form).
//   FF  : compensated "float-float" complex, each real part held as an
//         unevaluated sum hi + lo of two floats and combined with error-free
//         transformations (TwoSum, TwoProd via FMA).  It runs on the FP32
//         pipes -- GB300 has roughly 1/60 of its FP32 rate in FP64 -- and
//         keeps about 44 significant bits, which the syndrome decoder needs:
//         decisions on ill-conditioned bins flip under plain FP32 rounding
//         of the syndromes (relative 6e-8), but not under ~1e-12.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sft {

// ------------------------------------------------------------ FP64 complex
struct cdbl {
  double x, y;
};

__device__ __forceinline__ cdbl mk(double x, double y) { return cdbl{x, y}; }
__device__ __forceinline__ cdbl operator+(cdbl a, cdbl b) { return cdbl{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdbl operator-(cdbl a, cdbl b) { return cdbl{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdbl operator-(cdbl a) { return cdbl{-a.x, -a.y}; }
__device__ __forceinline__ cdbl operator*(cdbl a, cdbl b) {
  return cdbl{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__device__ __forceinline__ cdbl operator*(cdbl a, double s) { return cdbl{a.x * s, a.y * s}; }
__device__ __forceinline__ cdbl conjd(cdbl a) { return cdbl{a.x, -a.y}; }
// a b + c in four FMAs
__device__ __forceinline__ cdbl cfma(cdbl a, cdbl b, cdbl c) {
  return cdbl{fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
__device__ __forceinline__ double norm2(cdbl a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double absd(cdbl a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cdbl cdivd(cdbl a, cdbl b) {
  // Smith's scaled division: avoids overflow/underflow of |b|^2
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, den = b.x + b.y * r;
    return cdbl{(a.x + a.y * r) / den, (a.y - a.x * r) / den};
  } else {
    double r = b.x / b.y, den = b.x * r + b.y;
    return cdbl{(a.x * r + a.y) / den, (a.y * r - a.x) / den};
  }
}
// principal square root (branch cut on the negative real axis)
__device__ __forceinline__ cdbl csqrtd(cdbl v) {
  double r = hypot(v.x, v.y);
  if (r == 0.0) return cdbl{0.0, 0.0};
  if (v.x >= 0.0) {
    double t = sqrt(0.5 * (r + v.x));
    return cdbl{t, v.y / (2.0 * t)};
  }
  double t = sqrt(0.5 * (r - v.x));
  return cdbl{fabs(v.y) / (2.0 * t), copysign(t, v.y)};
}
// principal cube root, r^(1/3) e^{i arg(v)/3}
__device__ __forceinline__ cdbl ccbrtd(cdbl v) {
  double r = hypot(v.x, v.y);
  if (r == 0.0) return cdbl{0.0, 0.0};
  double th = atan2(v.y, v.x) / 3.0;
  double s, c;
  sincos(th, &s, &c);
  double m = cbrt(r);
  return cdbl{m * c, m * s};
}

// ----------------------------------------------------- omega^e from tables
// omega = e^{2 pi i / N}; omega^e = hi[e >> lo_bits] * lo[e & lo_mask] with
// both tables FP64 and correctly rounded (built on the host).
struct OmegaTab {
  const double2* hi;
  const double2* lo;
  int lo_bits;
  int64_t mask;  // N - 1
};
__device__ __forceinline__ cdbl omega_pow(const OmegaTab& t, int64_t e) {
  int64_t r = e & t.mask;  // e mod N for any sign (N is a power of two)
  double2 a = __ldg(t.hi + (r >> t.lo_bits));
  double2 b = __ldg(t.lo + (r & ((int64_t(1) << t.lo_bits) - 1)));
  return cdbl{a.x, a.y} * cdbl{b.x, b.y};
}

// ------------------------------------------------------- FFT value traits
// Shared-memory slot of FFT element i: one spare slot per 16 elements, so
// that the first Stockham pass (thread j writes elements 16j .. 16j+15)
// does not hit one bank with every lane of a half-warp.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// padded length of an M-point buffer
__host__ __device__ __forceinline__ int padded(int M) { return M + (M >> 4); }

// Constant twiddles e^{-2 pi i m/16}, m = 0..7, for the in-register radix-16
// butterflies (correctly rounded double literals).
#define SFT_C1 0.92387953251128675613
#define SFT_S1 0.38268343236508977173
#define SFT_R2 0.70710678118654752440
__device__ __forceinline__ double tw16_re(int m) {
  constexpr double v[8] = {1.0, SFT_C1, SFT_R2, SFT_S1, 0.0, -SFT_S1, -SFT_R2, -SFT_C1};
  return v[m];
}
__device__ __forceinline__ double tw16_im(int m) {
  constexpr double v[8] = {0.0, -SFT_S1, -SFT_R2, -SFT_C1, -1.0, -SFT_C1, -SFT_R2, -SFT_S1};
  return v[m];
}

struct F64 {
  struct V {
    double rx, ry;
  };
  typedef double2 Tw;                 // twiddle table entry
  typedef double2 In;                 // input element (complex128)
  static constexpr int kBytesPerPoint = 16;
  __device__ static __forceinline__ V add(V a, V b) { return V{a.rx + b.rx, a.ry + b.ry}; }
  __device__ static __forceinline__ V sub(V a, V b) { return V{a.rx - b.rx, a.ry - b.ry}; }
  __device__ static __forceinline__ V mul(V a, double wx, double wy) {
    return V{fma(a.rx, wx, -a.ry * wy), fma(a.rx, wy, a.ry * wx)};
  }
  __device__ static __forceinline__ V mul_tw(V a, Tw w) { return mul(a, w.x, w.y); }
  __device__ static __forceinline__ V mul_c16(V a, int m) { return mul(a, tw16_re(m), tw16_im(m)); }
  __device__ static __forceinline__ V mul_mi(V a) { return V{a.ry, -a.rx}; }  // * (-i)
  __device__ static __forceinline__ V from_in(In v) { return V{v.x, v.y}; }
  __device__ static __forceinline__ void st(char* sm, int M, int i, V v) {
    reinterpret_cast<double2*>(sm)[pad16(i)] = make_double2(v.rx, v.ry);
  }
  __device__ static __forceinline__ V ld(const char* sm, int M, int i) {
    double2 t = reinterpret_cast<const double2*>(sm)[pad16(i)];
    return V{t.x, t.y};
  }
  typedef double2 Out;
  __device__ static __forceinline__ double2 out(V v, double scale) {
    return make_double2(v.rx * scale, v.ry * scale);
  }
  __device__ static __forceinline__ V from_out(double2 o) { return V{o.x, o.y}; }
  __device__ static __forceinline__ double out_norm(double2 o) { return o.x * o.x + o.y * o.y; }
};

struct FF {
  struct V {
    float rh, rl, ih, il;
  };
  typedef float4 Tw;  // (re_hi, re_lo, im_hi, im_lo)
  typedef float2 In;  // input element (complex64)
  static constexpr int kBytesPerPoint = 16;

  // Knuth's TwoSum: s + e == a + b exactly (no FMA contraction possible
  // through the _rn intrinsics).
  __device__ static __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  }
  // Dekker's FastTwoSum, |a| >= |b|
  __device__ static __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
  }
  __device__ static __forceinline__ V add(V a, V b) {
    V r;
    float e;
    two_sum(a.rh, b.rh, r.rh, e);
    r.rl = __fadd_rn(__fadd_rn(a.rl, b.rl), e);
    two_sum(a.ih, b.ih, r.ih, e);
    r.il = __fadd_rn(__fadd_rn(a.il, b.il), e);
    return r;
  }
  __device__ static __forceinline__ V sub(V a, V b) {
    V r;
    float e;
    two_sum(a.rh, -b.rh, r.rh, e);
    r.rl = __fadd_rn(__fsub_rn(a.rl, b.rl), e);
    two_sum(a.ih, -b.ih, r.ih, e);
    r.il = __fadd_rn(__fsub_rn(a.il, b.il), e);
    return r;
  }
  // hi/lo product of two float-float reals (terms below 2^-44 dropped),
  // returned as an unnormalised pair (p, err)
  __device__ static __forceinline__ void prod(float ah, float al, float bh, float bl, float& p,
                                              float& err) {
    p = __fmul_rn(ah, bh);
    err = __fmaf_rn(ah, bh, -p);
    err = __fmaf_rn(ah, bl, err);
    err = __fmaf_rn(al, bh, err);
  }
  // (ah + al)(bh + bl) - (ch + cl)(dh + dl), renormalised
  __device__ static __forceinline__ void dot2(float ah, float al, float bh, float bl, float ch,
                                              float cl, float dh, float dl, float& rh, float& rl) {
    float p1, e1, p2, e2, s, e3;
    prod(ah, al, bh, bl, p1, e1);
    prod(ch, cl, dh, dl, p2, e2);
    two_sum(p1, -p2, s, e3);
    float lo = __fadd_rn(__fsub_rn(e1, e2), e3);
    fast_two_sum(s, lo, rh, rl);
  }
  __device__ static __forceinline__ V mul4(V a, float wrh, float wrl, float wih, float wil) {
    V r;
    dot2(a.rh, a.rl, wrh, wrl, a.ih, a.il, wih, wil, r.rh, r.rl);   // re
    dot2(a.rh, a.rl, wih, wil, -a.ih, -a.il, wrh, wrl, r.ih, r.il); // im
    return r;
  }
  __device__ static __forceinline__ V mul_tw(V a, Tw w) { return mul4(a, w.x, w.y, w.z, w.w); }
  // e^{-2 pi i m/16} split into float hi + lo parts (exact float literals);
  // m = 0 and m = 4 never reach here (identity and mul_mi).
  __device__ static __forceinline__ V mul_c16(V a, int m) {
    constexpr float ch[8] = {1.0f, 0.9238795042037964f, 0.7071067690849304f, 0.3826834261417389f,
                             0.0f, -0.3826834261417389f, -0.7071067690849304f, -0.9238795042037964f};
    constexpr float cl[8] = {0.0f, 2.830748968563057e-08f, 1.2101617485882343e-08f,
                             6.2233507236442165e-09f, 0.0f, -6.2233507236442165e-09f,
                             -1.2101617485882343e-08f, -2.830748968563057e-08f};
    constexpr float sh[8] = {0.0f, -0.3826834261417389f, -0.7071067690849304f, -0.9238795042037964f,
                             -1.0f, -0.9238795042037964f, -0.7071067690849304f, -0.3826834261417389f};
    constexpr float sl[8] = {0.0f, -6.2233507236442165e-09f, -1.2101617485882343e-08f,
                             -2.830748968563057e-08f, 0.0f, -2.830748968563057e-08f,
                             -1.2101617485882343e-08f, -6.223351167733426e-09f};
    return mul4(a, ch[m], cl[m], sh[m], sl[m]);
  }
  __device__ static __forceinline__ V mul_mi(V a) { return V{a.ih, a.il, -a.rh, -a.rl}; }
  __device__ static __forceinline__ V from_in(In v) { return V{v.x, 0.f, v.y, 0.f}; }
  // shared memory: hi plane (float2) followed by lo plane (float2)
  __device__ static __forceinline__ void st(char* sm, int M, int i, V v) {
    reinterpret_cast<float2*>(sm)[pad16(i)] = make_float2(v.rh, v.ih);
    reinterpret_cast<float2*>(sm)[padded(M) + pad16(i)] = make_float2(v.rl, v.il);
  }
  __device__ static __forceinline__ V ld(const char* sm, int M, int i) {
    float2 h = reinterpret_cast<const float2*>(sm)[pad16(i)];
    float2 l = reinterpret_cast<const float2*>(sm)[padded(M) + pad16(i)];
    return V{h.x, l.x, h.y, l.y};
  }
  // syndromes leave the FFT as float-float quadruples scaled by d (a power
  // of two, so the scaling is exact and stays on the FP32 pipes)
  typedef float4 Out;
  __device__ static __forceinline__ float4 out(V v, float scale) {
    return make_float4(v.rh * scale, v.rl * scale, v.ih * scale, v.il * scale);
  }
  __device__ static __forceinline__ float out_norm_hi(float4 o) { return o.x * o.x + o.z * o.z; }
  __device__ static __forceinline__ double out_norm(float4 o) { return (double)out_norm_hi(o); }
  __device__ static __forceinline__ V from_out(float4 o) { return V{o.x, o.y, o.z, o.w}; }
  __device__ static __forceinline__ V from4(float4 o) { return V{o.x, o.y, o.z, o.w}; }
  __device__ static __forceinline__ float4 to4(V v) { return make_float4(v.rh, v.rl, v.ih, v.il); }
  __device__ static __forceinline__ V mulv(V a, V b) { return mul4(a, b.rh, b.rl, b.ih, b.il); }
};

// Storage of held syndromes and recovered values: FP64 pairs on the plain
// path, float-float quadruples (hi, lo of re, hi, lo of im) on the mixed path;
// 16 bytes either way.  to_d/from_d convert for the FP64 solves.
template <class F>
struct Store;
template <>
struct Store<F64> {
  typedef double2 T;
  __device__ static __forceinline__ cdbl to_d(double2 v) { return cdbl{v.x, v.y}; }
  __device__ static __forceinline__ double2 from_d(cdbl c) { return make_double2(c.x, c.y); }
  __device__ static __forceinline__ double2 from_d_small(cdbl c) { return make_double2(c.x, c.y); }
};
// float -> double by moving the bits (sign, exponent rebiased by
// 1023 - 127 = 896, significand shifted by 52 - 23 = 29): exact, and on the
// integer pipes -- a conversion instruction occupies GB300's scarce FP64
// unit.  Zeros keep their sign; subnormals, infinities and NaNs take the
// conversion instruction.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)sign);
    return (double)f;
  }
  return __longlong_as_double(
      (long long)(sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29)));
}

template <>
struct Store<FF> {
  typedef float4 T;
  // hi + lo in FP64: both parts converted exactly, one FP64 addition each
  __device__ static __forceinline__ cdbl to_d(float4 v) {
    return cdbl{f2d_exact(v.x) + f2d_exact(v.y), f2d_exact(v.z) + f2d_exact(v.w)};
  }
  __device__ static __forceinline__ float4 from_d(cdbl c) {
    const float xh = (float)c.x, yh = (float)c.y;
    return make_float4(xh, (float)(c.x - (double)xh), yh, (float)(c.y - (double)yh));
  }
  // for residuals of accepted decodes (|r| <= res_tol |m|): the hi parts
  // alone carry them to well below the float-float precision of |m|
  __device__ static __forceinline__ float4 from_d_small(cdbl c) {
    return make_float4((float)c.x, 0.0f, (float)c.y, 0.0f);
  }
};

// omega^e as a float-float product of two table entries (mixed path)
struct OmegaTabFF {
  const float4* hi;
  const float4* lo;
  int lo_bits;
  int64_t mask;
};
__device__ __forceinline__ FF::V omega_ff(const OmegaTabFF& t, int64_t e) {
  const int64_t r = e & t.mask;
  const float4 a = __ldg(t.hi + (r >> t.lo_bits));
  const float4 b = __ldg(t.lo + (r & ((int64_t(1) << t.lo_bits) - 1)));
  return FF::mul4(FF::from4(a), b.x, b.y, b.z, b.w);
}

}  // namespace sft
