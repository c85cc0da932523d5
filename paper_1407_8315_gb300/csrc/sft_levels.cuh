// sft_levels.cuh -- the per-bin stages of the exact paths: the fold, peel
// and activity test of each level and the per-level decoder of Algorithm 1
// (ITER), and the activity scan and the decode rounds of the non-iterative
// method (FIXED).  Shared by the translation unit of the launchers and the
// one that instantiates the decoders of more than four aliases.
#pragma once

#include <type_traits>

#include "sft_decode.cuh"
#include "sft_device_util.cuh"
#include "sft_quad.cuh"

struct sft_plan_s;

namespace sft {

// ------------------------------------------------- per-level decode (ITER)
struct LevelArgs {
  int64_t N, M, d, M0;
  const void* prev;  // level l-1 rows, length 2M (Store<F>::T)
  void* cur;         // level l rows, length M
  int64_t held_elems;
  const uint8_t* Tprev;
  uint8_t* Tcur;
  uint8_t* slot_cnt;
  int64_t* slot_s;
  void* slot_p;  // Store<F>::T
  const unsigned long long* ymax2;
  int32_t* flags;
  double zero_tol, root_tol, res_tol;
  OmegaTab om;
  OmegaTabFF omff;
  float zero_tol2_f, root_tol2_f, res_tol2_f;  // the squared tolerances rounded to float
};

// The zero threshold theta^2 = zero_tol^2 max_k |Y_{d,0}[k]|^2 as a float,
// off the FP64 pipe: the max is stored as the double of an FP32 value (the
// FFT's running max of FP32 norms), so its bits move back to the float
// exactly; zero_tol^2 comes rounded to float.  The product is within two
// ulps of the float rounding of the FP64 threshold, far inside above_ff's
// 1e-4 margin.
__device__ __forceinline__ float theta2_f(float zero_tol2_f, unsigned long long ymax_bits) {
  const uint32_t e = (uint32_t)(ymax_bits >> 52) & 0x7FFu;
  if (e == 0u) return 0.0f;
  if (e < 897u || e > 1150u)  // outside the normal float range: convert
    return zero_tol2_f * (float)__longlong_as_double((long long)ymax_bits);
  const uint32_t fb = ((uint32_t)(ymax_bits >> 63) << 31) | ((e - 896u) << 23) |
                      (uint32_t)((ymax_bits >> 29) & 0x7FFFFFu);
  return zero_tol2_f * __uint_as_float(fb);
}

// |m|^2 > theta^2 decided from the float-float hi parts when they are
// clearly on one side (relative error of the hi-part norm < 1e-6; t2 the
// float threshold), in FP64 otherwise -- the same decision the FP64
// comparison takes.  The FP64 threshold is formed only in that rare case.
__device__ __forceinline__ bool above_ff(const FF::V& m, float t2, double zero_tol,
                                         unsigned long long ymax_bits) {
  const float nh = m.rh * m.rh + m.ih * m.ih;
  if (nh > t2 * 1.0001f) return true;
  if (nh < t2 * 0.9999f) return false;
  const double theta2 = zero_tol * zero_tol * __longlong_as_double((long long)ymax_bits);
  const double x = (double)m.rh + (double)m.rl, y = (double)m.ih + (double)m.il;
  return x * x + y * y > theta2;
}

constexpr int kFoldThreads = 256;
constexpr int kDecThreads = 128;

// Level l, phase 1, bin k (< M) of signal b: fold the held syndromes,
// SubFreq on the two new shifts, activity test of Algorithm 1, write the
// syndromes back; returns whether the bin is to be decoded.
template <class F, int A>
__device__ __forceinline__ bool fold_bin(const LevelArgs& g, int b, int64_t k) {
  constexpr int l = A - 1, nm = 2 * A;
  typedef typename Store<F>::T T;
  const int64_t M = g.M, M0 = g.M0;
  bool active = false;
  {
    const T* prev = reinterpret_cast<const T*>(g.prev) + (int64_t)b * g.held_elems;
    T* cur = reinterpret_cast<T*>(g.cur) + (int64_t)b * g.held_elems;
    const uint8_t* cnt = g.slot_cnt + (int64_t)b * M0;
    const int64_t* ss = g.slot_s + (int64_t)b * M0 * kSlots;
    const T* sp = reinterpret_cast<const T*>(g.slot_p) + (int64_t)b * M0 * kSlots;
    uint8_t t = 0;
    if (l > 0) t = (uint8_t)(g.Tprev[(int64_t)b * M0 + k] | g.Tprev[(int64_t)b * M0 + k + M]);
    const unsigned long long ymax_bits = g.ymax2[b];
    const int64_t nsub = int64_t(1) << l;  // M0 / M
    if constexpr (std::is_same<F, F64>::value) {
      cdbl m[nm];
      // fold the syndromes held from level l-1 (length 2M) to length M
#pragma unroll
      for (int j = 0; j < 2 * l; ++j)
        m[j] = Store<F>::to_d(prev[j * 2 * M + k]) + Store<F>::to_d(prev[j * 2 * M + k + M]);
      m[2 * l] = Store<F>::to_d(cur[(2 * l) * M + k]);
      m[2 * l + 1] = Store<F>::to_d(cur[(2 * l + 1) * M + k]);
      // SubFreq: remove every frequency recovered at earlier levels from the
      // two new shifts; they are filed under the level-0 bins k + u M
      bool peeled = false;
      if (l > 0) {
        for (int64_t u = 0; u < nsub; ++u) {
          const int64_t k0 = k + u * M;
          const int c = cnt[k0];
          peeled = peeled || c > 0;
          for (int e = 0; e < c; ++e) {
            const int64_t sl = ss[slot_ix(k0, e, M0)];
            const cdbl p = Store<F>::to_d(sp[slot_ix(k0, e, M0)]);
            m[2 * l] = m[2 * l] - p * omega_pow(g.om, sl * (2 * l));
            m[2 * l + 1] = m[2 * l + 1] - p * omega_pow(g.om, sl * (2 * l + 1));
          }
        }
      }
      const double theta2 = g.zero_tol * g.zero_tol * __longlong_as_double((long long)ymax_bits);
      active = t || norm2(m[2 * l]) > theta2 || norm2(m[2 * l + 1]) > theta2;
      // the folded rows are new; the two new shifts change only when peeled
#pragma unroll
      for (int j = 0; j < 2 * l; ++j) cur[j * M + k] = Store<F>::from_d(m[j]);
      if (peeled) {
        cur[(2 * l) * M + k] = Store<F>::from_d(m[2 * l]);
        cur[(2 * l + 1) * M + k] = Store<F>::from_d(m[2 * l + 1]);
      }
    } else {
      // the held rows fold first, each written back at once: they take no
      // part in the peel or the activity test, so none stays live (in
      // registers) across the peel walk
#pragma unroll
      for (int j = 0; j < 2 * l; ++j)
        cur[j * M + k] =
            FF::to4(FF::add(FF::from4(prev[j * 2 * M + k]), FF::from4(prev[j * 2 * M + k + M])));
      FF::V m[nm];
      m[2 * l] = FF::from4(cur[(2 * l) * M + k]);
      m[2 * l + 1] = FF::from4(cur[(2 * l + 1) * M + k]);
      bool peeled = false;
      if constexpr (l > 0) {
        // the 2^l level-0 bins folded into k, in chunks of up to 8.  A
        // chunk's counts (each <= kSlots = 8) are packed into the nibbles of
        // one word and its entries walked in one loop, sub-bin by sub-bin:
        // a warp then runs as many iterations as its busiest lane has
        // entries, not the sum over sub-bins of the busiest lane's count.
        constexpr int NS = 1 << l;
        constexpr int CH = NS < 8 ? NS : 8;
        static_assert(kSlots <= 15, "counts are packed in 4 bits");
        for (int u0 = 0; u0 < NS; u0 += CH) {
          uint32_t cp = 0u;
#pragma unroll
          for (int u = 0; u < CH; ++u) cp |= (uint32_t)cnt[k + (int64_t)(u0 + u) * M] << (4 * u);
          peeled = peeled || cp != 0u;
          int e = 0;
          while (cp != 0u) {
            const int u = (__ffs((int)cp) - 1) >> 2;
            const int cu = (int)((cp >> (4 * u)) & 15u);
            const int64_t k0 = k + (int64_t)(u0 + u) * M;
            const int64_t sl = ss[slot_ix(k0, e, M0)];
            const FF::V p = FF::from4(sp[slot_ix(k0, e, M0)]);
            m[2 * l] = FF::sub(m[2 * l], FF::mulv(p, omega_ff(g.omff, sl * (2 * l))));
            m[2 * l + 1] = FF::sub(m[2 * l + 1], FF::mulv(p, omega_ff(g.omff, sl * (2 * l + 1))));
            if (++e == cu) {
              cp &= ~(15u << (4 * u));
              e = 0;
            }
          }
        }
      }
      const float t2 = theta2_f(g.zero_tol2_f, ymax_bits);
      active = t || above_ff(m[2 * l], t2, g.zero_tol, ymax_bits) ||
               above_ff(m[2 * l + 1], t2, g.zero_tol, ymax_bits);
      if (peeled) {
        cur[(2 * l) * M + k] = FF::to4(m[2 * l]);
        cur[(2 * l + 1) * M + k] = FF::to4(m[2 * l + 1]);
      }
    }
    if (!active) g.Tcur[(int64_t)b * M0 + k] = 0;
  }
  return active;
}

// Level l, phase 1, one thread per bin: fold_bin, and the active bins queued
// for decoding.  Grid (bin tiles, signals); or, when a level has fewer bins
// than a CTA has threads, n_flat = signals x bins packed densely over
// blockIdx.x (thread f: signal f / M, bin f mod M), so that no CTA runs
// mostly idle threads.
// Mixed path: at most 64 registers, four CTAs per SM, so that more warps
// hide the peel walk's load latency (measured: the folds of levels 1-3
// 0.13 -> 0.11 ms per call at 608 signals, 383 k -> 399 k signals/s).
template <class F>
struct FoldOccupancy {
  static constexpr int kMinBlocks = std::is_same<F, FF>::value ? 4 : 1;
};
template <class F, int A>
__global__ void __launch_bounds__(kFoldThreads, FoldOccupancy<F>::kMinBlocks)
    k_iter_fold(LevelArgs g, int2* queue, int* qcount, int64_t n_flat) {
  int b;
  int64_t k;
  if (n_flat > 0) {
    const int64_t f = (int64_t)blockIdx.x * kFoldThreads + threadIdx.x;
    b = (int)(f >> (__ffsll(g.M) - 1));  // M is a power of two
    k = f < n_flat ? f - (int64_t)b * g.M : g.M;  // past the end: no bin
  } else {
    b = blockIdx.y;
    k = (int64_t)blockIdx.x * kFoldThreads + threadIdx.x;
  }
  const bool active = k < g.M && fold_bin<F, A>(g, b, k);
  block_queue_push<kFoldThreads>(active, b, (int)k, queue, qcount);
}

// Level l, phase 2, one queued bin k of signal b: SynDec with a = l + 1
// (Algorithm 1); a recovered bin is filed and its terms leave the held
// syndromes, an unsolved one is flagged in T.
template <class F, int A>
__device__ __forceinline__ void decode_level_bin(const LevelArgs& g, int b, int64_t k) {
  constexpr int nm = 2 * A;
  typedef typename Store<F>::T T;
  const BinGeom geom{g.N, g.M, g.d, g.om};
  {
    const int64_t M = g.M, M0 = g.M0;
    T* cur = reinterpret_cast<T*>(g.cur) + (int64_t)b * g.held_elems;
    const unsigned long long ymax_bits = g.ymax2[b];
    const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)ymax_bits),
                   g.root_tol * g.root_tol, g.res_tol * g.res_tol};
    const Tol2f tolf{theta2_f(g.zero_tol2_f, ymax_bits), g.root_tol2_f, g.res_tol2_f};
    T raw[nm];
#pragma unroll
    for (int j = 0; j < nm; ++j) raw[j] = cur[j * M + k];
    int64_t s[4];
    cdbl p[4];
    cdbl m[nm];
    uint8_t t = 1;
    bool ok = false, filed = false;
    float4 res[nm];
    // one alias on the mixed path: float-float unless a value lies at a
    // decision boundary (then the FP64 decoder below)
    int fast = -1;
    if constexpr (std::is_same<F, FF>::value && A <= 2) {
      float4 pf[A];
      if constexpr (A == 1)
        fast = decode_a1_ff<nm>(raw, k, geom, tolf, g.omff, s, pf, res);
      else
        fast = decode_a2_ff<nm>(raw, k, geom, tolf, g.omff, s, pf, res);
      if (fast == 1) {
        // level 0 (one alias): nothing is filed under a level-0 bin before
        // its own decode
#pragma unroll
        for (int j = 0; j < A; ++j)
          file_one_ff<A == 1>(s[j], pf[j], M0, g.slot_cnt + (int64_t)b * M0,
                              g.slot_s + (int64_t)b * M0 * kSlots,
                              reinterpret_cast<float4*>(g.slot_p) + (int64_t)b * M0 * kSlots,
                              g.flags + b);
        ok = filed = true;
      }
    }
    if (fast < 0) {
#pragma unroll
      for (int j = 0; j < nm; ++j) m[j] = Store<F>::to_d(raw[j]);
      if constexpr (std::is_same<F, FF>::value)
        ok = decode_bin<A, nm>(m, k, geom, tol, s, p, raw, &g.omff, res);
      else
        ok = decode_bin<A, nm>(m, k, geom, tol, s, p);
    }
    if (ok) {
      if (!filed)
        file_solution<F, A>(s, p, M0, g.slot_cnt + (int64_t)b * M0,
                            g.slot_s + (int64_t)b * M0 * kSlots,
                            reinterpret_cast<T*>(g.slot_p) + (int64_t)b * M0 * kSlots, g.flags + b);
      // the recovered terms leave every syndrome held for this bin
      if constexpr (std::is_same<F, FF>::value) {
#pragma unroll
        for (int j = 0; j < nm; ++j) cur[j * M + k] = res[j];
      } else {
#pragma unroll
        for (int j = 0; j < nm; ++j) cur[j * M + k] = Store<F>::from_d_small(m[j]);
      }
      t = 0;
    }
    g.Tcur[(int64_t)b * M0 + k] = t;
  }
}

// Level l, phase 2: decode the queued bins with a = l + 1 (SynDec, Algorithm 1),
// grid-stride over the queue so that every warp is full.
// The mixed path's two-alias decoder at four CTAs per SM (124 registers, no
// spills; 148 uncapped, three CTAs): more warps hide its float-float
// latencies (measured: level 1 0.142 -> 0.133 ms per call at 608 signals).
// The other decoders keep their natural register counts.
template <class F>
struct DecOccupancy {
  template <int A>
  static constexpr int min_blocks() { return std::is_same<F, FF>::value && A == 2 ? 4 : 1; }
  // FIXED rounds 1 and 2 on the mixed path (all 2 a_max syndromes held):
  // five and four CTAs per SM (96 and 128 registers, a few bytes spilled;
  // 128 and 168 uncapped): round 1 0.185 -> 0.169, round 2 0.263 -> 0.212 ms
  // per call at 608 signals
  template <int A>
  static constexpr int min_blocks_fixed() {
    return !std::is_same<F, FF>::value ? 1 : (A == 1 ? 5 : (A == 2 ? 4 : 1));
  }
};
template <class F, int A>
__global__ void __launch_bounds__(kDecThreads, DecOccupancy<F>::template min_blocks<A>())
    k_iter_decode(LevelArgs g, const int2* queue,
                                                             const int* qcount,
                                                             int n_quad_max = -1) {
  const int n = *qcount;
  if (n <= n_quad_max) return;  // the four-lane decoder takes short queues
  for (int e = blockIdx.x * kDecThreads + threadIdx.x; e < n; e += gridDim.x * kDecThreads) {
    const int2 q = queue[e];
    decode_level_bin<F, A>(g, q.x, q.y);
  }
}

// Level l >= 2 of the mixed path: the queued bins decoded with a = l + 1 in
// {3, 4} by four lanes each (decode_quad), eight bins per warp.  Four lanes
// per bin shorten a bin's FP64 chain but spend about twice the FP64 issue
// slots per bin, so this decoder takes a queue of at most n_quad_max bins
// and the one-lane decoder (launched beside it) a longer one.
template <int A>
__global__ void __launch_bounds__(kDecThreads) k_iter_decode_quad(LevelArgs g, const int2* queue,
                                                                  const int* qcount,
                                                                  int n_quad_max) {
  constexpr int nm = 2 * A, kGroups = kDecThreads / 4;
  const int n = *qcount;
  if (n > n_quad_max) return;
  const BinGeom geom{g.N, g.M, g.d, g.om};
  const int lane = (int)(threadIdx.x & 31u);
  const Quad G{0xFu << (lane & ~3), lane & 3};
  for (int e = blockIdx.x * kGroups + (int)(threadIdx.x >> 2); e < n; e += gridDim.x * kGroups) {
    const int2 qe = queue[e];
    const int b = qe.x;
    const int64_t k = qe.y, M = g.M, M0 = g.M0;
    float4* cur = reinterpret_cast<float4*>(g.cur) + (int64_t)b * g.held_elems;
    const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)g.ymax2[b]),
                   g.root_tol * g.root_tol, g.res_tol * g.res_tol};
    int64_t s[A];
    cdbl p[A];
    const bool ok = decode_quad<A, nm>(G, cur, cur, M, k, geom, tol, g.omff, s, p);
    if (G.q == 0) {
      if (ok)
        file_solution<FF, A>(s, p, M0, g.slot_cnt + (int64_t)b * M0,
                             g.slot_s + (int64_t)b * M0 * kSlots,
                             reinterpret_cast<float4*>(g.slot_p) + (int64_t)b * M0 * kSlots,
                             g.flags + b);
      g.Tcur[(int64_t)b * M0 + k] = ok ? 0 : 1;
    }
  }
}

// ---------------------------------------------- non-iterative decode (FIXED)
struct FixedArgs {
  int64_t N, M, d;
  int a_max;
  const void* Y;  // 2 a_max rows of length M (Store<F>::T)
  int64_t held_elems;
  uint8_t* T;
  uint8_t* slot_cnt;
  int64_t* slot_s;
  void* slot_p;
  const unsigned long long* ymax2;
  int32_t* flags;
  double zero_tol, root_tol, res_tol;
  OmegaTab om;
  OmegaTabFF omff;  // float-float omega tables (mixed path)
  float zero_tol2_f, root_tol2_f, res_tol2_f;  // the squared tolerances rounded to float
};

// activity of every bin (any of the 2 a_max syndromes above theta)
template <class F, int NM>
__global__ void __launch_bounds__(kFoldThreads) k_fixed_scan(FixedArgs g, int2* queue, int* qcount) {
  typedef typename Store<F>::T T;
  const int b = blockIdx.y;
  const int64_t M = g.M;
  const int64_t k = (int64_t)blockIdx.x * kFoldThreads + threadIdx.x;
  bool active = false;
  if (k < M) {
    const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
    const unsigned long long ymax_bits = g.ymax2[b];
#pragma unroll
    for (int j = 0; j < NM; ++j) {
      if constexpr (std::is_same<F, F64>::value) {
        const double theta2 = g.zero_tol * g.zero_tol * __longlong_as_double((long long)ymax_bits);
        active = active || norm2(Store<F>::to_d(Y[j * M + k])) > theta2;
      } else {
        active = active || above_ff(FF::from4(Y[j * M + k]), theta2_f(g.zero_tol2_f, ymax_bits),
                                    g.zero_tol, ymax_bits);
      }
    }
    g.T[(int64_t)b * M + k] = 0;
  }
  block_queue_push<kFoldThreads>(active, b, (int)k, queue, qcount);
}

// round a: decode the queued bins with a aliases; failures go to the next
// round's queue, or are marked unsolved after the last round (a = a_max)
template <class F, int A, int NM>
__global__ void __launch_bounds__(kDecThreads, DecOccupancy<F>::template min_blocks_fixed<A>())
    k_fixed_round(FixedArgs g, const int2* qin,
                                                             const int* nin, int2* qout,
                                                             int* nout, int n_quad_max = -1) {
  typedef typename Store<F>::T T;
  const int n = *nin;
  if (n <= n_quad_max) return;  // the four-lane decoder takes short queues
  const BinGeom geom{g.N, g.M, g.d, g.om};
  const int64_t M = g.M;
  for (int e0 = blockIdx.x * kDecThreads; e0 < n; e0 += gridDim.x * kDecThreads) {
    const int e = e0 + threadIdx.x;
    bool fail = false;
    int b = 0, k = 0;
    if (e < n) {
      const int2 q = qin[e];
      b = q.x;
      k = q.y;
      const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
      const unsigned long long ymax_bits = g.ymax2[b];
      const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)ymax_bits),
                     g.root_tol * g.root_tol, g.res_tol * g.res_tol};
      const Tol2f tolf{theta2_f(g.zero_tol2_f, ymax_bits), g.root_tol2_f, g.res_tol2_f};
      T raw[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) raw[j] = Y[j * M + k];
      int64_t s[4];
      cdbl p[4];
      bool ok = false, filed = false;
      int fast = -1;
      if constexpr (std::is_same<F, FF>::value && A <= 2) {
        float4 pf[A], res[NM];
        if constexpr (A == 1)
          fast = decode_a1_ff<NM>(raw, k, geom, tolf, g.omff, s, pf, res);
        else
          fast = decode_a2_ff<NM>(raw, k, geom, tolf, g.omff, s, pf, res);
        if (fast == 1) {
#pragma unroll
          for (int j = 0; j < A; ++j)
            file_one_ff<A == 1>(s[j], pf[j], M, g.slot_cnt + (int64_t)b * M,
                                g.slot_s + (int64_t)b * M * kSlots,
                                reinterpret_cast<float4*>(g.slot_p) + (int64_t)b * M * kSlots,
                                g.flags + b);
          ok = filed = true;
        }
      }
      if (fast < 0) {
        cdbl m[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) m[j] = Store<F>::to_d(raw[j]);
        if constexpr (std::is_same<F, FF>::value)
          ok = decode_bin<A, NM>(m, k, geom, tol, s, p, raw, &g.omff, nullptr);
        else
          ok = decode_bin<A, NM>(m, k, geom, tol, s, p);
      }
      if (ok) {
        if (!filed)
          file_solution<F, A>(s, p, M, g.slot_cnt + (int64_t)b * M, g.slot_s + (int64_t)b * M * kSlots,
                              reinterpret_cast<T*>(g.slot_p) + (int64_t)b * M * kSlots, g.flags + b);
      } else if (qout == nullptr) {
        g.T[(int64_t)b * M + k] = 1;
      } else {
        fail = true;
      }
    }
    if (qout != nullptr) queue_push(fail, b, k, qout, nout);
  }
}

// Round a in {3, 4} of the mixed path by four lanes per bin (decode_quad),
// for a queue of at most n_quad_max bins (the one-lane round, launched
// beside it, takes a longer one).  The syndromes stay as they are.
template <int A, int NM>
__global__ void __launch_bounds__(kDecThreads) k_fixed_round_quad(FixedArgs g, const int2* qin,
                                                                  const int* nin, int2* qout,
                                                                  int* nout, int n_quad_max) {
  constexpr int kGroups = kDecThreads / 4;
  const int n = *nin;
  if (n > n_quad_max) return;
  const BinGeom geom{g.N, g.M, g.d, g.om};
  const int64_t M = g.M;
  const int lane = (int)(threadIdx.x & 31u);
  const Quad G{0xFu << (lane & ~3), lane & 3};
  for (int e0 = blockIdx.x * kGroups; e0 < n; e0 += gridDim.x * kGroups) {
    const int e = e0 + (int)(threadIdx.x >> 2);
    bool fail = false;
    int b = 0, k = 0;
    if (e < n) {
      const int2 qe = qin[e];
      b = qe.x;
      k = qe.y;
      const float4* Y = reinterpret_cast<const float4*>(g.Y) + (int64_t)b * g.held_elems;
      const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)g.ymax2[b]),
                     g.root_tol * g.root_tol, g.res_tol * g.res_tol};
      int64_t s[A];
      cdbl p[A];
      const bool ok = decode_quad<A, NM>(G, Y, nullptr, M, k, geom, tol, g.omff, s, p);
      if (G.q == 0) {
        if (ok)
          file_solution<FF, A>(s, p, M, g.slot_cnt + (int64_t)b * M, g.slot_s + (int64_t)b * M * kSlots,
                               reinterpret_cast<float4*>(g.slot_p) + (int64_t)b * M * kSlots,
                               g.flags + b);
        else if (qout == nullptr)
          g.T[(int64_t)b * M + k] = 1;
        else
          fail = true;
      }
    }
    if (qout != nullptr) queue_push(fail, b, k, qout, nout);
  }
}

// Bins with more than four aliases (sft_wide.cu): ITER level A - 1 >= 4
// (fold, then the warp-per-bin decoder), and the FIXED scan and rounds for
// a_max = 8 (rounds 1-4 as above on 16 syndromes, rounds 5-8 warp-per-bin).
void launch_level_wide(sft_plan_s* P, int A, const LevelArgs& g, int2* q, int* c, dim3 fgrid,
                       int64_t maxq, int nsm, cudaStream_t st, const char* fold_name,
                       const char* dec_name);
void launch_fixed_wide(sft_plan_s* P, int64_t B, const FixedArgs& g, int nsm, cudaStream_t st);

}  // namespace sft
