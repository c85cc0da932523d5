// sft_exact.cu -- kernels of the exactly K-sparse transform (Algorithm 1 and
// its non-iterative variant) for sm_103a, and their launch sequence.
//
// Per call, batched over B signals of one plan:
//   ITER, level l = 0 .. L-1 (M = M0 / 2^l, d = 2^l d0):
//     k_gather_fft   shifts 2l, 2l+1:  Y_{d,j} = d FFT_M(x[n d + j])
//                    (syndrome step of Algorithm 1), written into the level's buffer
//     k_iter_fold    one thread per bin: fold the held syndromes
//                    (Y_{2d,j}[k] = Y_{d,j}[k] + Y_{d,j}[k + M]), SubFreq on
//                    the two new shifts (SubFreq), the activity test
//                    of Algorithm 1; active bins are queued
//     k_iter_decode  SynDec with a = l + 1 (Algorithm 1) over the queue, so
//                    the FP64-heavy decode runs with full warps
//   FIXED: k_gather_fft for the 2 a_max shifts at d0, k_fixed_scan (queue
//          the active bins), k_fixed_round for a = 1 .. a_max (the bins no
//          smaller a decoded).
//   k_fin_count,     compact the recovered frequencies into the result in
//   k_finalize       two tiled passes (tile sums, then offsets + writes).
//
// Two arithmetic flavours F (sft_common.cuh): F64 everywhere on the plain
// path; on the mixed path (FF) the FFT, the folds, the peels and the
// activity tests run in float-float on the FP32 pipes, held syndromes and
// recovered values are stored as float-float, and only the per-bin solves
// (sft_decode.cuh) run in FP64.
#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "sft_decode.cuh"
#include "sft_device_util.cuh"
#include "sft_fft.cuh"
#include "sft_internal.h"
#include "sft_levels.cuh"

namespace sft {

// ----------------------------------------------------------- gather + FFT
template <class F, int PTS>
__global__ void __launch_bounds__(8192 / PTS) k_gather_fft(
    const typename F::In* __restrict__ x, int64_t x_stride, int64_t N, int64_t d, int64_t dscale,
    int log2M, int shift0, int log2Mt, const typename F::Tw* __restrict__ tw, void* __restrict__ out_v,
    int64_t out_sig, int64_t out_row, int row0, unsigned long long* __restrict__ ymax2,
    const int64_t* __restrict__ shift_list, const void* const* __restrict__ x_table) {
  extern __shared__ __align__(16) char smem[];
  typedef typename F::Out Out;
  const int b = blockIdx.y;
  const int js = blockIdx.x;
  // consecutive shifts shift0 + js, or an explicit list (random CS shifts)
  const int64_t shift = shift_list != nullptr ? shift_list[js] : shift0 + js;
  const int M = 1 << log2M;
  const int tid = threadIdx.x, nthr = blockDim.x;
  // signal b: base + b * stride, or its own pointer (heterogeneous batches)
  const typename F::In* xs = x_table != nullptr
                                 ? reinterpret_cast<const typename F::In*>(x_table[b])
                                 : x + (int64_t)b * x_stride;
  // x_{d,shift}[n] = x[(n d + shift) mod N]: every load of the thread is
  // issued before the first store (at most PTS per thread)
  typename F::In v[PTS];
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    const int n = tid + i * nthr;
    if (n < M) v[i] = __ldg(xs + (((int64_t)n * d + shift) & (N - 1)));
  }
  int done = 0;
  if (M == PTS * nthr) {
    // the first pass from registers (the gathered samples are its inputs)
    first_pass_regs<F, PTS>(smem, M, v, tid);
    done = 1;
  } else {
#pragma unroll
    for (int i = 0; i < PTS; ++i) {
      const int n = tid + i * nthr;
      if (n < M) F::st(smem, M, n, F::from_in(v[i]));
    }
  }
  __syncthreads();
  Out* o = reinterpret_cast<Out*>(out_v) + (int64_t)b * out_sig + (int64_t)(row0 + js) * out_row;
  double lmax = 0.0;
  float fmax_hi = 0.0f;
  // Y[k] = d FFT(x)[k] to the held rows (and max |Y|^2 for the zero
  // threshold), written by the FFT's last pass directly
  auto emit = [&](int k, const typename F::V& val) {
    if constexpr (std::is_same<F, F64>::value) {
      const double2 w = F::out(val, (double)dscale);
      o[k] = w;
      lmax = fmax(lmax, w.x * w.x + w.y * w.y);
    } else {
      const float4 w = F::out(val, (float)dscale);
      o[k] = w;
      fmax_hi = fmaxf(fmax_hi, F::out_norm_hi(w));
    }
  };
  // (below 256 points a CTA is one warp and the separate, coalesced output
  // loop measured faster)
  if (M < 256 || !cta_fft_out<F, PTS>(smem, log2M, log2Mt, tw, tid, nthr, done, emit)) {
    if (M < 256) {
      cta_fft<F, PTS>(smem, log2M, log2Mt, tw, tid, nthr, done);
      __syncthreads();
    }
    // the transform's result is in smem
    for (int k = tid; k < M; k += nthr) emit(k, F::ld(smem, M, k));
  }
  if constexpr (!std::is_same<F, F64>::value) lmax = (double)fmax_hi;
  if (ymax2 != nullptr && shift == 0) {
    // block max of |Y_{d,0}|^2 -> per-signal atomic max on the bit pattern
    // (non-negative doubles order like their unsigned bit patterns)
    __shared__ double wmax[32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o2));
    if ((tid & 31) == 0) wmax[tid >> 5] = lmax;
    __syncthreads();
    if (tid < 32) {
      double w = tid < (nthr >> 5) ? wmax[tid] : 0.0;
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o2));
      if (tid == 0) atomicMax(ymax2 + b, (unsigned long long)__double_as_longlong(w));
    }
  }
}

// --------------------------------------------------- input extraction
// The samples every FFT of one call reads, copied once into shift-major
// contiguous arrays: each row n of the level-0 grid (x[n d .. n d + 2a_m))
// is read by one thread, so its 64-byte run of shifts 0..7 (complex64)
// crosses the memory system once instead of once per level; the FFTs then
// read coalesced.  ITER: level l keeps [2][M_l] at offset
// sum_{l' < l} 2 M_l', rows n = 2^l n'; FIXED: [2 a_m][M0].
// Read-only load asking L2 for a 64-byte prefetch (a row's run of shifts
// 0..7 of complex64 samples), not the default wider one.
__device__ __forceinline__ float2 ld_row64(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L2::64B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_row64(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L2::64B.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}

template <class In>
__device__ __forceinline__ In ld_row(const In* p, bool narrow) {
  return narrow ? ld_row64(p) : __ldg(p);
}

// Two complex64 samples in one 16-byte load (p 16-byte aligned).
__device__ __forceinline__ float4 ld_pair(const float4* p, bool narrow) {
  if (!narrow) return __ldg(p);
  float4 v;
  asm volatile("ld.global.nc.L2::64B.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// The run of `cnt` (even, <= 16) samples x[n d + j], j < cnt, of one row:
// for complex64 rows that cannot wrap (d >= 16) and 16-byte aligned signals,
// as cnt / 2 16-byte loads; otherwise one load per sample.
template <class In, bool kNarrow, int CAP = 16>
__device__ __forceinline__ void load_run(const In* xs, int64_t n, int64_t d, int64_t N, int cnt,
                                         In* v) {
  if constexpr (std::is_same<In, float2>::value) {
    if (d >= 16 && (reinterpret_cast<uintptr_t>(xs) & 15u) == 0) {
      const float4* p = reinterpret_cast<const float4*>(xs + n * d);
#pragma unroll
      for (int j = 0; j < CAP / 2; ++j)
        if (2 * j < cnt) {
          const float4 q = ld_pair(p + j, kNarrow);
          v[2 * j] = make_float2(q.x, q.y);
          v[2 * j + 1] = make_float2(q.z, q.w);
        }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < CAP; ++j)
    if (j < cnt) v[j] = ld_row(xs + ((n * d + j) & (N - 1)), kNarrow);
}

// ITER: the levels row n feeds (rows n with n mod 2^l == 0 feed level l,
// shifts 2l and 2l + 1)
__device__ __forceinline__ int row_levels(int64_t n, int levels) {
  return min(levels, (n == 0 ? 8 : __ffsll(n) - 1 + 1));
}

// Row n's run v[0..cnt) into the level arrays cb of its signal: FIXED
// (fixed_nsh > 0) shift-major [fixed_nsh][M0]; ITER level l at offset
// sum_{l' < l} 2 M_l', entry n >> l.
template <class In, int CAP>
__device__ __forceinline__ void store_run(In* cb, int64_t n, int64_t M0, int fixed_nsh, int cnt,
                                          const In* v) {
  if (fixed_nsh > 0) {
#pragma unroll
    for (int j = 0; j < CAP; ++j)
      if (j < cnt) cb[(int64_t)j * M0 + n] = v[j];
    return;
  }
  int64_t off = 0, Ml = M0;
#pragma unroll
  for (int l = 0; l < CAP / 2; ++l) {
    if (2 * l < cnt) {
      cb[off + (n >> l)] = v[2 * l];
      cb[off + Ml + (n >> l)] = v[2 * l + 1];
    }
    off += 2 * Ml;
    Ml >>= 1;
  }
}

// CTAs per SM of the extraction from page-locked host memory
constexpr int kExtractHostCtas = 1;

// One row n of signal b: its run of shifts into the level arrays.
template <class In, bool kNarrow>
__device__ __forceinline__ void extract_row(const In* __restrict__ x, int64_t x_stride,
                                            const void* const* __restrict__ x_table, int64_t N,
                                            int64_t d, int64_t M0, int levels, int fixed_nsh,
                                            In* __restrict__ C, int64_t c_sig, int b, int64_t n) {
  const In* xs = x_table != nullptr ? reinterpret_cast<const In*>(x_table[b]) : x + (int64_t)b * x_stride;
  In v[16];
  const int cnt = fixed_nsh > 0 ? fixed_nsh : 2 * row_levels(n, levels);
  load_run<In, kNarrow>(xs, n, d, N, cnt, v);
  store_run<In, 16>(C + (int64_t)b * c_sig, n, M0, fixed_nsh, cnt, v);
}

// Device input: grid (row tiles, signals), one thread per row.  Input in
// page-locked host memory (kNarrow false, n_flat > 0): a bounded grid
// striding over the rows of all signals -- they arrive over the host link
// far slower than the SMs could take them, and CTAs waiting on the link for
// the whole extraction would hold every SM, leaving none for the compute of
// the call's other sub-batches (measured: more CTAs, or more rows in flight
// per thread, only slowed the call).
template <class In, bool kNarrow>
__global__ void __launch_bounds__(256) k_extract(const In* __restrict__ x, int64_t x_stride,
                                                 const void* const* __restrict__ x_table,
                                                 int64_t N, int64_t d, int64_t M0, int levels,
                                                 int fixed_nsh, In* __restrict__ C, int64_t c_sig,
                                                 int64_t n_flat) {
  if constexpr (!kNarrow) {
    if (n_flat > 0) {
      // grid-stride over the n_flat = signals x M0 rows (row f: signal f / M0,
      // M0 a power of two)
      const int lm0 = __ffsll(M0) - 1;
      for (int64_t f = (int64_t)blockIdx.x * 256 + threadIdx.x; f < n_flat;
           f += (int64_t)gridDim.x * 256)
        extract_row<In, kNarrow>(x, x_stride, x_table, N, d, M0, levels, fixed_nsh, C, c_sig,
                                 (int)(f >> lm0), f & (M0 - 1));
      return;
    }
  }
  const int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (n >= M0) return;
  extract_row<In, kNarrow>(x, x_stride, x_table, N, d, M0, levels, fixed_nsh, C, c_sig,
                           (int)blockIdx.y, n);
}

// ------------------------------------------- four-step FFT for M > 8192
// M = M1 M2 with n = n1 M2 + n2 and k = k1 + M1 k2:
//   A[k1][n2] = sum_{n1} x_d[n1 M2 + n2] e^{-2 pi i n1 k1 / M1}        (cols)
//   Y[k1 + M1 k2] = sum_{n2} A[k1][n2] e^{-2 pi i n2 k1 / M} e^{-2 pi i n2 k2 / M2}
// A CTA holds P = blockDim * PTS points: k_fft4_cols runs P/M1 column FFTs
// (each on M1/PTS threads) and writes twiddled rows W[k1][n2]; k_fft4_rows
// runs P/M2 row FFTs and writes Y (times d).  Both move data in coalesced
// runs.  With 8 points per thread P = max(4096, M1): two CTAs per SM, so
// that one CTA's loads overlap the other's butterflies.
constexpr int kFft4Points = 8192;  // largest one-CTA FFT; P of the 16-point form
constexpr int kFft4Cta8 = 4096;
// automatic sub-batching: as many sub-batches (up to 4) as hold this many
// signals each
constexpr int64_t kSubMinSignals = 32;

template <class F, int PTS>
__global__ void __launch_bounds__(8192 / PTS) k_fft4_cols(
    const typename F::In* __restrict__ x, int64_t x_stride, int64_t N, int64_t d, int log2M1,
    int log2M2, int shift0, int log2Mt, const typename F::Tw* __restrict__ tw,
    typename F::Out* __restrict__ W, int64_t w_sig, int nshift,
    const int64_t* __restrict__ shift_list, const void* const* __restrict__ x_table) {
  extern __shared__ __align__(16) char smem[];
  const int b = blockIdx.z, js = blockIdx.y;
  const int64_t shift = shift_list != nullptr ? shift_list[js] : shift0 + js;
  const int M1 = 1 << log2M1, M2 = 1 << log2M2;
  const int log2M = log2M1 + log2M2;
  const int CB = (int)(blockDim.x * PTS) >> log2M1;  // columns per CTA
  const int tpg = M1 / PTS;              // threads per column
  const int tid = threadIdx.x, g = tid / tpg, t = tid % tpg;
  const int c0 = blockIdx.x * CB;
  const typename F::In* xs = x_table != nullptr
                                 ? reinterpret_cast<const typename F::In*>(x_table[b])
                                 : x + (int64_t)b * x_stride;
  char* buf = smem + (size_t)g * padded(M1) * F::kBytesPerPoint;
  typename F::In v[PTS];
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    const int64_t n = (int64_t)(t + i * tpg) * M2 + c0 + g;
    v[i] = __ldg(xs + ((n * d + shift) & (N - 1)));
  }
  // the column's first pass from registers (tpg = M1 / PTS)
  first_pass_regs<F, PTS>(buf, M1, v, t);
  __syncthreads();
  // the twiddle e^{-2 pi i n2 k1 / M} (table of e^{-2 pi i q / Mt}, Mt >= M)
  // applied by the column FFT's last pass as it stores
  auto twiddled = [&](int k1, const typename F::V& val) {
    const int64_t q = ((int64_t)(c0 + g) * k1) & ((int64_t(1) << log2M) - 1);
    F::st(buf, M1, k1, F::mul_tw(val, __ldg(tw + (q << (log2Mt - log2M)))));
  };
  if (!cta_fft_st<F, PTS>(buf, log2M1, log2Mt, tw, t, tpg, 1, twiddled)) {
    for (int i = 0; i < PTS; ++i) {
      const int k1 = t + i * tpg;
      twiddled(k1, F::ld(buf, M1, k1));
    }
    __syncthreads();
  }
  typename F::Out* Wo = W + (int64_t)b * w_sig + (int64_t)js * ((int64_t)M1 * M2);
  const int lcb = __ffs(CB) - 1;  // CB, M1, M2, RB are powers of two: shifts and masks
  for (int idx = tid; idx < CB * M1; idx += blockDim.x) {
    const int k1 = idx >> lcb, c = idx & (CB - 1);
    const char* bc = smem + (size_t)c * padded(M1) * F::kBytesPerPoint;
    Wo[(int64_t)k1 * M2 + c0 + c] = F::out(F::ld(bc, M1, k1), 1);
  }
}

template <class F, int PTS>
__global__ void __launch_bounds__(8192 / PTS) k_fft4_rows(
    const typename F::Out* __restrict__ W, int64_t w_sig, int log2M1, int log2M2, int64_t d,
    int log2Mt, const typename F::Tw* __restrict__ tw, void* __restrict__ out_v, int64_t out_sig,
    int64_t out_row, int row0, unsigned long long* __restrict__ ymax2, int shift0) {
  extern __shared__ __align__(16) char smem[];
  typedef typename F::Out Out;
  const int b = blockIdx.z, js = blockIdx.y;
  const int M1 = 1 << log2M1, M2 = 1 << log2M2;
  const int RB = (int)(blockDim.x * PTS) >> log2M2;  // rows per CTA
  const int tpg = M2 / PTS;
  const int tid = threadIdx.x, g = tid / tpg, t = tid % tpg;
  const int r0 = blockIdx.x * RB;
  const Out* Wi = W + (int64_t)b * w_sig + (int64_t)js * ((int64_t)M1 * M2);
  const int lrb = __ffs(RB) - 1;  // RB and M2 are powers of two: shifts and masks
  for (int idx = tid; idx < RB * M2; idx += blockDim.x) {
    const int gg = idx >> log2M2, c = idx & (M2 - 1);
    char* bg = smem + (size_t)gg * padded(M2) * F::kBytesPerPoint;
    F::st(bg, M2, c, F::from_out(Wi[(int64_t)(r0 + gg) * M2 + c]));
  }
  __syncthreads();
  char* buf = smem + (size_t)g * padded(M2) * F::kBytesPerPoint;
  cta_fft<F, PTS>(buf, log2M2, log2Mt, tw, t, tpg);
  __syncthreads();
  Out* o = reinterpret_cast<Out*>(out_v) + (int64_t)b * out_sig + (int64_t)(row0 + js) * out_row;
  // running max of |Y|^2 in the output's own precision (FP32 hi parts on
  // the mixed path: no FP64 instruction per element)
  typename std::conditional<std::is_same<F, F64>::value, double, float>::type lmax_t = 0;
  const auto scale = (typename std::conditional<std::is_same<F, F64>::value, double, float>::type)d;
  for (int idx = tid; idx < RB * M2; idx += blockDim.x) {
    const int k2 = idx >> lrb, gg = idx & (RB - 1);
    const char* bg = smem + (size_t)gg * padded(M2) * F::kBytesPerPoint;
    const Out w = F::out(F::ld(bg, M2, k2), scale);
    o[(int64_t)(r0 + gg) + (int64_t)M1 * k2] = w;
    if constexpr (std::is_same<F, F64>::value)
      lmax_t = fmax(lmax_t, F::out_norm(w));
    else
      lmax_t = fmaxf(lmax_t, F::out_norm_hi(w));
  }
  double lmax = (double)lmax_t;
  if (ymax2 != nullptr && js == 0 && shift0 == 0) {
    __shared__ double wmax[32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o2));
    if ((tid & 31) == 0) wmax[tid >> 5] = lmax;
    __syncthreads();
    if (tid < 32) {
      double w = tid < (int)(blockDim.x >> 5) ? wmax[tid] : 0.0;
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o2));
      if (tid == 0) atomicMax(ymax2 + b, (unsigned long long)__double_as_longlong(w));
    }
  }
}

// ------------------------------------------------------------- finalize
struct FinArgs {
  int64_t M0, M_last;
  const uint8_t* slot_cnt;
  const int64_t* slot_s;
  const void* slot_p;
  const uint8_t* T_last;
  const int32_t* flags;
  int64_t cap;
  int64_t* idx;
  double2* val;
  int64_t* count;
  int32_t* unresolved;
  int32_t* overflow;
  const sft_result* r_table;  // per-signal result buffers (heterogeneous batches)
  int* tile_sum;              // [B][n_tiles]: entries filed in each tile of bins
  int* tile_un;               // [B][n_tiles]: unresolved bins of the last level per tile
  int n_tiles;
  int64_t tile_bins;          // bins per tile (kFinTile, or M0 for one tile per signal)
};

// bins per finalize tile (1024 threads x 4 bins)
constexpr int kFinTile = 4096;
// entries staged in shared memory per window of the finalize (24 KB)
constexpr int kFinStage = 1024;
// steps of 32 bins a warp of the device-resident finalize loads at once,
// and that finalize's largest CTA (registers for the steps' loads)
constexpr int kFinSteps = 4;
constexpr int kFinDevThreads = 512;

// Block-wide exclusive scan of one int per thread (blockDim = 1024).
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;  // inclusive prefix of warp sums
  }
  __syncthreads();
  const int before = (w > 0 ? wsum[w - 1] : 0) + x - v;
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// Finalize pass 1: per tile of kFinTile level-0 bins, the number of filed
// frequencies and of unresolved bins of the last level (coalesced reads).
__global__ void __launch_bounds__(256) k_fin_count(FinArgs g) {
  const int b = blockIdx.y, tile = blockIdx.x, tid = threadIdx.x;
  const int64_t k_lo = (int64_t)tile * g.tile_bins;
  const uint8_t* cnt = g.slot_cnt + (int64_t)b * g.M0;
  const uint8_t* T_ = g.T_last + (int64_t)b * g.M0;
  int c = 0, u = 0;
  for (int64_t k = k_lo + tid; k < min(k_lo + g.tile_bins, g.M0); k += 256) {
    c += cnt[k];
    if (k < g.M_last) u += T_[k];
  }
  __shared__ int sc[8], su[8];
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_xor_sync(0xffffffffu, c, o);
    u += __shfl_xor_sync(0xffffffffu, u, o);
  }
  if ((tid & 31) == 0) {
    sc[tid >> 5] = c;
    su[tid >> 5] = u;
  }
  __syncthreads();
  if (tid == 0) {
    int tc = 0, tu = 0;
    for (int w = 0; w < 8; ++w) {
      tc += sc[w];
      tu += su[w];
    }
    g.tile_sum[(int64_t)b * g.n_tiles + tile] = tc;
    g.tile_un[(int64_t)b * g.n_tiles + tile] = tu;
  }
}

// Finalize pass 2: each tile's entries go to its offset (sum of the earlier
// tiles) plus the block scan of its bins, in bin order; tile 0 writes the
// counters.
template <class F, bool kStaged>
__global__ void __launch_bounds__(kStaged ? 1024 : kFinDevThreads) k_finalize(FinArgs g) {
  typedef typename Store<F>::T T;
  const int b = blockIdx.y, tile = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t M0 = g.M0;
  const uint8_t* cnt = g.slot_cnt + (int64_t)b * M0;
  const T* sp = reinterpret_cast<const T*>(g.slot_p);
  __shared__ int s_base;
  if (tid < 32) {
    int acc = 0;
    for (int j = tid; j < tile; j += 32) acc += g.tile_sum[(int64_t)b * g.n_tiles + j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (tid == 0) s_base = acc;
  }
  const int64_t t_lo = (int64_t)tile * g.tile_bins, t_hi = min(t_lo + g.tile_bins, M0);
  int64_t cap = g.cap;
  int64_t* idx = g.idx + (int64_t)b * g.cap;
  double2* val = g.val + (int64_t)b * g.cap;
  int64_t* count = g.count + b;
  int32_t* unresolved = g.unresolved + b;
  int32_t* overflow = g.overflow + b;
  if (g.r_table != nullptr) {
    const sft_result& rt = g.r_table[b];
    cap = rt.cap;
    idx = rt.idx;
    val = reinterpret_cast<double2*>(rt.val);
    count = rt.count;
    unresolved = rt.unresolved;
    overflow = rt.overflow;
  }
  int total_tile = 0;
  if constexpr (!kStaged) {
    // device-resident results: warp w owns a chunk of consecutive bins of
    // the tile (a multiple of 32) and walks it 32 bins at a time, lane l on
    // bin k0 + l, so that the counts, the slots (slot e of consecutive bins
    // is contiguous) and the output runs are all accessed coalesced.  Each
    // warp's output offset is the block scan of the chunk totals; inside a
    // step, a shuffle scan of the 32 counts.
    const int lane = tid & 31, w = tid >> 5, nw = (int)(blockDim.x >> 5);
    const int64_t chunk = (t_hi - t_lo + 32 * nw - 1) / (32 * nw) * 32;
    const int64_t c_lo = min(t_lo + w * chunk, t_hi), c_hi = min(c_lo + chunk, t_hi);
    const uint8_t* __restrict__ cn = cnt;
    const int64_t* __restrict__ ssb = g.slot_s + (int64_t)b * M0 * kSlots;
    const T* __restrict__ spb = sp + (int64_t)b * M0 * kSlots;
    int wsum = 0;
    for (int64_t k = c_lo + lane; k < c_hi; k += 32) wsum += cn[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    // lane 0 of each warp carries the chunk total: its exclusive prefix is
    // the chunk's offset in the tile (synchronises: s_base visible)
    const int wpre = block_excl_scan(lane == 0 ? wsum : 0, &total_tile);
    int pos0 = s_base + __shfl_sync(0xffffffffu, wpre, 0);
    // kFinSteps steps of 32 bins at a time: their counts, then the first
    // entry of every bin of the group loaded before any is stored (more
    // loads in flight per warp), then the rare further entries
    for (int64_t k0 = c_lo; k0 < c_hi; k0 += 32 * kFinSteps) {
      int c[kFinSteps], pos[kFinSteps];
#pragma unroll
      for (int j = 0; j < kFinSteps; ++j) {
        const int64_t k = k0 + 32 * j + lane;
        c[j] = k < c_hi ? (int)cn[k] : 0;
      }
#pragma unroll
      for (int j = 0; j < kFinSteps; ++j) {
        int incl = c[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        pos[j] = pos0 + incl - c[j];
        pos0 += __shfl_sync(0xffffffffu, incl, 31);
      }
      int64_t s0[kFinSteps];
      T v0[kFinSteps];
#pragma unroll
      for (int j = 0; j < kFinSteps; ++j) {
        if (c[j] > 0) {
          const int64_t k = k0 + 32 * j + lane;
          s0[j] = ssb[slot_ix(k, 0, M0)];
          v0[j] = spb[slot_ix(k, 0, M0)];
        }
      }
#pragma unroll
      for (int j = 0; j < kFinSteps; ++j) {
        if (c[j] > 0 && pos[j] < cap) {
          const cdbl v = Store<F>::to_d(v0[j]);
          idx[pos[j]] = s0[j];
          val[pos[j]] = make_double2(v.x, v.y);
        }
      }
#pragma unroll
      for (int j = 0; j < kFinSteps; ++j) {
        const int64_t k = k0 + 32 * j + lane;
        for (int e = 1; e < c[j]; ++e) {
          if (pos[j] + e < cap) {
            const int64_t s_e = ssb[slot_ix(k, e, M0)];
            const cdbl v = Store<F>::to_d(spb[slot_ix(k, e, M0)]);
            idx[pos[j] + e] = s_e;
            val[pos[j] + e] = make_double2(v.x, v.y);
          }
        }
      }
    }
  }
  // results in page-locked host memory (written over the host link): the
  // tile's entries form one contiguous run [base, base + total_tile) of the
  // output; they are gathered in shared memory in windows of kFinStage and
  // written out by consecutive threads, so that the stores are coalesced
  __shared__ int64_t s_idx[kStaged ? kFinStage : 1];
  __shared__ double2 s_val[kStaged ? kFinStage : 1];
  int64_t lo = 0, hi = 0;
  int mine = 0, lpos = 0;
  if constexpr (kStaged) {
    const int64_t per = (g.tile_bins + blockDim.x - 1) / blockDim.x;
    lo = min(t_lo + per * tid, t_hi);
    hi = min(lo + per, t_hi);
    for (int64_t k0 = lo; k0 < hi; ++k0) mine += cnt[k0];
    lpos = block_excl_scan(mine, &total_tile);  // synchronises: s_base visible
  }
  const int base = s_base;
  for (int w0 = 0; kStaged && w0 < total_tile; w0 += kFinStage) {
    if (lpos < w0 + kFinStage && lpos + mine > w0) {
      int p = lpos;
      for (int64_t k0 = lo; k0 < hi && p < w0 + kFinStage; ++k0) {
        const int c = cnt[k0];
        for (int e = 0; e < c; ++e, ++p) {
          if (p >= w0 && p < w0 + kFinStage) {
            s_idx[p - w0] = g.slot_s[(int64_t)b * M0 * kSlots + slot_ix(k0, e, M0)];
            const cdbl v = Store<F>::to_d(sp[(int64_t)b * M0 * kSlots + slot_ix(k0, e, M0)]);
            s_val[p - w0] = make_double2(v.x, v.y);
          }
        }
      }
    }
    __syncthreads();
    const int n = min(kFinStage, total_tile - w0);
    for (int i = tid; i < n; i += blockDim.x) {
      const int64_t gp = (int64_t)base + w0 + i;
      if (gp < cap) {
        idx[gp] = s_idx[i];
        val[gp] = s_val[i];
      }
    }
    __syncthreads();
  }
  if (g.n_tiles == 1) {
    // one tile per signal (no count pass): the unresolved bins here
    int un = 0;
    const uint8_t* T_ = g.T_last + (int64_t)b * M0;
    for (int64_t k = tid; k < g.M_last; k += blockDim.x) un += T_[k];
    int un_total = 0;
    (void)block_excl_scan(un, &un_total);
    if (tid == 0) {
      *count = total_tile < cap ? total_tile : cap;
      *unresolved = un_total;
      *overflow = (total_tile > cap || (g.flags[b] & 1)) ? 1 : 0;
    }
  } else if (tile == 0 && tid == 0) {
    int64_t total = 0, un = 0;
    for (int j = 0; j < g.n_tiles; ++j) {
      total += g.tile_sum[(int64_t)b * g.n_tiles + j];
      un += g.tile_un[(int64_t)b * g.n_tiles + j];
    }
    *count = total < cap ? total : cap;
    *unresolved = (int32_t)un;
    *overflow = (total > cap || (g.flags[b] & 1)) ? 1 : 0;
  }
}

// ------------------------------------------------------------ launchers
static int fft_threads(int log2M, int pts) {
  const int M = 1 << log2M;
  return M / pts > 32 ? M / pts : 32;
}

// The opt-in shared-memory limit is a property of the kernel, shared by every
// plan alive: it is raised once to the largest tile any plan launches
// (kFft4Points points), never lowered to one plan's size.  Occupancy follows
// the shared memory each launch actually requests.
template <class F>
static cudaError_t prepare_kernels_t() {
  const int smem = padded(kFft4Points) * 16;
  cudaError_t e = cudaFuncSetAttribute(k_gather_fft<F, 16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gather_fft<F, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft4_cols<F, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft4_rows<F, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft4_cols<F, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fft4_rows<F, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

cudaError_t prepare_kernels(sft_plan_s* P) {
  return P->p.precision == SFT_FP64 ? prepare_kernels_t<F64>() : prepare_kernels_t<FF>();
}

// one finalize tile per signal when the signals alone fill the GPU
static bool fin_single(const sft_plan_s* P, int64_t B, int nsm) {
  return B >= nsm && P->M0 <= 65536;
}

int sub_batches_for(const sft_plan_s* P, int64_t B);

// launches of one sub-batch of B signals
static int launches_one(const sft_plan_s* P, int64_t B, int nsm, bool quad) {
  const int fin = fin_single(P, B, nsm) ? 1 : 2;
  if (P->p.mode == SFT_GENERAL_UNPRUNED) return (P->M0 > kFft4Points ? 2 : 1) + 1 + fin;
  if (P->p.mode == SFT_GENERAL)
    return 2 * (P->M0 > kFft4Points ? 2 : 1) + 5 + (P->p.a_max >= 2 ? 2 : 1) +
           (P->mlp != nullptr ? 1 : 0) + fin;
  const int ext = P->ws.xc != nullptr ? 1 : 0;
  // with `quad`, the mixed path launches a four-lane decoder beside the
  // one-lane decoder of three and four aliases
  const bool q4 = quad && P->p.precision != SFT_FP64;
  if (P->p.mode == SFT_EXACT_FIXED) {
    const int nq = q4 && P->p.a_max <= 4 ? std::max(0, P->p.a_max - 2) : 0;
    return ext + (P->M0 > kFft4Points ? 2 : 1) + 1 + P->p.a_max + nq + fin;
  }
  int fft = 0;
  for (int l = 0; l < P->levels; ++l) fft += (P->M0 >> l) > kFft4Points ? 2 : 1;
  const int nq = q4 ? std::max(0, std::min(P->levels, 4) - 2) : 0;
  return ext + fft + 2 * P->levels + nq + fin;
}

int launches_per_call(const sft_plan_s* P) {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t B = P->max_signals;
  const int S = sub_batches_for(P, B);
  int n = 0;
  const bool quad = P->quad_ok && S <= 1;
  for (int s = 0; s < S; ++s) n += launches_one(P, B / S + (s < B % S ? 1 : 0), nsm, quad);
  return n;
}

static cudaEvent_t pool_event(sft_plan_s* P) {
  if (P->events_used == P->event_pool.size()) {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    P->event_pool.push_back(e);
  }
  return P->event_pool[P->events_used++];
}

void stage_begin(sft_plan_s* P, const char* name, cudaStream_t st) {
  if (!P->profiling) return;
  StageRec r{name, pool_event(P), pool_event(P), P->cur_sub};
  cudaEventRecord(r.t0, st);
  P->stage_recs.push_back(r);
}

void stage_end(sft_plan_s* P, cudaStream_t st) {
  if (!P->profiling || P->stage_recs.empty()) return;
  cudaEventRecord(P->stage_recs.back().t1, st);
}

// Where the gather reads: sample n of shift s of signal b is
// src.x[(n src.d + s) & (src.N - 1)] of that signal (src.table[b], or
// src.x + b src.stride).
struct GatherSrc {
  const void* x;
  int64_t stride, N, d;
  const void* const* table;
};

template <class F>
void launch_gather_fft(sft_plan_s* P, int64_t B, const GatherSrc& src, int64_t dscale, int log2M,
                       int shift0, int nshift, void* out, int64_t out_row, int row0,
                       bool want_ymax, cudaStream_t st, const int64_t* shift_list,
                       const char* stage) {
  static const char* names[] = {"gather_fft_l0", "gather_fft_l1", "gather_fft_l2", "gather_fft_l3",
                                "gather_fft_l4", "gather_fft_l5", "gather_fft_l6", "gather_fft_l7"};
  static const char* cnames[] = {"gather_cols_l0", "gather_cols_l1", "gather_cols_l2",
                                 "gather_cols_l3", "gather_cols_l4", "gather_cols_l5",
                                 "gather_cols_l6", "gather_cols_l7"};
  static const char* rnames[] = {"fft_rows_l0", "fft_rows_l1", "fft_rows_l2", "fft_rows_l3",
                                 "fft_rows_l4", "fft_rows_l5", "fft_rows_l6", "fft_rows_l7"};
  const int lvl = nshift > 2 ? 0 : shift0 / 2;
  const auto* xin = reinterpret_cast<const typename F::In*>(src.x);
  const auto* tw = reinterpret_cast<const typename F::Tw*>(P->tab.tw);
  if ((1 << log2M) <= kFft4Points) {
    dim3 grid(nshift, (unsigned)B);
    const int pts = P->fft_pts;
    const int nthr = fft_threads(log2M, pts);
    const size_t smem = (size_t)padded(1 << log2M) * F::kBytesPerPoint;
    stage_begin(P, stage ? stage : (nshift > 2 ? "gather_fft_fixed" : names[lvl]), st);
    if (pts == 8)
      k_gather_fft<F, 8><<<grid, nthr, smem, st>>>(xin, src.stride, src.N, src.d, dscale, log2M,
                                                   shift0, P->log2M0, tw, out, P->ws.held_elems,
                                                   out_row, row0,
                                                   want_ymax ? P->ws.ymax2 : nullptr, shift_list,
                                                   src.table);
    else
      k_gather_fft<F, 16><<<grid, nthr, smem, st>>>(xin, src.stride, src.N, src.d, dscale, log2M,
                                                    shift0, P->log2M0, tw, out, P->ws.held_elems,
                                                    out_row, row0,
                                                    want_ymax ? P->ws.ymax2 : nullptr, shift_list,
                                                    src.table);
    stage_end(P, st);
    return;
  }
  // four-step: columns of length M1, rows of length M2, M1 >= M2
  const int log2M2 = log2M / 2, log2M1 = log2M - log2M2;
  const int64_t Mlev = int64_t(1) << log2M;
  const int pcta = P->fft_pts == 8 ? std::max(kFft4Cta8, 1 << log2M1) : kFft4Points;
  const unsigned ctas = (unsigned)(Mlev / pcta);
  const size_t smem = (size_t)padded(pcta) * F::kBytesPerPoint;
  auto* W = reinterpret_cast<typename F::Out*>(P->ws.fft4);
  const int64_t w_sig = (int64_t)nshift * Mlev;
  const dim3 grid4(ctas, nshift, (unsigned)B);
  stage_begin(P, stage ? stage : cnames[lvl], st);
  if (P->fft_pts == 8)
    k_fft4_cols<F, 8><<<grid4, pcta / 8, smem, st>>>(xin, src.stride, src.N, src.d, log2M1, log2M2,
                                                 shift0, P->log2M0, tw, W, w_sig, nshift,
                                                 shift_list, src.table);
  else
    k_fft4_cols<F, 16><<<grid4, 512, smem, st>>>(xin, src.stride, src.N, src.d, log2M1, log2M2,
                                                 shift0, P->log2M0, tw, W, w_sig, nshift,
                                                 shift_list, src.table);
  stage_end(P, st);
  stage_begin(P, stage ? "fft_rows" : rnames[lvl], st);
  if (P->fft_pts == 8)
    k_fft4_rows<F, 8><<<grid4, pcta / 8, smem, st>>>(W, w_sig, log2M1, log2M2, dscale, P->log2M0, tw,
                                                 out, P->ws.held_elems, out_row, row0,
                                                 want_ymax ? P->ws.ymax2 : nullptr, shift0);
  else
    k_fft4_rows<F, 16><<<grid4, 512, smem, st>>>(W, w_sig, log2M1, log2M2, dscale, P->log2M0, tw,
                                                 out, P->ws.held_elems, out_row, row0,
                                                 want_ymax ? P->ws.ymax2 : nullptr, shift0);
  stage_end(P, st);
}

void launch_gather_fft_any(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int64_t d,
                           int log2M, int shift0, int nshift, void* out, int64_t out_row, int row0,
                           bool want_ymax, cudaStream_t st, const int64_t* shift_list,
                           const char* stage) {
  const GatherSrc src{x, x_stride, P->p.N, d, P->x_table};
  if (P->p.precision == SFT_FP64)
    launch_gather_fft<F64>(P, B, src, d, log2M, shift0, nshift, out, out_row, row0, want_ymax, st,
                           shift_list, stage);
  else
    launch_gather_fft<FF>(P, B, src, d, log2M, shift0, nshift, out, out_row, row0, want_ymax, st,
                          shift_list, stage);
}

// Copies the samples of the call into the compact arrays (P->ws.xc).
template <class F>
static void launch_extract(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int levels,
                           int fixed_nsh, int nsm, cudaStream_t st) {
  const dim3 grid((unsigned)((P->M0 + 255) / 256), (unsigned)B);
  stage_begin(P, "extract", st);
  // device-resident samples: 64-byte L2 requests (one row's run of shifts);
  // host-resident ones (read over NVLink-C2C): full-width requests, from a
  // grid of kExtractHostCtas CTAs per SM striding over all rows
  if (P->x_on_host) {
    const int64_t rows = B * P->M0;
    const unsigned hgrid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((rows + 255) / 256, (int64_t)kExtractHostCtas * nsm));
    k_extract<typename F::In, false><<<hgrid, 256, 0, st>>>(
        reinterpret_cast<const typename F::In*>(x), x_stride, P->x_table, P->p.N, P->p.d, P->M0,
        levels, fixed_nsh, reinterpret_cast<typename F::In*>(P->ws.xc), P->ws.xc_sig, rows);
  } else {
    k_extract<typename F::In, true><<<grid, 256, 0, st>>>(
        reinterpret_cast<const typename F::In*>(x), x_stride, P->x_table, P->p.N, P->p.d, P->M0,
        levels, fixed_nsh, reinterpret_cast<typename F::In*>(P->ws.xc), P->ws.xc_sig, 0);
  }
  stage_end(P, st);
  if (P->sub_extract_now != nullptr) cudaEventRecord(P->sub_extract_now, st);
}

// Queues of at most quad_max_bins bins (64 per SM) go to the four-lane
// decoders of three and four aliases: below that the one-lane decoder's
// warps leave most SM sub-partitions idle and its per-bin FP64 chain sets the
// time; above it the four-lane decoder's extra FP64 issue slots do.
static int quad_max_bins(int nsm) { return 64 * nsm; }
static unsigned quad_grid(const sft_plan_s* P, int64_t maxq, int nsm) {
  constexpr int kGroups = kDecThreads / 4;
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(maxq, quad_max_bins(nsm)) / kGroups + 1,
                           (int64_t)P->dec_ctas_per_sm * nsm));
}

template <class F>
static void launch_fixed(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                         const OmegaTab& om, int nsm, cudaStream_t st) {
  const Workspace& W = P->ws;
  const int nsh = 2 * P->p.a_max;
  if (W.xc != nullptr) {
    // rows j M0 .. of the compact array hold shift j (index space rounded
    // up to a power of two)
    launch_extract<F>(P, B, x, x_stride, 0, nsh, nsm, st);
    int64_t Nc = P->M0;
    while (Nc < nsh * P->M0) Nc <<= 1;
    const GatherSrc src{W.xc, W.xc_sig, Nc, 1, nullptr};
    launch_gather_fft<F>(P, B, src, P->p.d, P->log2M0, 0, nsh, W.held[0], P->M0, 0, true, st,
                         P->tab.xc_shifts, nullptr);
  } else {
    const GatherSrc src{x, x_stride, P->p.N, P->p.d, P->x_table};
    launch_gather_fft<F>(P, B, src, P->p.d, P->log2M0, 0, nsh, W.held[0], P->M0, 0, true, st,
                         nullptr, nullptr);
  }
  FixedArgs g{P->p.N, P->M0, P->p.d, P->p.a_max, W.held[0], W.held_elems, W.T[0], W.slot_cnt,
              W.slot_s, W.slot_p, W.ymax2, W.flags, P->p.zero_tol, P->p.root_tol,
              P->p.res_tol, om,
              OmegaTabFF{P->tab.om_hi_ff, P->tab.om_lo_ff, P->tab.om_lo_bits, P->p.N - 1},
              (float)(P->p.zero_tol * P->p.zero_tol), (float)(P->p.root_tol * P->p.root_tol),
              (float)(P->p.res_tol * P->p.res_tol)};
  if (P->p.a_max > 4) {
    // a_max = 8: 16 syndromes, rounds 5-8 by the warp-per-bin decoder
    launch_fixed_wide(P, B, g, nsm, st);
    return;
  }
  dim3 sgrid((unsigned)((P->M0 + kFoldThreads - 1) / kFoldThreads), (unsigned)B);
  const int64_t maxq = B * P->M0;
  const unsigned dgrid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((maxq + kDecThreads - 1) / kDecThreads, (int64_t)P->dec_ctas_per_sm * nsm));
  int2* q0 = W.queue[0];
  int2* q1 = W.queue[1];
  int* c = W.qcount;
  stage_begin(P, "decode_fixed_scan", st);
  switch (P->p.a_max) {
    case 1: k_fixed_scan<F, 2><<<sgrid, kFoldThreads, 0, st>>>(g, q0, c); break;
    case 2: k_fixed_scan<F, 4><<<sgrid, kFoldThreads, 0, st>>>(g, q0, c); break;
    case 3: k_fixed_scan<F, 6><<<sgrid, kFoldThreads, 0, st>>>(g, q0, c); break;
    default: k_fixed_scan<F, 8><<<sgrid, kFoldThreads, 0, st>>>(g, q0, c); break;
  }
  stage_end(P, st);
  static const char* rnames[] = {"decode_fixed_a1", "decode_fixed_a2", "decode_fixed_a3",
                                 "decode_fixed_a4"};
  // round a reads queue (a-1)&1 / counter a-1, writes queue a&1 / counter a
  auto round = [&](auto a_tag, auto nm_tag) {
    constexpr int A = decltype(a_tag)::value, NM = decltype(nm_tag)::value;
    const bool last = A == P->p.a_max;
    stage_begin(P, rnames[A - 1], st);
    const int2* qi = (A & 1) ? q0 : q1;
    int2* qo = last ? nullptr : ((A & 1) ? q1 : q0);
    int* co = last ? nullptr : c + A;
    // three and four aliases on the mixed path: the queue length picks the
    // one-lane or the four-lane round on the device
    constexpr bool kQuad = std::is_same<F, FF>::value && A >= 3;
    const int nq = kQuad && P->quad_now ? quad_max_bins(nsm) : -1;
    k_fixed_round<F, A, NM><<<dgrid, kDecThreads, 0, st>>>(g, qi, c + (A - 1), qo, co, nq);
    if constexpr (kQuad) {
      if (nq >= 0)
        k_fixed_round_quad<A, NM><<<quad_grid(P, maxq, nsm), kDecThreads, 0, st>>>(g, qi, c + (A - 1),
                                                                                qo, co, nq);
    }
    stage_end(P, st);
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  switch (P->p.a_max) {
    case 1: round(I1{}, std::integral_constant<int, 2>{}); break;
    case 2:
      round(I1{}, std::integral_constant<int, 4>{});
      round(I2{}, std::integral_constant<int, 4>{});
      break;
    case 3:
      round(I1{}, std::integral_constant<int, 6>{});
      round(I2{}, std::integral_constant<int, 6>{});
      round(I3{}, std::integral_constant<int, 6>{});
      break;
    default:
      round(I1{}, std::integral_constant<int, 8>{});
      round(I2{}, std::integral_constant<int, 8>{});
      round(I3{}, std::integral_constant<int, 8>{});
      round(I4{}, std::integral_constant<int, 8>{});
      break;
  }
}

template <class F>
static void launch_iter(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                        const OmegaTab& om, int nsm, cudaStream_t st, int64_t* M_last,
                        const uint8_t** T_last) {
  const Workspace& W = P->ws;
  const OmegaTabFF omff{P->tab.om_hi_ff, P->tab.om_lo_ff, P->tab.om_lo_bits, P->p.N - 1};
  int64_t M = P->M0, d = P->p.d, xc_off = 0;
  if (W.xc != nullptr) launch_extract<F>(P, B, x, x_stride, P->levels, 0, nsm, st);
  for (int l = 0; l < P->levels; ++l) {
    if (l > 0) {
      xc_off += 2 * M;
      M >>= 1;
      d <<= 1;
    }
    const int log2M = P->log2M0 - l;
    void* cur = W.held[l & 1];
    const void* prev = W.held[(l + 1) & 1];
    if (W.xc != nullptr) {
      // level l's two shifts are rows 0 and M of its block
      const GatherSrc src{reinterpret_cast<const typename F::In*>(W.xc) + xc_off, W.xc_sig, 2 * M,
                          1, nullptr};
      launch_gather_fft<F>(P, B, src, d, log2M, 2 * l, 2, cur, M, 2 * l, l == 0, st,
                           P->tab.xc_shifts + 2 * l, nullptr);
    } else {
      const GatherSrc src{x, x_stride, P->p.N, d, P->x_table};
      launch_gather_fft<F>(P, B, src, d, log2M, 2 * l, 2, cur, M, 2 * l, l == 0, st, nullptr,
                           nullptr);
    }
    LevelArgs g{P->p.N, M, d, P->M0, prev, cur, W.held_elems, W.T[(l + 1) & 1], W.T[l & 1],
                W.slot_cnt, W.slot_s, W.slot_p, W.ymax2, W.flags, P->p.zero_tol,
                P->p.root_tol, P->p.res_tol, om, omff, (float)(P->p.zero_tol * P->p.zero_tol),
                (float)(P->p.root_tol * P->p.root_tol), (float)(P->p.res_tol * P->p.res_tol)};
    int2* q = W.queue[l & 1];
    int* c = W.qcount + l;
    dim3 fgrid((unsigned)((M + kFoldThreads - 1) / kFoldThreads), (unsigned)B);
    // fewer bins than a CTA's threads: signals packed densely over the grid
    const int64_t n_flat = M < kFoldThreads ? B * M : 0;
    const dim3 fgrid_fold =
        n_flat > 0 ? dim3((unsigned)((n_flat + kFoldThreads - 1) / kFoldThreads), 1u) : fgrid;
    const int64_t maxq = B * M;
    const unsigned dgrid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((maxq + kDecThreads - 1) / kDecThreads, (int64_t)P->dec_ctas_per_sm * nsm));
    static const char* fnames[] = {"fold_l0", "fold_l1", "fold_l2", "fold_l3",
                                   "fold_l4", "fold_l5", "fold_l6", "fold_l7"};
    static const char* dnames[] = {"decode_l0", "decode_l1", "decode_l2", "decode_l3",
                                   "decode_l4", "decode_l5", "decode_l6", "decode_l7"};
    if (l >= 4) {
      // more than four aliases: Berlekamp-Massey and the candidate search
      launch_level_wide(P, l + 1, g, q, c, fgrid, maxq, nsm, st, fnames[l], dnames[l]);
      *M_last = M;
      *T_last = W.T[l & 1];
      continue;
    }
    stage_begin(P, fnames[l], st);
    switch (l) {
      case 0: k_iter_fold<F, 1><<<fgrid_fold, kFoldThreads, 0, st>>>(g, q, c, n_flat); break;
      case 1: k_iter_fold<F, 2><<<fgrid_fold, kFoldThreads, 0, st>>>(g, q, c, n_flat); break;
      case 2: k_iter_fold<F, 3><<<fgrid_fold, kFoldThreads, 0, st>>>(g, q, c, n_flat); break;
      default: k_iter_fold<F, 4><<<fgrid_fold, kFoldThreads, 0, st>>>(g, q, c, n_flat); break;
    }
    stage_end(P, st);
    stage_begin(P, dnames[l], st);
    // three and four aliases on the mixed path: both decoders are launched
    // and the queue length, read on the device, picks one (quad_grid)
    constexpr bool kQuad = std::is_same<F, FF>::value;
    const int nq = kQuad && P->quad_now ? quad_max_bins(nsm) : -1;
    switch (l) {
      case 0: k_iter_decode<F, 1><<<dgrid, kDecThreads, 0, st>>>(g, q, c); break;
      case 1: k_iter_decode<F, 2><<<dgrid, kDecThreads, 0, st>>>(g, q, c); break;
      case 2:
        k_iter_decode<F, 3><<<dgrid, kDecThreads, 0, st>>>(g, q, c, nq);
        if (nq >= 0) k_iter_decode_quad<3><<<quad_grid(P, maxq, nsm), kDecThreads, 0, st>>>(g, q, c, nq);
        break;
      default:
        k_iter_decode<F, 4><<<dgrid, kDecThreads, 0, st>>>(g, q, c, nq);
        if (nq >= 0) k_iter_decode_quad<4><<<quad_grid(P, maxq, nsm), kDecThreads, 0, st>>>(g, q, c, nq);
        break;
    }
    stage_end(P, st);
    *M_last = M;
    *T_last = W.T[l & 1];
  }
}

static cudaError_t launch_one(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                              const sft_result* r, cudaStream_t st) {
  const Workspace& W = P->ws;
  const OmegaTab om{P->tab.om_hi, P->tab.om_lo, P->tab.om_lo_bits, P->p.N - 1};
  const bool fp64 = P->p.precision == SFT_FP64;
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t M_last = P->M0;
  const uint8_t* T_last = W.T[0];
  if (is_general_mode(P->p.mode)) {
    launch_general(P, B, x, x_stride, nsm, st);
    M_last = 0;  // no unsolved-bin flags on the general path
  } else if (P->p.mode == SFT_EXACT_FIXED) {
    if (fp64)
      launch_fixed<F64>(P, B, x, x_stride, om, nsm, st);
    else
      launch_fixed<FF>(P, B, x, x_stride, om, nsm, st);
  } else {
    if (fp64)
      launch_iter<F64>(P, B, x, x_stride, om, nsm, st, &M_last, &T_last);
    else
      launch_iter<FF>(P, B, x, x_stride, om, nsm, st, &M_last, &T_last);
  }
  // One tile per signal when the signals alone fill the GPU (and a thread
  // walks at most 64 bins); else tiles of kFinTile bins, whose sums live in
  // the second queue (free once the decoders are done).
  const bool single = fin_single(P, B, nsm);
  const int n_tiles = single ? 1 : (int)((P->M0 + kFinTile - 1) / kFinTile);
  int* tiles = reinterpret_cast<int*>(W.queue[1]);
  FinArgs f{P->M0,    M_last,   W.slot_cnt, W.slot_s, W.slot_p, T_last, W.flags, r->cap, r->idx,
            reinterpret_cast<double2*>(r->val), r->count, r->unresolved, r->overflow, P->r_table,
            tiles,    tiles + B * n_tiles, n_tiles, single ? P->M0 : (int64_t)kFinTile};
  const dim3 fgrid((unsigned)n_tiles, (unsigned)B);
  // at most 1024 threads (results in host memory, staged) or
  // kFinDevThreads; a tile of fewer bins gets whole warps, a thread per bin
  const int fmax = P->r_on_host ? 1024 : kFinDevThreads;
  const int fthr = single ? (int)std::min<int64_t>(fmax, std::max<int64_t>(32, (P->M0 + 31) / 32 * 32))
                          : fmax;
  stage_begin(P, "finalize", st);
  if (!single) k_fin_count<<<fgrid, 256, 0, st>>>(f);
  if (fp64)
    P->r_on_host ? k_finalize<F64, true><<<fgrid, fthr, 0, st>>>(f)
                 : k_finalize<F64, false><<<fgrid, fthr, 0, st>>>(f);
  else
    P->r_on_host ? k_finalize<FF, true><<<fgrid, fthr, 0, st>>>(f)
                 : k_finalize<FF, false><<<fgrid, fthr, 0, st>>>(f);
  stage_end(P, st);
  return cudaGetLastError();
}

int sub_batches_for(const sft_plan_s* P, int64_t B) {
  if (P->sub_fork == nullptr) return 1;  // a plan without streams (sft_exact_noalloc)
  int S = P->sub_batches;
  if (S <= 0) S = (int)std::min<int64_t>(kMaxSub, std::max<int64_t>(1, B / kSubMinSignals));
  if (S > kMaxSub) S = kMaxSub;
  if (S > B) S = (int)std::max<int64_t>(B, 1);
  return S;
}

// Splits the call into sub-batches of consecutive signals, each enqueued on
// its own stream after a fork from `st` and joined back into `st`: the
// latency-bound stages of one sub-batch (the decoders of the later levels,
// FP64-pipe bound and few warps) run beside the FFTs of another (FP32
// pipes).  Each sub-batch works in its own slice of the workspace.
cudaError_t launch_exact(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                         const sft_result* r, cudaStream_t st) {
  const int S = sub_batches_for(P, B);
  P->last_sub = S;
  P->quad_now = P->quad_ok && S <= 1;
  if (S <= 1) return launch_one(P, B, x, x_stride, r, st);
  cudaError_t e = cudaSuccess;
  const size_t esize = P->p.precision == SFT_FP64 ? 16 : 8;
  const Workspace W0 = P->ws;
  const void* const* xt0 = P->x_table;
  const sft_result* rt0 = P->r_table;
  const int64_t* kt0 = P->K_table;
  int16_t* prop0 = P->mlp_prop;
  e = cudaEventRecord(P->sub_fork, st);
  int64_t b0 = 0;
  for (int s = 0; s < S && e == cudaSuccess; ++s) {
    const int64_t Bs = B / S + (s < B % S ? 1 : 0);
    cudaStream_t ss = s == 0 ? st : P->sub_st[s];
    if (s > 0) e = cudaStreamWaitEvent(ss, P->sub_fork, 0);
    // host-resident input: extract after the previous sub-batch has
    if (e == cudaSuccess && s > 0 && P->x_on_host)
      e = cudaStreamWaitEvent(ss, P->sub_extracted[s - 1], 0);
    if (e != cudaSuccess) break;
    if (P->x_on_host) {
      // recorded again after the extraction (a mode without one still
      // releases the next sub-batch)
      P->sub_extract_now = P->sub_extracted[s];
      e = cudaEventRecord(P->sub_extract_now, ss);
      if (e != cudaSuccess) break;
    }
    P->ws = sub_workspace(W0, b0, s);
    P->cur_sub = s;
    P->x_table = xt0 ? xt0 + b0 : nullptr;
    P->r_table = rt0 ? rt0 + b0 : nullptr;
    P->K_table = kt0 ? kt0 + b0 : nullptr;
    P->mlp_prop = prop0 ? prop0 + b0 * P->M0 * 8 : nullptr;
    sft_result rs = *r;
    if (r->idx) rs.idx = r->idx + b0 * r->cap;
    if (r->val) rs.val = r->val + 2 * b0 * r->cap;
    if (r->count) rs.count = r->count + b0;
    if (r->unresolved) rs.unresolved = r->unresolved + b0;
    if (r->overflow) rs.overflow = r->overflow + b0;
    const void* xs = x ? static_cast<const char*>(x) + (size_t)b0 * (size_t)x_stride * esize : x;
    e = launch_one(P, Bs, xs, x_stride, &rs, ss);
    if (e == cudaSuccess && s > 0) e = cudaEventRecord(P->sub_join[s], ss);
    b0 += Bs;
  }
  P->ws = W0;
  P->cur_sub = 0;
  P->x_table = xt0;
  P->r_table = rt0;
  P->K_table = kt0;
  P->mlp_prop = prop0;
  P->sub_extract_now = nullptr;
  for (int s = 1; s < S && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(st, P->sub_join[s], 0);
  return e;
}

}  // namespace sft
