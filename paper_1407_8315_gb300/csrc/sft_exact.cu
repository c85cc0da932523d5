// sft_exact.cu -- kernels of the exactly K-sparse transform (Algorithm 1 and
// its non-iterative variant) for sm_103a, and their launch sequence.
//
// Per call, batched over B signals of one plan:
//   ITER, level l = 0 .. L-1 (M = M0 / 2^l, d = 2^l d0):
//     k_gather_fft   shifts 2l, 2l+1:  Y_{d,j} = d FFT_M(x[n d + j])
//                    (Alg. 1 lines 03-06), written into the level's buffer
//     k_iter_level   one thread per bin: fold the held syndromes
//                    (Y_{2d,j}[k] = Y_{d,j}[k] + Y_{d,j}[k + M]), SubFreq on
//                    the two new shifts (lines 17-22), the activity test
//                    (line 09), SynDec with a = l + 1 (lines 23-35)
//   FIXED: k_gather_fft for the 2 a_max shifts at d0, then k_fixed_decode.
//   k_finalize       compacts the recovered frequencies into the result.
#include <cstdio>

#include "sft_decode.cuh"
#include "sft_fft.cuh"
#include "sft_internal.h"

namespace sft {

// ----------------------------------------------------------- gather + FFT
template <class F>
__global__ void __launch_bounds__(512) k_gather_fft(
    const typename F::In* __restrict__ x, int64_t x_stride, int64_t N, int64_t d, int log2M,
    int shift0, int log2Mt, const typename F::Tw* __restrict__ tw, double2* __restrict__ out,
    int64_t out_sig, int64_t out_row, int row0, unsigned long long* __restrict__ ymax2) {
  extern __shared__ __align__(16) char smem[];
  const int b = blockIdx.y;
  const int js = blockIdx.x;
  const int64_t shift = shift0 + js;
  const int M = 1 << log2M;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const typename F::In* xs = x + (int64_t)b * x_stride;
  // x_{d,shift}[n] = x[(n d + shift) mod N]
  for (int n = tid; n < M; n += nthr) {
    const int64_t e = ((int64_t)n * d + shift) & (N - 1);
    F::st(smem, M, n, F::from_in(__ldg(xs + e)));
  }
  __syncthreads();
  cta_fft<F>(smem, log2M, log2Mt, tw, tid, nthr);
  double2* o = out + (int64_t)b * out_sig + (int64_t)(row0 + js) * out_row;
  const double scale = (double)d;
  double lmax = 0.0;
  for (int k = tid; k < M; k += nthr) {
    const double2 v = F::out(F::ld(smem, M, k), scale);
    o[k] = v;
    lmax = fmax(lmax, v.x * v.x + v.y * v.y);
  }
  if (ymax2 != nullptr && shift == 0) {
    // block max of |Y_{d,0}|^2 -> per-signal atomic max on the bit pattern
    // (non-negative doubles order like their unsigned bit patterns)
    __shared__ double wmax[32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o2));
    if ((tid & 31) == 0) wmax[tid >> 5] = lmax;
    __syncthreads();
    if (tid < 32) {
      double v = tid < (nthr >> 5) ? wmax[tid] : 0.0;
#pragma unroll
      for (int o2 = 16; o2 > 0; o2 >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o2));
      if (tid == 0) atomicMax(ymax2 + b, (unsigned long long)__double_as_longlong(v));
    }
  }
}

// ------------------------------------------------- per-level decode (ITER)
struct LevelArgs {
  int64_t N, M, d, M0;
  const double2* prev;  // level l-1 rows, length 2M
  double2* cur;         // level l rows, length M
  int64_t held_elems;
  const uint8_t* Tprev;
  uint8_t* Tcur;
  uint8_t* slot_cnt;
  int64_t* slot_s;
  double2* slot_p;
  const unsigned long long* ymax2;
  int32_t* flags;
  double zero_tol, root_tol, res_tol;
  OmegaTab om;
};

__device__ __forceinline__ cdbl ld2(const double2* p) {
  double2 v = *p;
  return mk(v.x, v.y);
}

// File the a recovered frequencies of one decode event under their level-0
// bins (the calling thread owns every level-0 bin congruent to its bin).
template <int A>
__device__ __forceinline__ void file_solution(const int64_t* s, const cdbl* p, int64_t M0,
                                              uint8_t* cnt, int64_t* ss, double2* sp,
                                              int32_t* flag) {
#pragma unroll
  for (int j = 0; j < A; ++j) {
    const int64_t k0 = s[j] & (M0 - 1);
    const int c = cnt[k0];
    if (c < 4) {
      ss[k0 * 4 + c] = s[j];
      sp[k0 * 4 + c] = make_double2(p[j].x, p[j].y);
      cnt[k0] = (uint8_t)(c + 1);
    } else {
      atomicOr(flag, 1);
    }
  }
}

template <int A>
__global__ void __launch_bounds__(128) k_iter_level(LevelArgs g) {
  constexpr int l = A - 1, nm = 2 * A;
  const int b = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.M) return;
  const int64_t M = g.M, M0 = g.M0;
  const double2* prev = g.prev + (int64_t)b * g.held_elems;
  double2* cur = g.cur + (int64_t)b * g.held_elems;
  uint8_t* cnt = g.slot_cnt + (int64_t)b * M0;
  int64_t* ss = g.slot_s + (int64_t)b * M0 * 4;
  double2* sp = g.slot_p + (int64_t)b * M0 * 4;

  cdbl m[nm];
  // fold the syndromes held from level l-1 (length 2M) to length M
#pragma unroll
  for (int j = 0; j < 2 * l; ++j) m[j] = ld2(prev + j * 2 * M + k) + ld2(prev + j * 2 * M + k + M);
  m[2 * l] = ld2(cur + (2 * l) * M + k);
  m[2 * l + 1] = ld2(cur + (2 * l + 1) * M + k);
  // SubFreq: remove every frequency recovered at earlier levels from the
  // two new shifts; they are filed under the level-0 bins k + i M
  if (l > 0) {
    const int64_t nsub = M0 / M;
    for (int64_t i = 0; i < nsub; ++i) {
      const int64_t k0 = k + i * M;
      const int c = cnt[k0];
      for (int e = 0; e < c; ++e) {
        const int64_t s = ss[k0 * 4 + e];
        const cdbl p = ld2(sp + k0 * 4 + e);
        m[2 * l] = m[2 * l] - p * omega_pow(g.om, s * (2 * l));
        m[2 * l + 1] = m[2 * l + 1] - p * omega_pow(g.om, s * (2 * l + 1));
      }
    }
  }
  uint8_t t = 0;
  if (l > 0) t = (uint8_t)(g.Tprev[(int64_t)b * M0 + k] | g.Tprev[(int64_t)b * M0 + k + M]);
  const double theta = g.zero_tol * sqrt(__longlong_as_double((long long)g.ymax2[b]));
  const bool active = t || absd(m[2 * l]) > theta || absd(m[2 * l + 1]) > theta;
  if (active) {
    BinGeom geom{g.N, M, g.d, g.om};
    Tol tol{theta, g.root_tol, g.res_tol};
    int64_t s[4];
    cdbl p[4];
    if (decode_bin<A>(m, nm, k, geom, tol, s, p)) {
      file_solution<A>(s, p, M0, cnt, ss, sp, g.flags + b);
      // the recovered terms leave every syndrome held for this bin
#pragma unroll
      for (int j = 0; j < A; ++j)
#pragma unroll
        for (int i = 0; i < nm; ++i) m[i] = m[i] - p[j] * omega_pow(g.om, s[j] * i);
      t = 0;
    } else {
      t = 1;
    }
  }
#pragma unroll
  for (int j = 0; j < nm; ++j) cur[j * M + k] = make_double2(m[j].x, m[j].y);
  g.Tcur[(int64_t)b * M0 + k] = t;
}

// ---------------------------------------------- non-iterative decode (FIXED)
struct FixedArgs {
  int64_t N, M, d;
  int a_max;
  const double2* Y;  // 2 a_max rows of length M
  int64_t held_elems;
  uint8_t* T;
  uint8_t* slot_cnt;
  int64_t* slot_s;
  double2* slot_p;
  const unsigned long long* ymax2;
  int32_t* flags;
  double zero_tol, root_tol, res_tol;
  OmegaTab om;
};

template <int A>
__device__ __forceinline__ bool try_fixed(const cdbl* m, int nm, int64_t k, const BinGeom& geom,
                                          const Tol& tol, int64_t M0, uint8_t* cnt, int64_t* ss,
                                          double2* sp, int32_t* flag) {
  int64_t s[4];
  cdbl p[4];
  if (!decode_bin<A>(m, nm, k, geom, tol, s, p)) return false;
  file_solution<A>(s, p, M0, cnt, ss, sp, flag);
  return true;
}

__global__ void __launch_bounds__(128) k_fixed_decode(FixedArgs g) {
  const int b = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.M) return;
  const int64_t M = g.M;
  const int nm = 2 * g.a_max;
  const double2* Y = g.Y + (int64_t)b * g.held_elems;
  cdbl m[8];
  const double theta = g.zero_tol * sqrt(__longlong_as_double((long long)g.ymax2[b]));
  bool active = false;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j < nm) {
      m[j] = ld2(Y + j * M + k);
      active = active || absd(m[j]) > theta;
    }
  }
  uint8_t t = 0;
  if (active) {
    BinGeom geom{g.N, M, g.d, g.om};
    Tol tol{theta, g.root_tol, g.res_tol};
    uint8_t* cnt = g.slot_cnt + (int64_t)b * M;
    int64_t* ss = g.slot_s + (int64_t)b * M * 4;
    double2* sp = g.slot_p + (int64_t)b * M * 4;
    int32_t* fl = g.flags + b;
    bool ok = try_fixed<1>(m, nm, k, geom, tol, M, cnt, ss, sp, fl);
    if (!ok && g.a_max >= 2) ok = try_fixed<2>(m, nm, k, geom, tol, M, cnt, ss, sp, fl);
    if (!ok && g.a_max >= 3) ok = try_fixed<3>(m, nm, k, geom, tol, M, cnt, ss, sp, fl);
    if (!ok && g.a_max >= 4) ok = try_fixed<4>(m, nm, k, geom, tol, M, cnt, ss, sp, fl);
    t = ok ? 0 : 1;
  }
  g.T[(int64_t)b * M + k] = t;
}

// ------------------------------------------------------------- finalize
struct FinArgs {
  int64_t M0, M_last;
  const uint8_t* slot_cnt;
  const int64_t* slot_s;
  const double2* slot_p;
  const uint8_t* T_last;
  const int32_t* flags;
  int64_t cap;
  int64_t* idx;
  double2* val;
  int64_t* count;
  int32_t* unresolved;
  int32_t* overflow;
};

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

__global__ void __launch_bounds__(1024) k_finalize(FinArgs g) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t M0 = g.M0;
  const uint8_t* cnt = g.slot_cnt + (int64_t)b * M0;
  const int64_t chunk = (M0 + nthr - 1) / nthr;
  const int64_t lo = min((int64_t)tid * chunk, M0), hi = min(lo + chunk, M0);
  int mine = 0;
  for (int64_t k0 = lo; k0 < hi; ++k0) mine += cnt[k0];
  int total = 0;
  int pos = block_excl_scan(mine, &total);
  int64_t* idx = g.idx + (int64_t)b * g.cap;
  double2* val = g.val + (int64_t)b * g.cap;
  for (int64_t k0 = lo; k0 < hi; ++k0) {
    const int c = cnt[k0];
    for (int e = 0; e < c; ++e, ++pos) {
      if (pos < g.cap) {
        idx[pos] = g.slot_s[((int64_t)b * M0 + k0) * 4 + e];
        val[pos] = g.slot_p[((int64_t)b * M0 + k0) * 4 + e];
      }
    }
  }
  // unresolved bins at the last level
  int un = 0;
  const uint8_t* T = g.T_last + (int64_t)b * M0;
  for (int64_t k = tid; k < g.M_last; k += nthr) un += T[k];
  int un_total = 0;
  (void)block_excl_scan(un, &un_total);
  if (tid == 0) {
    g.count[b] = total < g.cap ? total : g.cap;
    g.unresolved[b] = un_total;
    g.overflow[b] = (total > g.cap || (g.flags[b] & 1)) ? 1 : 0;
  }
}

// ------------------------------------------------------------ launchers
static int fft_threads(int log2M) {
  const int M = 1 << log2M;
  return M / 16 > 32 ? M / 16 : 32;
}

cudaError_t prepare_kernels(sft_plan_s* P) {
  const int smem = (int)(P->M0 * 16);
  cudaError_t e;
  if (P->p.precision == SFT_FP64)
    e = cudaFuncSetAttribute(k_gather_fft<F64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  else
    e = cudaFuncSetAttribute(k_gather_fft<FF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

int launches_per_call(const sft_plan_s* P) {
  if (P->p.mode == SFT_EXACT_FIXED) return 3;
  return 2 * P->levels + 1;
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
  StageRec r{name, pool_event(P), pool_event(P)};
  cudaEventRecord(r.t0, st);
  P->stage_recs.push_back(r);
}

void stage_end(sft_plan_s* P, cudaStream_t st) {
  if (!P->profiling || P->stage_recs.empty()) return;
  cudaEventRecord(P->stage_recs.back().t1, st);
}

template <class F>
static void launch_gather_fft(const sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                              int64_t d, int log2M, int shift0, int nshift, double2* out,
                              int64_t out_row, int row0, bool want_ymax, cudaStream_t st) {
  dim3 grid(nshift, (unsigned)B);
  const int nthr = fft_threads(log2M);
  const size_t smem = (size_t)(1 << log2M) * F::kBytesPerPoint;
  static const char* names[] = {"gather_fft_l0", "gather_fft_l1", "gather_fft_l2", "gather_fft_l3"};
  stage_begin(const_cast<sft_plan_s*>(P), nshift > 2 ? "gather_fft_fixed" : names[shift0 / 2], st);
  k_gather_fft<F><<<grid, nthr, smem, st>>>(
      reinterpret_cast<const typename F::In*>(x), x_stride, P->p.N, d, log2M, shift0, P->log2M0,
      reinterpret_cast<const typename F::Tw*>(P->tab.tw), out, P->ws.held_elems, out_row, row0,
      want_ymax ? P->ws.ymax2 : nullptr);
  stage_end(const_cast<sft_plan_s*>(P), st);
}

cudaError_t launch_exact(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                         const sft_result* r, cudaStream_t st) {
  const Workspace& W = P->ws;
  OmegaTab om{P->tab.om_hi, P->tab.om_lo, P->tab.om_lo_bits, P->p.N - 1};
  const bool fp64 = P->p.precision == SFT_FP64;
  const int64_t d0 = P->p.d;
  int64_t M_last = P->M0;
  const uint8_t* T_last = W.T[0];

  if (P->p.mode == SFT_EXACT_FIXED) {
    const int nsh = 2 * P->p.a_max;
    if (fp64)
      launch_gather_fft<F64>(P, B, x, x_stride, d0, P->log2M0, 0, nsh, W.held[0], P->M0, 0, true, st);
    else
      launch_gather_fft<FF>(P, B, x, x_stride, d0, P->log2M0, 0, nsh, W.held[0], P->M0, 0, true, st);
    FixedArgs g{P->p.N, P->M0, d0, P->p.a_max, W.held[0], W.held_elems, W.T[0], W.slot_cnt,
                W.slot_s, W.slot_p, W.ymax2, W.flags, P->p.zero_tol, P->p.root_tol,
                P->p.res_tol, om};
    dim3 grid((unsigned)((P->M0 + 127) / 128), (unsigned)B);
    stage_begin(P, "decode_fixed", st);
    k_fixed_decode<<<grid, 128, 0, st>>>(g);
    stage_end(P, st);
  } else {
    int64_t M = P->M0, d = d0;
    for (int l = 0; l < P->levels; ++l) {
      if (l > 0) {
        M >>= 1;
        d <<= 1;
      }
      const int log2M = P->log2M0 - l;
      double2* cur = W.held[l & 1];
      const double2* prev = W.held[(l + 1) & 1];
      if (fp64)
        launch_gather_fft<F64>(P, B, x, x_stride, d, log2M, 2 * l, 2, cur, M, 2 * l, l == 0, st);
      else
        launch_gather_fft<FF>(P, B, x, x_stride, d, log2M, 2 * l, 2, cur, M, 2 * l, l == 0, st);
      LevelArgs g{P->p.N, M, d, P->M0, prev, cur, W.held_elems, W.T[(l + 1) & 1], W.T[l & 1],
                  W.slot_cnt, W.slot_s, W.slot_p, W.ymax2, W.flags, P->p.zero_tol,
                  P->p.root_tol, P->p.res_tol, om};
      dim3 grid((unsigned)((M + 127) / 128), (unsigned)B);
      static const char* dnames[] = {"decode_l0", "decode_l1", "decode_l2", "decode_l3"};
      stage_begin(P, dnames[l], st);
      switch (l) {
        case 0: k_iter_level<1><<<grid, 128, 0, st>>>(g); break;
        case 1: k_iter_level<2><<<grid, 128, 0, st>>>(g); break;
        case 2: k_iter_level<3><<<grid, 128, 0, st>>>(g); break;
        default: k_iter_level<4><<<grid, 128, 0, st>>>(g); break;
      }
      stage_end(P, st);
      M_last = M;
      T_last = W.T[l & 1];
    }
  }
  FinArgs f{P->M0, M_last, W.slot_cnt, W.slot_s, W.slot_p, T_last, W.flags, r->cap, r->idx,
            reinterpret_cast<double2*>(r->val), r->count, r->unresolved, r->overflow};
  stage_begin(P, "finalize", st);
  k_finalize<<<(unsigned)B, 1024, 0, st>>>(f);
  stage_end(P, st);
  return cudaGetLastError();
}

}  // namespace sft
