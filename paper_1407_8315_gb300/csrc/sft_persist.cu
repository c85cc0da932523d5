// sft_persist.cu -- the persistent kernel of heterogeneous batches: every
// exactly sparse signal of a batch (Algorithm 1, mixed precision, a_max <= 4,
// N/d <= 4096) is one item of a device work queue, and one launch of
// resident CTAs drains the queue.
//
// A CTA claims the next item with one atomic on the queue head and runs the
// whole of Algorithm 1 for that signal by itself: per level l the gather and
// FFT of the two new shifts (Eq. (2); the same Stockham radix-8 passes, in
// the same order, as the per-shape launch sequence), the fold, SubFreq and
// activity test of every bin, the decode of the active bins (SynDec with
// a = l + 1), and at the end the compaction of the recovered frequencies
// into the signal's result buffers.  The items are independent, so no CTA
// ever waits on another: the only shared state is the queue head.  Items
// are ordered largest first, so that the resident CTAs finish together.
//
// Why: a batch of many small signals of many shapes launched as one
// launch sequence per shape runs each shape's chain of latency-bound stages
// (the later levels' decoders) one after another on its stream; here every
// signal's chain runs beside all the others'.
#include <algorithm>

#include "sft_decode.cuh"
#include "sft_device_util.cuh"
#include "sft_fft.cuh"
#include "sft_internal.h"
#include "sft_levels.cuh"

namespace sft {

// 128 threads per CTA and two CTAs per SM (255 registers each): while one
// CTA's signal sits in a barrier-bound stage (few bins to decode), the
// other's runs.
constexpr int kPThreads = 128;

// Block-wide exclusive scan of one int per thread (blockDim = kPThreads);
// *total receives the sum.  Synchronises the block.
__device__ __forceinline__ int pblock_scan(int v, int* total) {
  __shared__ int wsum[kPThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int before = x - v, tot = 0;
#pragma unroll
  for (int i = 0; i < kPThreads / 32; ++i) {
    if (i < w) before += wsum[i];
    tot += wsum[i];
  }
  *total = tot;
  __syncthreads();
  return before;
}

// The forward FFT of buf[0..M) (float-float), M <= 4096, by the CTA's 128
// threads: radix-8 passes, then one radix-4 or radix-2 pass for the rest --
// the pass sequence of the one-CTA FFT at 8 points per thread, each thread
// here owning four radix-8 groups, so every output is rounded as there.
__device__ __forceinline__ void pcta_fft8(char* buf, int log2M, int log2Mt, const float4* tw,
                                          int tid) {
  const int M = 1 << log2M;
  int Ns = 1, rem = log2M;
  while (rem >= 3) {
    stockham_pass<FF, 8, 32>(buf, M, Ns, log2Mt, tw, tid, kPThreads);
    Ns <<= 3;
    rem -= 3;
  }
  if (rem == 2) stockham_pass<FF, 4, 32>(buf, M, Ns, log2Mt, tw, tid, kPThreads);
  if (rem == 1) stockham_pass<FF, 2, 32>(buf, M, Ns, log2Mt, tw, tid, kPThreads);
}

// The fold stage and the decode stage of level A - 1 for this thread's bins.
// Separate functions, so that each is register-allocated on its own; the
// level's arguments stay in shared memory (g), so that next to nothing is
// live across the calls.
template <int A>
__device__ __noinline__ void pfold(const LevelArgs& g, int* q, int* qn) {
  for (int k = threadIdx.x; k < (int)g.M; k += kPThreads)
    if (fold_bin<FF, A>(g, 0, k)) q[atomicAdd(qn, 1)] = k;
}
template <int A>
__device__ __noinline__ void pdecode(const LevelArgs& g, const int* q, int n) {
  for (int e = threadIdx.x; e < n; e += kPThreads) decode_level_bin<FF, A>(g, 0, q[e]);
}

// The two new shifts' syndromes of level l (Eq. (2)) into the level's rows:
// gather x_{d,j}[n] = x[(n d + j) mod N], FFT, times d; at level 0 also
// max_k |Y_{d,0}[k]|^2 for the zero threshold.
__device__ __noinline__ void pshifts(const PSig& S, const LevelArgs& g, int l, char* buf,
                                     unsigned long long* ymax) {
  const int tid = threadIdx.x;
  const int M = (int)g.M;
  const int log2M = S.log2M0 - l;
  float4* cur = reinterpret_cast<float4*>(g.cur);
  float fmx = 0.0f;
#pragma unroll 1
  for (int j = 2 * l; j <= 2 * l + 1; ++j) {
    for (int n = tid; n < M; n += kPThreads)
      FF::st(buf, M, n, FF::from_in(__ldg(S.x + (((int64_t)n * g.d + j) & (S.N - 1)))));
    __syncthreads();
    pcta_fft8(buf, log2M, S.log2M0, S.tw, tid);
    for (int k = tid; k < M; k += kPThreads) {
      const float4 w = FF::out(FF::ld(buf, M, k), (float)g.d);
      cur[(int64_t)j * M + k] = w;
      if (j == 0) fmx = fmaxf(fmx, FF::out_norm_hi(w));
    }
    __syncthreads();
  }
  if (l == 0) {
    // order-preserving on the bit pattern of the non-negative double
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fmx = fmaxf(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
    if ((tid & 31) == 0) atomicMax(ymax, (unsigned long long)__double_as_longlong((double)fmx));
    __syncthreads();
    if (tid == 0) *S.ymax2 = *ymax;
  }
}

// Level l = A - 1 of one signal, by the whole CTA: the two new shifts, then
// fold_bin on every bin (the active ones queued in shared memory, q), then
// decode_level_bin on the queue.
template <int A>
__device__ __forceinline__ void plevel(const PSig& S, const LevelArgs& g, char* buf, int* q,
                                       int* qn, unsigned long long* ymax) {
  pshifts(S, g, A - 1, buf, ymax);
  if (threadIdx.x == 0) *qn = 0;
  __syncthreads();
  pfold<A>(g, q, qn);
  __syncthreads();
  pdecode<A>(g, q, *qn);
  __syncthreads();
}

// The recovered frequencies of one signal into its result buffers: bin by
// bin (level-0 bins, slot order), each thread a run of consecutive bins
// placed by one block scan; then the counts.
__device__ __noinline__ void pfinalize(const PSig& S, int64_t M_last, const uint8_t* T_last, int tid) {
  const int64_t M0 = S.M0;
  const int64_t per = (M0 + kPThreads - 1) / kPThreads;
  const int64_t lo = min(per * tid, M0), hi = min(lo + per, M0);
  int mine = 0;
  for (int64_t k0 = lo; k0 < hi; ++k0) mine += S.slot_cnt[k0];
  int total = 0;
  const int pos0 = pblock_scan(mine, &total);
  const int64_t cap = S.r.cap;
  double2* val = reinterpret_cast<double2*>(S.r.val);
  int64_t pos = pos0;
  for (int64_t k0 = lo; k0 < hi; ++k0) {
    const int c = S.slot_cnt[k0];
    for (int e = 0; e < c; ++e, ++pos) {
      if (pos < cap) {
        S.r.idx[pos] = S.slot_s[slot_ix(k0, e, M0)];
        const cdbl v = Store<FF>::to_d(S.slot_p[slot_ix(k0, e, M0)]);
        val[pos] = make_double2(v.x, v.y);
      }
    }
  }
  int un = 0;
  for (int64_t k = tid; k < M_last; k += kPThreads) un += T_last[k];
  int un_total = 0;
  (void)pblock_scan(un, &un_total);
  if (tid == 0) {
    *S.r.count = total < cap ? total : cap;
    *S.r.unresolved = un_total;
    *S.r.overflow = (total > cap || (*S.flags & 1)) ? 1 : 0;
  }
}

constexpr size_t kPBufBytes = (size_t)(kPersistMaxM + (kPersistMaxM >> 4)) * 16;  // padded FFT
constexpr size_t kPSmemBytes = kPBufBytes + (size_t)kPersistMaxM * sizeof(int);

// The persistent kernel: resident CTAs claim signals (largest first) until
// the queue is empty; each runs Algorithm 1 for its signal alone.
__global__ void __launch_bounds__(kPThreads, 2)
    k_exact_persistent(const PSig* __restrict__ sigs, const int* __restrict__ order, int n,
                       int* __restrict__ head) {
  extern __shared__ __align__(16) char psmem[];
  char* buf = psmem;
  int* q = reinterpret_cast<int*>(psmem + kPBufBytes);
  __shared__ PSig s_sig;
  __shared__ LevelArgs s_g;
  __shared__ int s_item, s_qn;
  __shared__ unsigned long long s_ymax;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int it = atomicAdd(head, 1);
      s_item = it;
      if (it < n) s_sig = sigs[order[it]];
      s_ymax = 0ull;
    }
    __syncthreads();
    if (s_item >= n) break;
    const PSig& S = s_sig;
    // the per-signal state the launch sequence clears before a call
    for (int64_t k = tid; k < S.M0; k += kPThreads) S.slot_cnt[k] = 0;
    if (tid == 0) {
      *S.flags = 0;
      *S.ymax2 = 0ull;
    }
    for (int l = 0; l < S.levels; ++l) {
      __syncthreads();
      if (tid == 0) {
        const int64_t M = S.M0 >> l, d = S.d0 << l;
        s_g = LevelArgs{S.N,
                        M,
                        d,
                        S.M0,
                        S.held[(l + 1) & 1],
                        S.held[l & 1],
                        S.held_elems,
                        S.T[(l + 1) & 1],
                        S.T[l & 1],
                        S.slot_cnt,
                        S.slot_s,
                        S.slot_p,
                        S.ymax2,
                        S.flags,
                        S.zero_tol,
                        S.root_tol,
                        S.res_tol,
                        OmegaTab{S.om_hi, S.om_lo, S.om_lo_bits, S.N - 1},
                        OmegaTabFF{S.om_hi_ff, S.om_lo_ff, S.om_lo_bits, S.N - 1},
                        (float)(S.zero_tol * S.zero_tol),
                        (float)(S.root_tol * S.root_tol),
                        (float)(S.res_tol * S.res_tol)};
      }
      __syncthreads();
      switch (l) {
        case 0: plevel<1>(S, s_g, buf, q, &s_qn, &s_ymax); break;
        case 1: plevel<2>(S, s_g, buf, q, &s_qn, &s_ymax); break;
        case 2: plevel<3>(S, s_g, buf, q, &s_qn, &s_ymax); break;
        default: plevel<4>(S, s_g, buf, q, &s_qn, &s_ymax); break;
      }
    }
    pfinalize(S, S.M0 >> (S.levels - 1), S.T[(S.levels - 1) & 1], tid);
    __syncthreads();
  }
}

int persistent_ctas_per_sm() {
  int per = 0;
  if (cudaFuncSetAttribute(k_exact_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kPSmemBytes) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_exact_persistent, kPThreads,
                                                    kPSmemBytes) != cudaSuccess)
    return 0;
  return per;
}

cudaError_t launch_exact_persistent(const PSig* sigs, const int* order, int n, int* head, int ctas,
                                    cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(head, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_exact_persistent<<<(unsigned)std::max(1, std::min(ctas, n)), kPThreads, kPSmemBytes, st>>>(
      sigs, order, n, head);
  return cudaGetLastError();
}

}  // namespace sft
