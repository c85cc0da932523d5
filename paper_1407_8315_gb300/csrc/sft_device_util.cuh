// sft_device_util.cuh -- device helpers shared by the kernel files: filing
// recovered frequencies under their level-0 bins and warp-aggregated queue
// appends.
#pragma once

#include "sft_common.cuh"
#include "sft_slots.h"

namespace sft {

// Index of slot e of level-0 bin k0 within one signal's slot arrays
// (M0 x kSlots entries).  Slot-major: slot e of every bin is one contiguous
// run, so consecutive bins' first slots -- the only ones most bins use --
// share sectors, and a warp reading the slots of 32 consecutive bins reads
// them coalesced.
__device__ __forceinline__ int64_t slot_ix(int64_t k0, int e, int64_t M0) {
  return (int64_t)e * M0 + k0;
}

// File the a recovered frequencies of one decode event under their level-0
// bins (the calling thread owns every level-0 bin congruent to its bin).
template <class F, int A>
__device__ __forceinline__ void file_solution(const int64_t* s, const cdbl* p, int64_t M0,
                                              uint8_t* cnt, int64_t* ss,
                                              typename Store<F>::T* sp, int32_t* flag) {
#pragma unroll
  for (int j = 0; j < A; ++j) {
    const int64_t k0 = s[j] & (M0 - 1);
    const int c = cnt[k0];
    if (c < kSlots) {
      ss[slot_ix(k0, c, M0)] = s[j];
      sp[slot_ix(k0, c, M0)] = Store<F>::from_d(p[j]);
      cnt[k0] = (uint8_t)(c + 1);
    } else {
      atomicOr(flag, 1);
    }
  }
}

// File one recovered frequency whose value is already float-float.  With
// kFirst the bin is known to hold nothing yet (level 0 of ITER: the counts
// are zeroed per call and only bin k's own thread files under k), so its
// count is not read -- one dependent load fewer per decoded bin.
template <bool kFirst = false>
__device__ __forceinline__ void file_one_ff(int64_t s, float4 p, int64_t M0, uint8_t* cnt,
                                            int64_t* ss, float4* sp, int32_t* flag) {
  const int64_t k0 = s & (M0 - 1);
  const int c = kFirst ? 0 : cnt[k0];
  if (c < kSlots) {
    ss[slot_ix(k0, c, M0)] = s;
    sp[slot_ix(k0, c, M0)] = p;
    cnt[k0] = (uint8_t)(c + 1);
  } else {
    atomicOr(flag, 1);
  }
}

// Append (b, k) to a device queue when `pred`; one atomic per block of NT
// threads (a per-warp atomic on one counter serialises in L2 when the
// queues are long).  Every thread of the block must call this.
template <int NT>
__device__ __forceinline__ void block_queue_push(bool pred, int b, int k, int2* q, int* count) {
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
  __shared__ int wofs[NT / 32];
  const int lane = (int)(threadIdx.x & 31u), w = (int)(threadIdx.x >> 5);
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) wofs[w] = __popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
      const int c = wofs[i];
      wofs[i] = tot;
      tot += c;
    }
    const int base = tot > 0 ? atomicAdd(count, tot) : 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) wofs[i] += base;
  }
  __syncthreads();
  if (pred) q[wofs[w] + __popc(mask & ((1u << lane) - 1u))] = make_int2(b, k);
}

// Append (b, k) to a device queue when `pred`; one atomic per warp.  Every
// lane of the warp must call this (inactive lanes with pred = false).
__device__ __forceinline__ void queue_push(bool pred, int b, int k, int2* q, int* count) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  if (mask == 0u) return;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if ((int)lane == leader) base = atomicAdd(count, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) q[base + __popc(mask & ((1u << lane) - 1u))] = make_int2(b, k);
}

// File n recovered frequencies (n known only at run time).
template <class F>
__device__ __forceinline__ void file_n(int n, const int64_t* s, const cdbl* p, int64_t M0,
                                       uint8_t* cnt, int64_t* ss, typename Store<F>::T* sp,
                                       int32_t* flag) {
  for (int j = 0; j < n; ++j) {
    const int64_t k0 = s[j] & (M0 - 1);
    const int c = cnt[k0];
    if (c < kSlots) {
      ss[slot_ix(k0, c, M0)] = s[j];
      sp[slot_ix(k0, c, M0)] = Store<F>::from_d(p[j]);
      cnt[k0] = (uint8_t)(c + 1);
    } else {
      atomicOr(flag, 1);
    }
  }
}

}  // namespace sft
