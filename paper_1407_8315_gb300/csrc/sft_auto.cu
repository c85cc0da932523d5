// sft_auto.cu -- unknown K (Sec. II-E, the bottom-up strategy).
//
// Every signal starts at d = N / M_start; while a run leaves a bin unsolved
// (or a level-0 bin overflowed its solution slots) the signal is run
// again with d halved (M doubled).  All signals still running at one M go
// through one launch sequence of a plan for that M, reading their inputs
// and writing their results through per-signal pointer tables, so each
// signal's result buffers end up holding its last run.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sft_internal.h"

namespace {

sft_status fail(sft_status st, const char* msg) {
  sft::set_error_detail(msg);
  return st;
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= v) ++l;
  return l;
}

}  // namespace

extern "C" sft_status sft_exact_auto(const sft_params* p_in, int64_t n, const void* x,
                                     int64_t x_stride, int64_t M_start, int64_t M_max,
                                     const sft_result* r, int64_t* m_out, void* stream) {
  if (!p_in || !x || !r) return fail(SFT_EINVAL, "sft_exact_auto: NULL argument");
  sft_params p = *p_in;
  p.K = 0;
  p.d = 1;
  sft::normalize_params(&p);
  if (p.mode != SFT_EXACT_ITER && p.mode != SFT_EXACT_FIXED)
    return fail(SFT_EINVAL, "sft_exact_auto: mode must be SFT_EXACT_ITER or SFT_EXACT_FIXED");
  if (n < 1) return fail(SFT_EINVAL, "sft_exact_auto: n_signals < 1");
  if (x_stride < p.N) return fail(SFT_EINVAL, "sft_exact_auto: x_stride < N");
  if (M_max <= 0) M_max = p.N;
  if (!pow2(M_start) || !pow2(M_max) || M_start > M_max || M_max > p.N)
    return fail(SFT_EINVAL, "sft_exact_auto: M_start <= M_max must be powers of two <= N");
  if (M_max > (int64_t(1) << 26)) return fail(SFT_EUNSUPPORTED, "sft_exact_auto: M_max above 2^26");
  if (r->cap < 1 || !r->idx || !r->val || !r->count || !r->unresolved || !r->overflow)
    return fail(SFT_EINVAL, "sft_exact_auto: NULL result array or cap < 1");
  const size_t esize = p.precision == SFT_FP64 ? 16 : 8;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  std::vector<int64_t> active((size_t)n), stop((size_t)n, 0);
  for (int64_t i = 0; i < n; ++i) active[(size_t)i] = i;
  std::vector<const void*> hx((size_t)n);
  std::vector<sft_result> hr((size_t)n);
  std::vector<int32_t> un((size_t)n), ov((size_t)n);
  void** dx = nullptr;
  sft_result* dr = nullptr;
  cudaError_t e = cudaMalloc(&dx, (size_t)n * sizeof(void*));
  if (!e) e = cudaMalloc(&dr, (size_t)n * sizeof(sft_result));
  sft_status status = SFT_OK;
  for (int64_t M = M_start; !e && status == SFT_OK && M <= M_max && !active.empty(); M *= 2) {
    sft_params q = p;
    q.d = p.N / M;
    if (q.mode == SFT_EXACT_ITER) q.max_iters = std::min<int32_t>(p.a_max, ilog2(M) + 1);
    const int64_t na = (int64_t)active.size();
    sft_plan_t P = nullptr;
    status = sft_plan_create(&q, na, &P);
    if (status != SFT_OK) break;
    for (int64_t j = 0; j < na; ++j) {
      const int64_t i = active[(size_t)j];
      hx[(size_t)j] = static_cast<const char*>(x) + (size_t)i * (size_t)x_stride * esize;
      sft_result ri = *r;
      ri.idx = r->idx + i * r->cap;
      ri.val = r->val + 2 * i * r->cap;
      ri.count = r->count + i;
      ri.unresolved = r->unresolved + i;
      ri.overflow = r->overflow + i;
      hr[(size_t)j] = ri;
    }
    e = cudaMemcpyAsync(dx, hx.data(), (size_t)na * sizeof(void*), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(dr, hr.data(), (size_t)na * sizeof(sft_result), cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemsetAsync(P->ws.zero_base, 0, P->ws.zero_bytes, st);
    if (!e) {
      P->x_table = reinterpret_cast<const void* const*>(dx);
      P->r_table = dr;
      sft_result dummy{};
      e = sft::launch_exact(P, na, nullptr, p.N, &dummy, st);
      P->x_table = nullptr;
      P->r_table = nullptr;
    }
    if (!e) e = cudaMemcpyAsync(un.data(), r->unresolved, (size_t)n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(ov.data(), r->overflow, (size_t)n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    sft_plan_destroy(P);
    if (e) break;
    std::vector<int64_t> next;
    for (int64_t i : active) {
      stop[(size_t)i] = M;
      if (un[(size_t)i] != 0 || ov[(size_t)i] != 0) next.push_back(i);
    }
    active.swap(next);
  }
  cudaFree(dx);
  cudaFree(dr);
  if (e) {
    sft::set_error_detail(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
  }
  if (status != SFT_OK) return status;
  if (m_out) std::memcpy(m_out, stop.data(), (size_t)n * sizeof(int64_t));
  return SFT_OK;
}
