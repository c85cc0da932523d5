// sft_api.cu -- the C ABI (include/sft.h): parameter validation, plans
// (device tables + workspace), and the device / host entry points.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "sft_internal.h"

namespace {

thread_local char g_cuda_err[256] = "";

void note_cuda(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e),
                cudaGetErrorString(e));
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

constexpr int64_t kMaxM = int64_t(1) << 26;  // largest M = N/d (four-step FFT of 2^13 x 2^13)

sft_status fill_defaults(sft_params* p) {
  const bool gen = sft::is_general_mode(p->mode);
  if (p->a_max == 0) p->a_max = gen ? 3 : 4;
  if (gen && p->n_cs_shifts == 0) p->n_cs_shifts = 3 * p->a_max;
  if (p->max_iters == 0) p->max_iters = p->a_max;
  const bool fp64 = p->precision == SFT_FP64;
  if (!(p->zero_tol > 0)) p->zero_tol = fp64 ? 1e-10 : 1e-6;
  if (!(p->root_tol > 0)) p->root_tol = 0.1;
  if (!(p->res_tol > 0)) p->res_tol = fp64 ? 1e-9 : 1e-6;
  return SFT_OK;
}

sft_status why(sft_status st, const char* msg) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg);
  return st;
}

sft_status validate(const sft_params& p) {
  if (!is_pow2(p.N) || p.N < 8 || p.N > (int64_t(1) << 30))
    return why(SFT_EINVAL, "N must be a power of two in [2^3, 2^30]");
  if (p.K < 0 || p.K > p.N) return why(SFT_EINVAL, "K must lie in [0, N]");
  if (!is_pow2(p.d) || p.d > p.N) return why(SFT_EINVAL, "d must be a power of two <= N");
  if (p.a_max < 1 || p.a_max > 8) return why(SFT_EINVAL, "a_max must lie in [1, 8]");
  if (sft::is_general_mode(p.mode) && p.a_max > 4)
    return why(SFT_EUNSUPPORTED, "the general modes take a_max <= 4");
  if (p.mode == SFT_EXACT_FIXED && p.a_max > 4 && p.a_max != 8)
    return why(SFT_EUNSUPPORTED, "SFT_EXACT_FIXED takes a_max <= 4 or a_max = 8");
  if (p.precision != SFT_FP64 && p.precision != SFT_MIXED)
    return why(SFT_EINVAL, "unknown precision");
  if (p.mode != SFT_EXACT_ITER && p.mode != SFT_EXACT_FIXED && !sft::is_general_mode(p.mode))
    return why(SFT_EINVAL, "unknown mode");
  if (sft::is_general_mode(p.mode) &&
      (p.n_cs_shifts < 1 || p.n_cs_shifts > 16 || p.n_cs_shifts > p.d))
    return why(SFT_EINVAL, "n_cs_shifts must lie in [1, min(16, d)]");
  if (p.mode == SFT_GENERAL_UNPRUNED && p.d > 4096)
    return why(SFT_EUNSUPPORTED, "SFT_GENERAL_UNPRUNED needs d <= 4096");
  if (p.reserved_ != 0) return why(SFT_EINVAL, "reserved_ must be 0");
  const int64_t M0 = p.N / p.d;
  if (p.mode == SFT_EXACT_ITER) {
    if (p.max_iters < 1 || p.max_iters > p.a_max)
      return why(SFT_EINVAL, "max_iters must lie in [1, a_max]");
    if ((M0 >> (p.max_iters - 1)) < 1) return why(SFT_EINVAL, "N/d too small for max_iters");
    // Levels 4..7 locate 5..8 aliases among 2^l d candidates from syndromes
    // that carry complex64 input's rounding; there the decision rule of
    // Algorithm 1 itself is decided by rounding, so no result is defined
    // well enough to reproduce.  Those levels are offered for complex128
    // input only.
    if (p.precision == SFT_MIXED && p.max_iters > 4)
      return why(SFT_EUNSUPPORTED,
                 "SFT_EXACT_ITER above four levels needs SFT_FP64 (complex128 input)");
  }
  if (M0 > kMaxM) return why(SFT_EUNSUPPORTED, "N/d above 2^26");
  return SFT_OK;
}

template <class T>
cudaError_t dalloc(T** ptr, size_t count, size_t* total) {
  *total += count * sizeof(T);
  return cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
}

void free_plan_memory(sft_plan_s* P) {
  void* ptrs[] = {P->tab.om_hi, P->tab.om_lo,    P->tab.tw,  P->tab.om_hi_ff, P->tab.om_lo_ff,
                  P->tab.cs_shifts, P->tab.xc_shifts, P->ws_base, P->x_stage, P->r_stage,
                  P->mlp_prop};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (int s = 0; s < sft::kMaxSub; ++s) {
    if (P->sub_st[s]) cudaStreamDestroy(P->sub_st[s]);
    if (P->sub_join[s]) cudaEventDestroy(P->sub_join[s]);
    if (P->sub_extracted[s]) cudaEventDestroy(P->sub_extracted[s]);
    P->sub_st[s] = nullptr;
    P->sub_join[s] = nullptr;
    P->sub_extracted[s] = nullptr;
  }
  if (P->sub_fork) cudaEventDestroy(P->sub_fork);
  P->sub_fork = nullptr;
}

// SplitMix64 (Steele, Lea, Flood 2014), output i of the stream of `seed`
uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// The r random shifts of the general path: r distinct values in [0, d) by
// a partial Fisher-Yates shuffle of 0..d-1, draw i exchanging positions i
// and i + (u_i mod (d - i)).
std::vector<int64_t> draw_cs_shifts(uint64_t seed, int64_t d, int r) {
  std::vector<int64_t> a((size_t)d), out((size_t)r);
  for (int64_t i = 0; i < d; ++i) a[(size_t)i] = i;
  for (int i = 0; i < r; ++i) {
    const int64_t j = i + (int64_t)(splitmix64(seed, (uint64_t)i) % (uint64_t)(d - i));
    std::swap(a[(size_t)i], a[(size_t)j]);
    out[(size_t)i] = a[(size_t)i];
  }
  return out;
}

// omega^e = e^{2 pi i e / N} and e^{-2 pi i q / M0}, rounded from long double
cudaError_t upload_tables(sft_plan_s* P, size_t* total) {
  const int64_t N = P->p.N, M0 = P->M0;
  const int lo_bits = P->log2N / 2;
  const int64_t n_lo = int64_t(1) << lo_bits, n_hi = N >> lo_bits;
  const long double two_pi = 6.283185307179586476925286766559005768L;
  std::vector<double2> lo(n_lo), hi(n_hi);
  for (int64_t i = 0; i < n_lo; ++i) {
    long double t = two_pi * (long double)i / (long double)N;
    lo[i] = make_double2((double)cosl(t), (double)sinl(t));
  }
  for (int64_t i = 0; i < n_hi; ++i) {
    long double t = two_pi * (long double)(i << lo_bits) / (long double)N;
    hi[i] = make_double2((double)cosl(t), (double)sinl(t));
  }
  cudaError_t e;
  if (sft::is_general_mode(P->p.mode)) {
    P->cs_host = draw_cs_shifts(P->p.seed, P->p.d, P->p.n_cs_shifts);
    if ((e = dalloc(&P->tab.cs_shifts, P->cs_host.size(), total)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(P->tab.cs_shifts, P->cs_host.data(), P->cs_host.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice)))
      return e;
  }
  if (!sft::is_general_mode(P->p.mode)) {
    // the shifts' row offsets in the compact samples: ITER level l reads
    // rows 0 and M0 / 2^l of its block; FIXED shift j is row j M0
    std::vector<int64_t> xs;
    if (P->p.mode == SFT_EXACT_FIXED) {
      for (int j = 0; j < 2 * P->p.a_max; ++j) xs.push_back((int64_t)j * P->M0);
    } else {
      for (int l = 0; l < P->levels; ++l) {
        xs.push_back(0);
        xs.push_back(P->M0 >> l);
      }
    }
    if ((e = dalloc(&P->tab.xc_shifts, xs.size(), total)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(P->tab.xc_shifts, xs.data(), xs.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice)))
      return e;
  }
  if ((e = dalloc(&P->tab.om_lo, n_lo, total)) != cudaSuccess) return e;
  if ((e = dalloc(&P->tab.om_hi, n_hi, total)) != cudaSuccess) return e;
  P->tab.om_lo_bits = lo_bits;
  if ((e = cudaMemcpy(P->tab.om_lo, lo.data(), n_lo * sizeof(double2), cudaMemcpyHostToDevice)))
    return e;
  if ((e = cudaMemcpy(P->tab.om_hi, hi.data(), n_hi * sizeof(double2), cudaMemcpyHostToDevice)))
    return e;
  if (P->p.precision != SFT_FP64) {
    // the same omega tables split into float-float for the FP32 peels
    auto split = [](double2 v) {
      const float xh = (float)v.x, yh = (float)v.y;
      return make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
    };
    std::vector<float4> lof(n_lo), hif(n_hi);
    for (int64_t i = 0; i < n_lo; ++i) lof[i] = split(lo[i]);
    for (int64_t i = 0; i < n_hi; ++i) hif[i] = split(hi[i]);
    if ((e = dalloc(&P->tab.om_lo_ff, n_lo, total)) != cudaSuccess) return e;
    if ((e = dalloc(&P->tab.om_hi_ff, n_hi, total)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(P->tab.om_lo_ff, lof.data(), n_lo * sizeof(float4), cudaMemcpyHostToDevice)))
      return e;
    if ((e = cudaMemcpy(P->tab.om_hi_ff, hif.data(), n_hi * sizeof(float4), cudaMemcpyHostToDevice)))
      return e;
  }
  if (P->p.precision == SFT_FP64) {
    std::vector<double2> tw(M0);
    for (int64_t q = 0; q < M0; ++q) {
      long double t = two_pi * (long double)q / (long double)M0;
      tw[q] = make_double2((double)cosl(t), (double)-sinl(t));
    }
    double2* d;
    if ((e = dalloc(&d, M0, total)) != cudaSuccess) return e;
    P->tab.tw = d;
    return cudaMemcpy(d, tw.data(), M0 * sizeof(double2), cudaMemcpyHostToDevice);
  }
  std::vector<float4> tw(M0);
  for (int64_t q = 0; q < M0; ++q) {
    long double t = two_pi * (long double)q / (long double)M0;
    long double c = cosl(t), s = -sinl(t);
    float ch = (float)c, sh = (float)s;
    tw[q] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(s - (long double)sh));
  }
  float4* d;
  if ((e = dalloc(&d, M0, total)) != cudaSuccess) return e;
  P->tab.tw = d;
  return cudaMemcpy(d, tw.data(), M0 * sizeof(float4), cudaMemcpyHostToDevice);
}

cudaError_t alloc_workspace(sft_plan_s* P, size_t* total) {
  const int esize = P->p.precision == SFT_FP64 ? 16 : 8;
  const size_t bytes = sft::layout_workspace(nullptr, nullptr, P->max_signals, P->M0, P->p.mode,
                                             P->p.a_max, P->p.n_cs_shifts, P->levels, esize);
  char* base = nullptr;
  cudaError_t e = dalloc(&base, bytes, total);
  if (e != cudaSuccess) return e;
  P->ws_base = base;
  sft::layout_workspace(&P->ws, base, P->max_signals, P->M0, P->p.mode, P->p.a_max,
                        P->p.n_cs_shifts, P->levels, esize);
  return cudaSuccess;
}

}  // namespace

namespace sft {
sft_status normalize_params(sft_params* p) { return fill_defaults(p); }
sft_status validate_params(const sft_params& p) { return validate(p); }
// Records `msg` as the calling thread's error detail (read back through
// sft_last_cuda_error).
void set_error_detail(const char* msg) { std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg); }
}  // namespace sft

extern "C" {

sft_status sft_params_default(sft_params* p, int64_t N, int64_t K, int64_t d, int32_t mode,
                              int32_t precision) {
  if (!p) return SFT_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->N = N;
  p->K = K;
  p->d = d;
  p->a_max = 4;
  p->max_iters = 4;
  p->mode = mode;
  p->precision = precision;
  p->a_max = 0;
  p->max_iters = 0;
  fill_defaults(p);
  return SFT_OK;
}

sft_status sft_plan_create(const sft_params* pin, int64_t max_signals, sft_plan_t* out) {
  if (!pin || !out || max_signals < 1) return SFT_EINVAL;
  *out = nullptr;
  sft_params p = *pin;
  fill_defaults(&p);
  sft_status st = validate(p);
  if (st != SFT_OK) return st;
  sft_plan_s* P = new (std::nothrow) sft_plan_s();
  if (!P) return SFT_ENOMEM;
  P->p = p;
  P->max_signals = max_signals;
  P->M0 = p.N / p.d;
  P->log2N = ilog2(p.N);
  P->log2M0 = ilog2(P->M0);
  P->levels = p.mode == SFT_EXACT_ITER ? p.max_iters : 1;
  size_t total = 0;
  cudaError_t e = upload_tables(P, &total);
  if (e == cudaSuccess) e = alloc_workspace(P, &total);
  if (e == cudaSuccess) e = sft::prepare_kernels(P);
  // the sub-batch streams and events (created here, outside any capture)
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->sub_fork, cudaEventDisableTiming);
  for (int s = 1; e == cudaSuccess && s < sft::kMaxSub; ++s) {
    e = cudaStreamCreateWithFlags(&P->sub_st[s], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->sub_join[s], cudaEventDisableTiming);
  }
  for (int s = 0; e == cudaSuccess && s < sft::kMaxSub; ++s)
    e = cudaEventCreateWithFlags(&P->sub_extracted[s], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    note_cuda(e);
    free_plan_memory(P);
    delete P;
    return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
  }
  P->device_bytes = total;
  *out = P;
  return SFT_OK;
}

static void drop_stage_recs(sft_plan_s* P);
static void free_event_pool(sft_plan_s* P);

sft_status sft_plan_get_params(sft_plan_t P, sft_params* out) {
  if (!P || !out) return SFT_EINVAL;
  *out = P->p;
  return SFT_OK;
}

void sft_plan_destroy(sft_plan_t P) {
  if (!P) return;
  cudaDeviceSynchronize();
  drop_stage_recs(P);
  free_event_pool(P);
  free_plan_memory(P);
  delete P;
}

size_t sft_plan_workspace_bytes(sft_plan_t P) { return P ? P->device_bytes : 0; }

int32_t sft_plan_launches_per_call(sft_plan_t P) { return P ? sft::launches_per_call(P) : 0; }

int32_t sft_plan_queue_lengths(sft_plan_t P, int64_t* out, int32_t cap) {
  if (!P || (cap > 0 && !out)) return -1;
  if (P->p.mode == SFT_GENERAL_UNPRUNED) return 0;
  const bool gen = P->p.mode == SFT_GENERAL;
  const int n = gen ? 3 : P->p.mode == SFT_EXACT_ITER ? P->levels : P->p.a_max;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  // each sub-batch keeps 16 counters: exact modes, level l (round l + 1) is
  // counter l; general mode, counter 1 the bins whose singular values are
  // computed, counters 0 and 2 the voted bins with one and with more aliases
  static const int kGen[3] = {1, 0, 2};
  int32_t c[16 * sft::kMaxSub];
  if (cudaMemcpy(c, P->ws.qcount, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  for (int i = 0; i < n && i < cap; ++i) {
    const int ci = gen ? kGen[i] : i;
    int64_t t = 0;
    for (int s = 0; s < P->last_sub; ++s) t += c[16 * s + ci];
    out[i] = t;
  }
  return n;
}

static sft_status reject(const char* fmt, long long a, long long b) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), fmt, a, b);
  return SFT_EINVAL;
}

static sft_status check_call(sft_plan_t P, int64_t n, const void* x, int64_t x_stride,
                             const sft_result* r) {
  if (!P || !x || !r) return reject("NULL plan, input or result (%lld %lld)", 0, 0);
  if (n < 1 || n > P->max_signals)
    return reject("n_signals %lld outside [1, max_signals = %lld]", n, P->max_signals);
  if (x_stride < P->p.N) return reject("x_stride %lld < N %lld", x_stride, P->p.N);
  if (r->cap < P->p.K || r->cap < 1) return reject("result cap %lld < K %lld", r->cap, P->p.K);
  if (!r->idx || !r->val || !r->count || !r->unresolved || !r->overflow)
    return reject("NULL result array (%lld %lld)", 0, 0);
  return SFT_OK;
}

static sft_status run_device(sft_plan_t P, int64_t n, const void* x, int64_t x_stride,
                             const sft_result* r, void* stream) {
  sft_status st = check_call(P, n, x, x_stride, r);
  if (st != SFT_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(P->ws.zero_base, 0, P->ws.zero_bytes, s);
  if (e == cudaSuccess) e = sft::launch_exact(P, n, x, x_stride, r, s);
  if (e != cudaSuccess) {
    note_cuda(e);
    return SFT_ECUDA;
  }
  return SFT_OK;
}

// Device address of page-locked host memory (nullptr for pageable memory).
static void* mapped(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of a failed query
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

static sft_status run_host(sft_plan_t P, int64_t n, const void* x_host, int64_t x_stride,
                           const sft_result* rh, void* stream) {
  sft_status st = check_call(P, n, x_host, x_stride, rh);
  if (st != SFT_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t elem = P->p.precision == SFT_FP64 ? 16 : 8;
  const int64_t cap = rh->cap;
  cudaError_t e = cudaSuccess;

  // inputs: read in place when page-locked (the kernels touch only the
  // samples of the shifts, a small fraction of each signal), else staged
  const void* xd = mapped(x_host);
  if (xd == nullptr) {
    const size_t xbytes = (size_t)n * (size_t)P->p.N * elem;
    if (P->x_stage_bytes < xbytes) {
      if (P->x_stage) cudaFree(P->x_stage);
      P->x_stage = nullptr;
      P->x_stage_bytes = 0;
      if ((e = cudaMalloc(&P->x_stage, xbytes)) != cudaSuccess) {
        note_cuda(e);
        return SFT_ENOMEM;
      }
      P->x_stage_bytes = xbytes;
    }
    const char* xh = static_cast<const char*>(x_host);
    if (x_stride == P->p.N || n == 1) {
      e = cudaMemcpyAsync(P->x_stage, xh, xbytes, cudaMemcpyHostToDevice, s);
    } else {
      const size_t row = (size_t)P->p.N * elem;
      e = cudaMemcpy2DAsync(P->x_stage, row, xh, (size_t)x_stride * elem, row, (size_t)n,
                            cudaMemcpyHostToDevice, s);
    }
    xd = P->x_stage;
    x_stride = P->p.N;
  }

  // results: written in place when every array is page-locked, else staged
  sft_result rd;
  rd.cap = cap;
  rd.idx = static_cast<int64_t*>(mapped(rh->idx));
  rd.val = static_cast<double*>(mapped(rh->val));
  rd.count = static_cast<int64_t*>(mapped(rh->count));
  rd.unresolved = static_cast<int32_t*>(mapped(rh->unresolved));
  rd.overflow = static_cast<int32_t*>(mapped(rh->overflow));
  const bool in_place = rd.idx && rd.val && rd.count && rd.unresolved && rd.overflow;
  if (!in_place) {
    const size_t rbytes = (size_t)n * (size_t)cap * 24 + (size_t)n * 16;
    if (P->r_stage_bytes < rbytes) {
      if (P->r_stage) cudaFree(P->r_stage);
      P->r_stage = nullptr;
      P->r_stage_bytes = 0;
      if ((e = cudaMalloc(&P->r_stage, rbytes)) != cudaSuccess) {
        note_cuda(e);
        return SFT_ENOMEM;
      }
      P->r_stage_bytes = rbytes;
    }
    char* rs = static_cast<char*>(P->r_stage);
    rd.idx = reinterpret_cast<int64_t*>(rs);
    rd.val = reinterpret_cast<double*>(rs + (size_t)n * cap * 8);
    rd.count = reinterpret_cast<int64_t*>(rs + (size_t)n * cap * 24);
    rd.unresolved = reinterpret_cast<int32_t*>(rs + (size_t)n * cap * 24 + (size_t)n * 8);
    rd.overflow = reinterpret_cast<int32_t*>(rs + (size_t)n * cap * 24 + (size_t)n * 12);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(P->ws.zero_base, 0, P->ws.zero_bytes, s);
  // host-resident samples are read over NVLink-C2C, where wide requests pay
  P->x_on_host = xd != P->x_stage;
  P->r_on_host = in_place;
  if (e == cudaSuccess) e = sft::launch_exact(P, n, xd, x_stride, &rd, s);
  P->x_on_host = false;
  P->r_on_host = false;
  if (!in_place) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rh->idx, rd.idx, (size_t)n * cap * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rh->val, rd.val, (size_t)n * cap * 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rh->count, rd.count, (size_t)n * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rh->unresolved, rd.unresolved, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rh->overflow, rd.overflow, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    note_cuda(e);
    return SFT_ECUDA;
  }
  return SFT_OK;
}

static sft_status want_mode(sft_plan_t P, bool general) {
  if (!P) return reject("NULL plan (%lld %lld)", 0, 0);
  if (sft::is_general_mode(P->p.mode) != general)
    return reject(general ? "plan mode %lld is not a general mode (%lld)"
                          : "plan mode %lld is a general mode (%lld): use sft_general",
                  P->p.mode, 0);
  return SFT_OK;
}

sft_status sft_exact(sft_plan_t P, int64_t n, const void* x, int64_t x_stride,
                     const sft_result* r, void* stream) {
  sft_status st = want_mode(P, false);
  return st != SFT_OK ? st : run_device(P, n, x, x_stride, r, stream);
}

sft_status sft_exact_host(sft_plan_t P, int64_t n, const void* x_host, int64_t x_stride,
                          const sft_result* rh, void* stream) {
  sft_status st = want_mode(P, false);
  return st != SFT_OK ? st : run_host(P, n, x_host, x_stride, rh, stream);
}

sft_status sft_general(sft_plan_t P, int64_t n, const void* x, int64_t x_stride,
                       const sft_result* r, void* stream) {
  sft_status st = want_mode(P, true);
  return st != SFT_OK ? st : run_device(P, n, x, x_stride, r, stream);
}

sft_status sft_general_host(sft_plan_t P, int64_t n, const void* x_host, int64_t x_stride,
                            const sft_result* rh, void* stream) {
  sft_status st = want_mode(P, true);
  return st != SFT_OK ? st : run_host(P, n, x_host, x_stride, rh, stream);
}

int32_t sft_plan_cs_shifts(sft_plan_t P, int64_t* out, int32_t cap) {
  if (!P) return -1;
  const int32_t n = (int32_t)P->cs_host.size();
  for (int32_t i = 0; i < n && i < cap && out; ++i) out[i] = P->cs_host[(size_t)i];
  return n;
}

static void drop_stage_recs(sft_plan_s* P) {
  P->stage_recs.clear();
  P->events_used = 0;
}

static void free_event_pool(sft_plan_s* P) {
  for (cudaEvent_t e : P->event_pool) cudaEventDestroy(e);
  P->event_pool.clear();
  P->events_used = 0;
}

sft_status sft_plan_set_sub_batches(sft_plan_t P, int32_t n) {
  if (!P || n < 0 || n > sft::kMaxSub) return SFT_EINVAL;
  P->sub_batches = n;
  return SFT_OK;
}

int32_t sft_plan_sub_batches(sft_plan_t P, int64_t n_signals) {
  return P ? sft::sub_batches_for(P, n_signals) : 0;
}

sft_status sft_plan_set_quad_decoders(sft_plan_t P, int32_t enable) {
  if (!P) return SFT_EINVAL;
  P->quad_ok = enable != 0;
  return SFT_OK;
}

sft_status sft_plan_set_profiling(sft_plan_t P, int32_t enable) {
  if (!P) return SFT_EINVAL;
  if (!enable) {
    cudaDeviceSynchronize();
    drop_stage_recs(P);
  }
  P->profiling = enable != 0;
  return SFT_OK;
}

sft_status sft_plan_stage_times(sft_plan_t P, int32_t cap, const char** names, double* ms,
                                int64_t* launches, int32_t* n) {
  if (!P || !n || cap < 0 || (cap > 0 && (!names || !ms || !launches))) return SFT_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    note_cuda(e);
    return SFT_ECUDA;
  }
  std::vector<const char*> nm;
  std::vector<double> tot;
  std::vector<int64_t> cnt;
  for (auto& r : P->stage_recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.t0, r.t1) != cudaSuccess) continue;
    size_t i = 0;
    while (i < nm.size() && std::strcmp(nm[i], r.name) != 0) ++i;
    if (i == nm.size()) {
      nm.push_back(r.name);
      tot.push_back(0.0);
      cnt.push_back(0);
    }
    tot[i] += t;
    cnt[i] += 1;
  }
  drop_stage_recs(P);
  *n = (int32_t)nm.size();
  for (int32_t i = 0; i < cap && i < (int32_t)nm.size(); ++i) {
    names[i] = nm[i];
    ms[i] = tot[i];
    launches[i] = cnt[i];
  }
  return SFT_OK;
}

sft_status sft_plan_stage_timeline(sft_plan_t P, int32_t cap, const char** names, int32_t* sub,
                                   double* t0_ms, double* t1_ms, int32_t* n) {
  if (!P || !n || cap < 0 || (cap > 0 && (!names || !sub || !t0_ms || !t1_ms))) return SFT_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    note_cuda(e);
    return SFT_ECUDA;
  }
  int32_t k = 0;
  for (auto& r : P->stage_recs) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, P->stage_recs.front().t0, r.t0) != cudaSuccess ||
        cudaEventElapsedTime(&b, P->stage_recs.front().t0, r.t1) != cudaSuccess)
      continue;
    if (k < cap) {
      names[k] = r.name;
      sub[k] = r.sub;
      t0_ms[k] = a;
      t1_ms[k] = b;
    }
    ++k;
  }
  drop_stage_recs(P);
  *n = k;
  return SFT_OK;
}

sft_status sft_device_math_check(const double* x, int64_t n, double* out, int32_t which,
                                 void* stream) {
  if (n < 0 || which < 0 || which > 2 || (n > 0 && (x == nullptr || out == nullptr)))
    return SFT_EINVAL;
  if (n == 0) return SFT_OK;
  const cudaError_t e = sft::launch_selfcheck(x, n, out, which, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    note_cuda(e);
    return SFT_ECUDA;
  }
  return SFT_OK;
}

const char* sft_strerror(sft_status s) {
  switch (s) {
    case SFT_OK: return "SFT_OK";
    case SFT_EINVAL: return "SFT_EINVAL: invalid argument";
    case SFT_ENOMEM: return "SFT_ENOMEM: allocation failed";
    case SFT_ECUDA: return "SFT_ECUDA: CUDA call failed";
    case SFT_ETIMEOUT: return "SFT_ETIMEOUT: bounded device wait expired";
    case SFT_EUNSUPPORTED: return "SFT_EUNSUPPORTED: not supported by this build";
  }
  return "unknown sft_status";
}

const char* sft_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
