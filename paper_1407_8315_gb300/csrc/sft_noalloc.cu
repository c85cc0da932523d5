// sft_noalloc.cu -- sft_exact_noalloc: the exactly K-sparse transform for
// callers that must not allocate device memory.
//
// Who needs this.  Some callers cannot call cudaMalloc/cudaFree at the point
// where they want a transform: a component that lives inside another
// framework's memory manager (which owns every device byte and forbids raw
// allocations behind its back), a latency-critical loop where cudaFree's
// implicit device-wide synchronisation or an allocation failure halfway
// through is unacceptable, or an embedded deployment with a fixed memory
// budget decided at start-up.  A plan (sft_plan_create) allocates its tables
// and workspace, so those callers cannot use it.
//
// What it does instead.  The tables and the workspace of one call live in
// one file-scope __device__ array of SFT_NOALLOC_SCRATCH_BYTES bytes.  The
// CUDA runtime creates that array when the library's module is loaded on a
// device, and every device that loads the library keeps it until the process
// exits.  Host code cannot use the array's name as a device address (on the
// host it only names a stand-in object), so the first call on each device
// asks the runtime for the array's device address with
// cudaGetSymbolAddress, with that device current, and remembers it together
// with the identity of the device's current context.  The library's module
// is loaded lazily, so that first call is also where the array's memory is
// committed on the device.  It should therefore happen at start-up, before
// any stream capture and before another memory manager reserves the device.
// If the context is later destroyed (cudaDeviceReset) and a new one created,
// the module is loaded again and the array may sit at a new address, with
// the kernels' raised shared-memory limits gone: a call that finds a context
// other than the remembered one repeats the look-up and the set-up.
//
// Every call shares the same array and leaves its contents behind: the call
// rebuilds the tables and clears the per-call counters itself.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array and corrupt each other; callers
// must serialise them.
#include <cuda.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "sft_internal.h"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[SFT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// per device: the array's address in the context it was looked up in
struct ScratchSlot {
  unsigned long long ctx_id;
  void* ptr;
};
ScratchSlot g_scratch_dev[kMaxDevices] = {};

char* noalloc_msg() {
  thread_local char buf[256];
  return buf;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int lg2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// Tables of omega^e (two-level) and of the FFT twiddles e^{-2 pi i q / M0},
// written into the scratch by the device (the plan path computes the same
// values on the host; both are correctly rounded to within an ulp).
__device__ __forceinline__ float4 ff_split(double c, double s) {
  const float ch = (float)c, sh = (float)s;
  return make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
}

__global__ void k_noalloc_tables(double2* om_lo, int64_t n_lo, double2* om_hi, int64_t n_hi,
                                 int lo_bits, int64_t N, void* tw, int64_t M0, int ff,
                                 float4* om_lo_ff, float4* om_hi_ff) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s, c;
  if (i < n_lo) {
    sincospi(2.0 * (double)i / (double)N, &s, &c);
    om_lo[i] = make_double2(c, s);
    if (ff) om_lo_ff[i] = ff_split(c, s);
  }
  if (i < n_hi) {
    sincospi(2.0 * (double)(i << lo_bits) / (double)N, &s, &c);
    om_hi[i] = make_double2(c, s);
    if (ff) om_hi_ff[i] = ff_split(c, s);
  }
  if (i < M0) {
    sincospi(2.0 * (double)i / (double)M0, &s, &c);
    s = -s;
    if (ff) {
      const float ch = (float)c, sh = (float)s;
      reinterpret_cast<float4*>(tw)[i] =
          make_float4(ch, (float)(c - (double)ch), sh, (float)(s - (double)sh));
    } else {
      reinterpret_cast<double2*>(tw)[i] = make_double2(c, s);
    }
  }
}

sft_status fail(sft_status st, const char* msg) {
  sft::set_error_detail(msg);
  return st;
}

// The unique identity of the calling thread's current context (driver entry
// points resolved through the runtime, so the library needs no link to the
// driver library).  Called with g_setup_mu held.
cudaError_t current_context_id(unsigned long long* id) {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (get_current == nullptr || get_id == nullptr) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                     cudaEnableDefault, &q1);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorNotSupported;
    get_current = reinterpret_cast<GetCurrent>(f1);
    get_id = reinterpret_cast<GetId>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return cudaErrorDeviceUninitialized;
  if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

// Device address of the scratch array on the current device, in its current
// context.  The look-up (which also loads the module and so commits the
// array) and the kernels' shared-memory set-up run on the first call in a
// context and again whenever the device's context has changed.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  // makes the device's primary context current (created if need be)
  void* ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  unsigned long long id = 0;
  e = current_context_id(&id);
  if (e != cudaSuccess) return e;
  ScratchSlot& slot = g_scratch_dev[dev];
  if (slot.ptr == nullptr || slot.ctx_id != id) {
    // largest dynamic shared memory any gather/FFT launch of this build asks for
    for (int prec = 0; prec < 2; ++prec) {
      sft_plan_s tmp;
      tmp.p.precision = prec;
      tmp.M0 = 8192;
      e = sft::prepare_kernels(&tmp);
      if (e != cudaSuccess) return e;
    }
    slot.ctx_id = id;
    slot.ptr = ptr;
  }
  *out = slot.ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" sft_status sft_exact_noalloc(const sft_params* pin, int64_t n, const void* x,
                                        int64_t x_stride, const sft_result* r, void* stream) {
  if (!pin || !x || !r) return fail(SFT_EINVAL, "NULL params, input or result");
  sft_params p = *pin;
  // defaults and validation, as sft_plan_create applies them
  if (p.a_max == 0) p.a_max = 4;
  if (p.max_iters == 0) p.max_iters = p.a_max;
  const bool fp64 = p.precision == SFT_FP64;
  if (!(p.zero_tol > 0)) p.zero_tol = fp64 ? 1e-10 : 1e-6;
  if (!(p.root_tol > 0)) p.root_tol = 0.1;
  if (!(p.res_tol > 0)) p.res_tol = fp64 ? 1e-9 : 1e-6;
  if (!pow2(p.N) || p.N < 8 || p.N > (int64_t(1) << 30) || p.K < 0 || p.K > p.N ||
      !pow2(p.d) || p.d > p.N || p.a_max < 1 || p.a_max > 8 || p.reserved_ != 0 ||
      (p.precision != SFT_FP64 && p.precision != SFT_MIXED))
    return fail(SFT_EINVAL, "invalid parameters");
  if (p.mode != SFT_EXACT_ITER && p.mode != SFT_EXACT_FIXED)
    return fail(p.mode == SFT_GENERAL ? SFT_EUNSUPPORTED : SFT_EINVAL, "mode not supported");
  if (p.mode == SFT_EXACT_FIXED && p.a_max > 4 && p.a_max != 8)
    return fail(SFT_EUNSUPPORTED, "SFT_EXACT_FIXED takes a_max <= 4 or a_max = 8");
  const int64_t M0 = p.N / p.d;
  if (M0 > 8192) return fail(SFT_EUNSUPPORTED, "N/d above 8192");
  if (p.mode == SFT_EXACT_ITER &&
      (p.max_iters < 1 || p.max_iters > p.a_max || (M0 >> (p.max_iters - 1)) < 1))
    return fail(SFT_EINVAL, "invalid max_iters");
  if (p.mode == SFT_EXACT_ITER && p.precision == SFT_MIXED && p.max_iters > 4)
    return fail(SFT_EUNSUPPORTED,
                "SFT_EXACT_ITER above four levels needs SFT_FP64 (complex128 input)");
  if (n < 1 || x_stride < p.N) return fail(SFT_EINVAL, "n_signals < 1 or x_stride < N");
  if (r->cap < p.K || r->cap < 1 || !r->idx || !r->val || !r->count || !r->unresolved ||
      !r->overflow)
    return fail(SFT_EINVAL, "result cap < K or NULL result array");

  // scratch layout: tables, then the workspace of n signals
  const int log2N = lg2(p.N);
  const int lo_bits = log2N / 2;
  const int64_t n_lo = int64_t(1) << lo_bits, n_hi = p.N >> lo_bits;
  size_t off = 0;
  const size_t o_lo = off;
  off = align256(off + n_lo * 16);
  const size_t o_hi = off;
  off = align256(off + n_hi * 16);
  const size_t o_tw = off;
  off = align256(off + M0 * 16);
  const size_t o_loff = off;
  off = align256(off + n_lo * 16);
  const size_t o_hiff = off;
  off = align256(off + n_hi * 16);
  const size_t o_ws = off;
  off += sft::layout_workspace(nullptr, nullptr, n, M0, p.mode, p.a_max);
  if (off > (size_t)SFT_NOALLOC_SCRATCH_BYTES) {
    std::snprintf(noalloc_msg(), 256,
                  "sft_exact_noalloc: %lld signals of N/d = %lld need %zu bytes of scratch; the "
                  "static maximum is %zu (use fewer signals per call)",
                  (long long)n, (long long)M0, off, (size_t)SFT_NOALLOC_SCRATCH_BYTES);
    return fail(SFT_EINVAL, noalloc_msg());
  }

  void* base_v = nullptr;
  cudaError_t e = scratch_address(&base_v);
  if (e != cudaSuccess) {
    std::snprintf(noalloc_msg(), 256, "scratch set-up: %s", cudaGetErrorString(e));
    return fail(SFT_ECUDA, noalloc_msg());
  }
  char* base = static_cast<char*>(base_v);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // a plan object that only points into the scratch (nothing is allocated)
  sft_plan_s P;
  P.p = p;
  P.max_signals = n;
  P.M0 = M0;
  P.log2N = log2N;
  P.log2M0 = lg2(M0);
  P.levels = p.mode == SFT_EXACT_ITER ? p.max_iters : 1;
  P.tab.om_lo = reinterpret_cast<double2*>(base + o_lo);
  P.tab.om_hi = reinterpret_cast<double2*>(base + o_hi);
  P.tab.om_lo_bits = lo_bits;
  P.tab.tw = base + o_tw;
  P.tab.om_lo_ff = reinterpret_cast<float4*>(base + o_loff);
  P.tab.om_hi_ff = reinterpret_cast<float4*>(base + o_hiff);
  sft::layout_workspace(&P.ws, base + o_ws, n, M0, p.mode, p.a_max);

  const int64_t nt = n_lo > n_hi ? n_lo : n_hi;
  const int64_t ntab = nt > M0 ? nt : M0;
  k_noalloc_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(
      P.tab.om_lo, n_lo, P.tab.om_hi, n_hi, lo_bits, p.N, P.tab.tw, M0, fp64 ? 0 : 1,
      P.tab.om_lo_ff, P.tab.om_hi_ff);
  e = cudaGetLastError();
  // counters and thresholds that the kernels accumulate into start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(P.ws.zero_base, 0, P.ws.zero_bytes, st);
  if (e == cudaSuccess) e = sft::launch_exact(&P, n, x, x_stride, r, st);
  if (e != cudaSuccess) {
    std::snprintf(noalloc_msg(), 256, "launch: %s", cudaGetErrorString(e));
    return fail(SFT_ECUDA, noalloc_msg());
  }
  return SFT_OK;
}
