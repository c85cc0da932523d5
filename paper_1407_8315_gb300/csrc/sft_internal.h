// sft_internal.h -- plan layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sft.h"
#include "sft_slots.h"

namespace sft {

// Algorithm 2 with or without the pruning strategy
inline bool is_general_mode(int mode) {
  return mode == SFT_GENERAL || mode == SFT_GENERAL_UNPRUNED;
}

// A call may be split into up to kMaxSub sub-batches of signals, each on
// its own stream (its launches overlap the others'), each with its own
// block of 16 queue counters.
constexpr int kMaxSub = 4;

// Device workspace of one call for up to B signals.  Per signal:
//   held[2]   ping-pong syndrome buffers, `held_elems` double2 each
//             (ITER level l keeps rows j < 2l+2 of length M_l; FIXED keeps
//             2 a_max rows of length M0)
//   T[2]      unsolved-bin flags per level, M0 bytes each
//   queue[2]  active (signal, bin) pairs awaiting decoding, M0 int2 each
//   slot_*    frequencies recovered so far, filed by their level-0 bin
//             k0 = s mod M0 (at most kSlots = 8 per bin): count, location, value
//   ymax2     bit pattern of max_k |Y_{d,0}[k]|^2 (zero threshold)
//   flags     bit 0: a level-0 bin received more than kSlots frequencies
// plus qcount[16 kMaxSub], the queue fill counters of one call (16 per
// sub-batch).  ymax2, flags, qcount and slot_cnt form one contiguous region
// cleared before each call.
struct Workspace {
  void* held[2] = {nullptr, nullptr};  // double2 or float-float float4 elements
  int64_t held_elems = 0;
  uint8_t* T[2] = {nullptr, nullptr};
  int2* queue[2] = {nullptr, nullptr};
  uint8_t* slot_cnt = nullptr;
  int64_t* slot_s = nullptr;
  void* slot_p = nullptr;  // double2 (FP64 path) or float-float float4 (mixed path)
  unsigned long long* ymax2 = nullptr;
  int32_t* flags = nullptr;
  int32_t* qcount = nullptr;
  void* zero_base = nullptr;  // ymax2 | flags | qcount | slot_cnt
  size_t zero_bytes = 0;
  void* fft4 = nullptr;  // four-step FFT intermediate (only when N/d > 8192)
  double* sv = nullptr;  // general path: a_m singular values per bin
  void* xc = nullptr;    // exact paths: the call's samples, shift-major (input type)
  int64_t xc_sig = 0;    // elements of xc per signal
  // bytes per signal of the per-signal arrays (sub-batch views)
  int64_t M0 = 0, fft4_sig_bytes = 0, sv_sig = 0, xc_sig_bytes = 0;
};

// The workspace seen by signals [b0, ...) of a call as sub-batch `sub`:
// every per-signal array offset by b0 signals, the queues by b0 M0 entries
// and the counters by 16 sub.
inline Workspace sub_workspace(const Workspace& W, int64_t b0, int sub) {
  Workspace V = W;
  const int64_t M0 = W.M0;
  for (int i = 0; i < 2; ++i) {
    if (W.held[i]) V.held[i] = static_cast<char*>(W.held[i]) + b0 * W.held_elems * 16;
    if (W.T[i]) V.T[i] = W.T[i] + b0 * M0;
    if (W.queue[i]) V.queue[i] = W.queue[i] + b0 * M0;
  }
  V.slot_cnt = W.slot_cnt + b0 * M0;
  V.slot_s = W.slot_s + b0 * M0 * kSlots;
  V.slot_p = static_cast<char*>(W.slot_p) + b0 * M0 * kSlots * 16;
  V.ymax2 = W.ymax2 + b0;
  V.flags = W.flags + b0;
  V.qcount = W.qcount + 16 * sub;
  if (W.fft4) V.fft4 = static_cast<char*>(W.fft4) + b0 * W.fft4_sig_bytes;
  if (W.sv) V.sv = W.sv + b0 * W.sv_sig;
  if (W.xc) V.xc = static_cast<char*>(W.xc) + b0 * W.xc_sig_bytes;
  return V;
}

// Lays the workspace of B signals out from `base` (or only sizes it when
// base is null) and returns its byte size; every array is 256-byte aligned.
//
// With xc_esize > 0 (exact modes; the input element size) the workspace also
// holds the compact copy of the samples each call reads: ITER, `levels`
// blocks [2][M0 / 2^l]; FIXED, [2 a_max][M0].
inline size_t layout_workspace(Workspace* W, char* base, int64_t B, int64_t M0, int mode,
                               int a_max, int n_cs = 0, int levels = 0, int xc_esize = 0) {
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const bool gen = is_general_mode(mode);
  const int64_t held_elems = mode == SFT_EXACT_FIXED ? 2 * a_max * M0
                             : gen                   ? (2 * a_max + n_cs) * M0
                                                     : 2 * M0;
  const int nbuf = mode == SFT_EXACT_ITER ? 2 : 1;  // only ITER keeps two levels
  size_t off = 0;
  size_t o_held[2] = {0, 0}, o_T[2] = {0, 0}, o_q[2];
  for (int i = 0; i < 2; ++i) {
    if (i < nbuf) {
      o_held[i] = off;
      off = al(off + (size_t)(B * held_elems) * 16);
      o_T[i] = off;
      off = al(off + (size_t)(B * M0));
    }
    o_q[i] = off;
    off = al(off + (size_t)(B * M0) * 8);
  }
  const size_t o_zero = off;
  const size_t zero_bytes = (size_t)B * 16 + 64 * kMaxSub + (size_t)(B * M0);
  off = al(off + zero_bytes);
  const size_t o_ss = off;
  off = al(off + (size_t)(B * M0 * kSlots) * 8);
  const size_t o_sp = off;
  off = al(off + (size_t)(B * M0 * kSlots) * 16);
  // singular values of every bin (general path)
  const size_t o_sv = off;
  if (mode == SFT_GENERAL) off = al(off + (size_t)(B * M0 * a_max) * 8);
  // four-step FFT intermediate: one M0-point plane per shift of a launch
  const int nsh = mode == SFT_EXACT_FIXED ? 2 * a_max
                  : gen                   ? (2 * a_max > n_cs ? 2 * a_max : n_cs)
                                          : 2;
  const size_t o_f4 = off;
  if (M0 > 8192) off = al(off + (size_t)(B * nsh * M0) * 16);
  // compact samples of the exact modes
  int64_t xc_sig = 0;
  if (xc_esize > 0 && mode == SFT_EXACT_FIXED) xc_sig = 2 * a_max * M0;
  if (xc_esize > 0 && mode == SFT_EXACT_ITER)
    for (int l = 0; l < levels; ++l) xc_sig += 2 * (M0 >> l);
  const size_t o_xc = off;
  if (xc_sig > 0) off = al(off + (size_t)(B * xc_sig) * (size_t)xc_esize);
  if (W != nullptr && base != nullptr) {
    W->held_elems = held_elems;
    for (int i = 0; i < 2; ++i) {
      W->held[i] = i < nbuf ? base + o_held[i] : nullptr;
      W->T[i] = i < nbuf ? reinterpret_cast<uint8_t*>(base + o_T[i]) : nullptr;
      W->queue[i] = reinterpret_cast<int2*>(base + o_q[i]);
    }
    char* z = base + o_zero;
    W->zero_base = z;
    W->zero_bytes = zero_bytes;
    W->ymax2 = reinterpret_cast<unsigned long long*>(z);
    W->flags = reinterpret_cast<int32_t*>(z + (size_t)B * 8);
    W->qcount = reinterpret_cast<int32_t*>(z + (size_t)B * 16);
    W->slot_cnt = reinterpret_cast<uint8_t*>(z + (size_t)B * 16 + 64 * kMaxSub);
    W->slot_s = reinterpret_cast<int64_t*>(base + o_ss);
    W->slot_p = base + o_sp;
    W->fft4 = M0 > 8192 ? base + o_f4 : nullptr;
    W->sv = mode == SFT_GENERAL ? reinterpret_cast<double*>(base + o_sv) : nullptr;
    W->xc = xc_sig > 0 ? base + o_xc : nullptr;
    W->xc_sig = xc_sig;
    W->M0 = M0;
    W->fft4_sig_bytes = (int64_t)nsh * M0 * 16;
    W->sv_sig = M0 * a_max;
    W->xc_sig_bytes = xc_sig * xc_esize;
  }
  return off;
}

struct Tables {
  double2* om_hi = nullptr;  // omega^(i << lo_bits)
  double2* om_lo = nullptr;  // omega^i, i < 2^lo_bits
  int om_lo_bits = 0;
  void* tw = nullptr;        // e^{-2 pi i q / M0}: double2 (FP64) or float4 (FF)
  float4* om_hi_ff = nullptr;  // the omega tables as float-float (mixed path only)
  float4* om_lo_ff = nullptr;
  int64_t* cs_shifts = nullptr;  // general path: the r random shifts n_l (device)
  int64_t* xc_shifts = nullptr;  // exact paths: row offsets of the shifts in the compact samples
};

}  // namespace sft

namespace sft {
// Events bracketing one launch (profiling only).
struct StageRec {
  const char* name;
  cudaEvent_t t0, t1;
  int sub;  // sub-batch (stream) of the launch
};
}  // namespace sft

struct sft_plan_s {
  sft_params p;
  int64_t max_signals = 0;
  int64_t M0 = 0;
  int log2N = 0, log2M0 = 0;
  int levels = 0;  // ITER: max_iters; FIXED: 1
  sft::Tables tab;
  sft::Workspace ws;
  void* ws_base = nullptr;  // one allocation holding the workspace
  size_t device_bytes = 0;
  // staging for the host entry point (allocated on first use)
  void* x_stage = nullptr;
  size_t x_stage_bytes = 0;
  void* r_stage = nullptr;
  size_t r_stage_bytes = 0;
  std::vector<int64_t> cs_host;  // general path: the random shifts (host copy)
  // heterogeneous batches: per-signal input pointers and result buffers
  // (device tables; null for the strided single-shape entry points)
  const void* const* x_table = nullptr;
  const sft_result* r_table = nullptr;
  const int64_t* K_table = nullptr;  // per-signal K for the general vote
  // launch shape chosen by the batch autotuner
  int dec_ctas_per_sm = 8;
  // the four-lane decoders of three and four aliases: enabled on this plan
  // (sft_plan_set_quad_decoders), and in use for the current call (one
  // sub-batch: nothing else runs beside the decoders)
  bool quad_ok = false;
  bool quad_now = false;
  // points per thread of the one-CTA FFT (8: M/8 threads, radix-8 passes,
  // at most 64 registers, twice the resident warps of 16 points per thread;
  // measured faster on every level of the exact transforms)
  int fft_pts = 8;
  // the current call reads page-locked host memory in place (the compact
  // extraction then asks for full-width L2 lines)
  bool x_on_host = false;
  // the current call writes its results in place into page-locked host
  // memory (the finalize then stages them for coalesced stores)
  bool r_on_host = false;
  // learned proposal (general plans): the attached network (not owned) and
  // 8 proposed candidates t per queued bin (int16, -1 = none)
  struct sft_mlp_s* mlp = nullptr;
  int16_t* mlp_prop = nullptr;
  // sub-batches per call (0: chosen from the batch size) and their streams
  // (created on first use; stream 0 is the caller's)
  int sub_batches = 0;
  int last_sub = 1;  // sub-batches of the last call (its queue counters)
  int cur_sub = 0;   // sub-batch being enqueued (profiling records)
  cudaStream_t sub_st[sft::kMaxSub] = {};
  cudaEvent_t sub_fork = nullptr;
  cudaEvent_t sub_join[sft::kMaxSub] = {};
  // host-resident input: sub-batch s + 1 extracts its samples after sub-batch
  // s has (the extractions share the host link; chained, each sub-batch's
  // computation overlaps the next one's extraction).  sub_extracted[s] is
  // recorded after sub-batch s's extraction; sub_extract_now is the event
  // of the sub-batch being enqueued (null outside a split host call).
  cudaEvent_t sub_extracted[sft::kMaxSub] = {};
  cudaEvent_t sub_extract_now = nullptr;
  // profiling
  bool profiling = false;
  std::vector<sft::StageRec> stage_recs;   // records since the last read
  std::vector<cudaEvent_t> event_pool;     // reused across reads
  size_t events_used = 0;
};

namespace sft {
// One exactly sparse signal (ITER, mixed precision, a_max <= 4, N/d <= 4096)
// of a heterogeneous batch, as the persistent batch kernel sees it: the
// signal's input and result buffers, the shape and tables of its group's
// plan, and its own slice of that plan's workspace.
struct PSig {
  const float2* x;
  int64_t N, d0, M0;
  int levels, log2M0;
  double zero_tol, root_tol, res_tol;
  const float4* tw;                  // e^{-2 pi i q / M0}, float-float
  const double2* om_hi;              // omega tables (FP64 and float-float)
  const double2* om_lo;
  const float4* om_hi_ff;
  const float4* om_lo_ff;
  int om_lo_bits;
  void* held[2];                     // float4 rows, held_elems each
  int64_t held_elems;
  uint8_t* T[2];
  uint8_t* slot_cnt;
  int64_t* slot_s;
  float4* slot_p;
  unsigned long long* ymax2;
  int32_t* flags;
  sft_result r;                      // one signal's result buffers
};
// Largest N/d the persistent kernel takes (one CTA's FFT: 128 threads x 32 points).
constexpr int64_t kPersistMaxM = 4096;
// Enqueue the persistent kernel over n signals (device descriptors `sigs`,
// processed in the order `order`, items claimed through the device counter
// `head`, which the call clears); `ctas` CTAs (0: as many as fit).
cudaError_t launch_exact_persistent(const PSig* sigs, const int* order, int n, int* head, int ctas,
                                    cudaStream_t st);
// CTAs of the persistent kernel resident per SM (its launch bound).
int persistent_ctas_per_sm();

// Enqueue one sft_exact call (all launches) on `stream`.
cudaError_t launch_exact(sft_plan_s* plan, int64_t n_signals, const void* x, int64_t x_stride,
                         const sft_result* r, cudaStream_t stream);
// One-time per-plan kernel attributes (dynamic shared memory limits).
cudaError_t prepare_kernels(sft_plan_s* plan);
int launches_per_call(const sft_plan_s* plan);
// sub-batches of a call of B signals (sft_plan_set_sub_batches)
int sub_batches_for(const sft_plan_s* plan, int64_t B);
// Gather + FFT of `nshift` shifts (consecutive from shift0, or shift_list)
// into rows row0.. of `out`, either precision; `stage` names the profiling
// stage (nullptr: the level's default name).
void launch_gather_fft_any(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int64_t d,
                           int log2M, int shift0, int nshift, void* out, int64_t out_row, int row0,
                           bool want_ymax, cudaStream_t st, const int64_t* shift_list,
                           const char* stage);
// The general path (Algorithm 2) of one call, before k_finalize (with the
// learned proposal when a network is attached).
void launch_general(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                    cudaStream_t st);
// The general path up to the vote, then the features of every voted bin
// (training data for the learned proposal).
void launch_general_features(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                             float* feat, int32_t* rows, int64_t cap_rows, cudaStream_t st);
// Learned proposal kernels (sft_mlp.cu): features + forward + the 2 a_k
// largest support logits of every queued voted bin into P->mlp_prop; and
// the features alone, written out.
void mlp_propose(sft_plan_s* P, int64_t B, int nsm, cudaStream_t st);
cudaError_t launch_selfcheck(const double* x, int64_t n, double* out, int which,
                             cudaStream_t st);
void mlp_features(sft_plan_s* P, int64_t B, int nsm, float* feat, int32_t* rows, int64_t cap_rows,
                  cudaStream_t st);
// Sets the calling thread's error detail returned by sft_last_cuda_error.
void set_error_detail(const char* msg);
// Defaults of zero fields (as sft_plan_create applies them) and validation.
sft_status normalize_params(sft_params* p);
sft_status validate_params(const sft_params& p);
// Profiling brackets around one launch (no-ops unless plan->profiling).
void stage_begin(sft_plan_s* plan, const char* name, cudaStream_t st);
void stage_end(sft_plan_s* plan, cudaStream_t st);
}  // namespace sft
