// sft_internal.h -- plan layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/sft.h"

namespace sft {

// Device workspace of one plan for up to `max_signals` signals.  Per signal:
//   held[2]   ping-pong syndrome buffers, `held_elems` double2 each
//             (ITER level l keeps rows j < 2l+2 of length M_l; FIXED keeps
//             2 a_max rows of length M0)
//   T[2]      unsolved-bin flags per level, M0 bytes each
//   slot_*    frequencies recovered so far, filed by their level-0 bin
//             k0 = s mod M0 (at most 4 per bin): count, location, value
//   ymax2     bit pattern of max_k |Y_{d,0}[k]|^2 (zero threshold)
//   flags     bit 0: a level-0 bin received more than 4 frequencies
struct Workspace {
  double2* held[2] = {nullptr, nullptr};
  int64_t held_elems = 0;
  uint8_t* T[2] = {nullptr, nullptr};
  uint8_t* slot_cnt = nullptr;
  int64_t* slot_s = nullptr;
  double2* slot_p = nullptr;
  unsigned long long* ymax2 = nullptr;
  int32_t* flags = nullptr;
  void* zero_base = nullptr;  // ymax2 | flags | slot_cnt, cleared per call
};

struct Tables {
  double2* om_hi = nullptr;  // omega^(i << lo_bits)
  double2* om_lo = nullptr;  // omega^i, i < 2^lo_bits
  int om_lo_bits = 0;
  void* tw = nullptr;        // e^{-2 pi i q / M0}: double2 (FP64) or float4 (FF)
};

}  // namespace sft

namespace sft {
// Events bracketing one launch (profiling only).
struct StageRec {
  const char* name;
  cudaEvent_t t0, t1;
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
  size_t device_bytes = 0;
  // staging for the host entry point (allocated on first use)
  void* x_stage = nullptr;
  size_t x_stage_bytes = 0;
  void* r_stage = nullptr;
  size_t r_stage_bytes = 0;
  // profiling
  bool profiling = false;
  std::vector<sft::StageRec> stage_recs;   // records since the last read
  std::vector<cudaEvent_t> event_pool;     // reused across reads
  size_t events_used = 0;
};

namespace sft {
// Enqueue one sft_exact call (all launches) on `stream`.
cudaError_t launch_exact(sft_plan_s* plan, int64_t n_signals, const void* x, int64_t x_stride,
                         const sft_result* r, cudaStream_t stream);
// One-time per-plan kernel attributes (dynamic shared memory limits).
cudaError_t prepare_kernels(sft_plan_s* plan);
int launches_per_call(const sft_plan_s* plan);
// Sets the calling thread's error detail returned by sft_last_cuda_error.
void set_error_detail(const char* msg);
// Profiling brackets around one launch (no-ops unless plan->profiling).
void stage_begin(sft_plan_s* plan, const char* name, cudaStream_t st);
void stage_end(sft_plan_s* plan, cudaStream_t st);
}  // namespace sft
