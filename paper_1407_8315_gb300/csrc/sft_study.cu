// sft_study.cu -- the collision-count study of Sec. II-C (Lemma 2, Fig. 2):
// for sampled supports S (K distinct locations of [0, N)), the number of
// bins k < M = N/d that hold exactly a members of S (k = s mod M), summed
// over the sampled sets.
//
// One CTA per support set (grid-stride): shared-memory counters for the M
// bins, one atomic increment per location, then a histogram of the counts in
// shared memory, added to the global histogram once per set.
#include <cstdio>

#include "sft_internal.h"

namespace {

constexpr int kStudyThreads = 512;
constexpr int64_t kStudyMaxM = int64_t(1) << 15;  // 128 KB of 32-bit counters

__global__ void __launch_bounds__(kStudyThreads) k_alias_hist(const int64_t* __restrict__ supp,
                                                              int64_t n_sets, int64_t K,
                                                              int64_t M, int n_cells,
                                                              unsigned long long* hist) {
  extern __shared__ unsigned cnt[];
  __shared__ unsigned long long h[33];
  const int tid = threadIdx.x;
  for (int64_t set = blockIdx.x; set < n_sets; set += gridDim.x) {
    for (int64_t i = tid; i < M; i += blockDim.x) cnt[i] = 0u;
    if (tid < n_cells) h[tid] = 0ull;
    __syncthreads();
    const int64_t* s = supp + set * K;
    for (int64_t i = tid; i < K; i += blockDim.x) atomicAdd(&cnt[__ldg(s + i) & (M - 1)], 1u);
    __syncthreads();
    for (int64_t i = tid; i < M; i += blockDim.x) {
      const unsigned c = cnt[i];
      const unsigned cell = c < (unsigned)(n_cells - 1) ? c : (unsigned)(n_cells - 1);
      // one atomic per distinct cell in the warp (most bins share cell 0)
      const unsigned peers = __match_any_sync(__activemask(), cell);
      if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(&h[cell], (unsigned long long)__popc(peers));
    }
    __syncthreads();
    if (tid < n_cells && h[tid] != 0ull) atomicAdd(hist + tid, h[tid]);
    __syncthreads();
  }
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

extern "C" sft_status sft_alias_histogram(const int64_t* supports, int64_t n_sets, int64_t K,
                                          int64_t M, int32_t n_cells, int64_t* hist,
                                          void* stream) {
  if ((!supports && n_sets > 0 && K > 0) || !hist || n_sets < 0 || K < 0 || n_cells < 2 ||
      n_cells > 33) {
    sft::set_error_detail("sft_alias_histogram: NULL pointer or bad sizes");
    return SFT_EINVAL;
  }
  if (!pow2(M) || M > kStudyMaxM) {
    sft::set_error_detail("sft_alias_histogram: M must be a power of two <= 2^15");
    return M > kStudyMaxM ? SFT_EUNSUPPORTED : SFT_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)n_cells * sizeof(int64_t), st);
  if (e == cudaSuccess && n_sets > 0) {
    const size_t smem = (size_t)M * sizeof(unsigned);
    e = cudaFuncSetAttribute(k_alias_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kStudyMaxM * sizeof(unsigned)));
    int dev = 0, nsm = 152;
    if (e == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ctas = n_sets < (int64_t)nsm * 4 ? n_sets : (int64_t)nsm * 4;
    if (e == cudaSuccess) {
      k_alias_hist<<<(unsigned)ctas, kStudyThreads, smem, st>>>(
          supports, n_sets, K, M, n_cells, reinterpret_cast<unsigned long long*>(hist));
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    sft::set_error_detail(cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}
