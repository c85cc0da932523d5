// sft_selfcheck.cu -- the device arithmetic the decoders build on, evaluated
// elementwise on caller data, so that it can be checked against correctly
// rounded references: the reciprocal (an FP32 seed whose operand and result
// move between precisions by bit moves, then two Newton steps), the exact
// float-to-double widening by bit moves, and the complex square root of
// the closed-form roots.
#include "sft_decode.cuh"
#include "sft_internal.h"

namespace sft {

__global__ void k_selfcheck(const double* __restrict__ x, int64_t n, double* __restrict__ out,
                            int which) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (which == 2) {
    // x and out hold n complex values as (re, im) pairs
    if (i < n) {
      const cdbl r = csqrt_fast(cdbl{x[2 * i], x[2 * i + 1]});
      out[2 * i] = r.x;
      out[2 * i + 1] = r.y;
    }
    return;
  }
  if (i >= n) return;
  if (which == 0)
    out[i] = rcp_d(x[i]);
  else
    out[i] = f2d_exact((float)x[i]);
}

cudaError_t launch_selfcheck(const double* x, int64_t n, double* out, int which,
                             cudaStream_t st) {
  const unsigned grid = (unsigned)((n + 255) / 256);
  k_selfcheck<<<grid, 256, 0, st>>>(x, n, out, which);
  return cudaGetLastError();
}

}  // namespace sft
