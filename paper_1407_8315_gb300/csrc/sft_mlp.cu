// sft_mlp.cu -- the learned support proposal of the generally K-sparse path
// (not in the paper): features, forward pass, proposal, training (forward,
// backward, Adam) for sm_103a.
//
// The network n_in -> 128 -> 128 -> n_out (ReLU) is small enough that one
// CTA keeps all its weights in shared memory as FP16 (80 KB) and pushes a
// tile of 32 rows through every layer with FP32 accumulation.  Every
// layer's product -- forward, the backward deltas and the weight gradients
// -- runs on the tensor cores as 16 x 8 output tiles of mma.sync m16n8k8
// with TF32 operands and FP32 accumulators, one tile per warp at a time.
// FP16 weights are exact in TF32; an FP32 operand (activations, deltas) is
// split into a TF32 high part and the TF32 rounding of its remainder, so
// that the two (or, with both operands split, three) products carry about
// 22 significant bits of every operand: the FP32 results of the FP16-weight
// network, not a TF32-rounded one.  Row pitches are chosen for
// bank-conflict-free fragment loads.
//
//   k_mlp_propose<F>   per queued voted bin: features from the held
//                      syndromes (FP64 de-rotation), forward, the min(2a_k,
//                      d) largest support logits -> P->mlp_prop
//   k_mlp_features<F>  the same features, written out (training data)
//   k_mlp_forward      logits of given feature rows
//   k_mlp_train        one minibatch tile: forward, loss, backward; weight
//                      gradients summed over the tile, added atomically
//   k_mlp_adam         Adam update of the FP32 master weights and their
//                      FP16 copy; clears the gradient
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sft_common.cuh"
#include "sft_internal.h"

namespace sft {

constexpr int kH = 128;         // hidden width
constexpr int kMaxIn = 48;      // 2 (2 a_m + r) <= 2 (8 + 16)
constexpr int kMaxOut = 136;    // d + a_m + 2 <= 128 + 6, rounded up
constexpr int kRows = 32;       // rows per tile
constexpr int kThr = 256;       // threads per CTA
// Row pitches of the shared-memory operands, chosen so that the fragment
// loads of the tensor-core tiles (lane l reads row l/4 [+ 8] at column
// l%4 [+ 4] of an FP32 operand, or column l/4 at row l%4 [+ 4] of an FP16
// one) fall into 32 distinct banks, or pairs of lanes share one word:
constexpr int kP1 = 136;        // W1, halves (68 words = 4 mod 32)
constexpr int kP2 = 136;        // W2, halves (68 words)
constexpr int kP3 = 138;        // W3, halves (69 words = 5 mod 32)
constexpr int kXP = 52;         // features, floats (52 = 20 mod 32)
constexpr int kAP = 132;        // hidden activations and their deltas, floats (4 mod 32)
constexpr int kZP = 140;        // logits / output deltas, floats (12 mod 32), >= kMaxOut
constexpr int kMaxSyn = 24;     // 2 a_m + r

struct MlpDims {
  int n_in, n_out, n_sup, n_cls;
};
// offsets of the parameter blocks in the flat FP32 vector
struct MlpOffsets {
  int64_t W1, b1, W2, b2, W3, b3, n;
};
__host__ __device__ inline MlpOffsets mlp_offsets(const MlpDims& D) {
  MlpOffsets o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)D.n_in * kH;
  o.W2 = o.b1 + kH;
  o.b2 = o.W2 + (int64_t)kH * kH;
  o.W3 = o.b2 + kH;
  o.b3 = o.W3 + (int64_t)kH * D.n_out;
  o.n = o.b3 + D.n_out;
  return o;
}

// FP16 weights (W1 | W2 | W3, each row-major as in the flat vector) and the
// FP32 biases inside the master vector
struct MlpW {
  const __half* w16;
  const float* master;
};

struct WSmem {
  __half W1[kMaxIn * kP1];
  __half W2[kH * kP2];
  __half W3[kH * kP3];
  float b1[kH], b2[kH], b3[kMaxOut];
};
struct FwdSmem {
  WSmem w;
  float X[kRows * kXP];
  float A1[kRows * kAP];
  float A2[kRows * kAP];
  float Z[kRows * kZP];
  double2 MT[kRows * kMaxSyn];  // de-rotated syndromes of the tile
  double2 SC[kRows];            // per-row phase / norm factor
};
struct TrainSmem {
  WSmem w;
  float X[kRows * kXP];
  float A1[kRows * kAP];
  float A2[kRows * kAP];  // second hidden layer, later the first layer's delta
  float D3[kRows * kZP];
  float D2[kRows * kAP];
  float rowloss[kRows];
  int cls[kRows];
  uint32_t sup[kRows * 4];
};

// n rounded up to the tensor-core K step (8)
__device__ __forceinline__ int pad8(int n) { return (n + 7) & ~7; }

__device__ void load_weights(WSmem& s, const MlpDims& D, const MlpW& w, int tid) {
  const MlpOffsets o = mlp_offsets(D);
  const __half* w1 = w.w16;
  const __half* w2 = w1 + (int64_t)D.n_in * kH;
  const __half* w3 = w2 + (int64_t)kH * kH;
  for (int i = tid; i < D.n_in * kH; i += kThr) s.W1[(i >> 7) * kP1 + (i & 127)] = w1[i];
  // rows of W1 and columns of W3 up to the next multiple of 8 are read by
  // the tensor-core K steps: zero, so that they add nothing
  for (int i = D.n_in * kH + tid; i < pad8(D.n_in) * kH; i += kThr)
    s.W1[(i >> 7) * kP1 + (i & 127)] = __float2half_rn(0.f);
  for (int i = tid; i < kH * kH; i += kThr) s.W2[(i >> 7) * kP2 + (i & 127)] = w2[i];
  for (int i = tid; i < kH * D.n_out; i += kThr) s.W3[(i / D.n_out) * kP3 + i % D.n_out] = w3[i];
  const int npad = pad8(D.n_out) - D.n_out;
  for (int i = tid; i < kH * npad; i += kThr)
    s.W3[(i / npad) * kP3 + D.n_out + i % npad] = __float2half_rn(0.f);
  for (int i = tid; i < kH; i += kThr) {
    s.b1[i] = w.master[o.b1 + i];
    s.b2[i] = w.master[o.b2 + i];
  }
  for (int i = tid; i < pad8(D.n_out); i += kThr) s.b3[i] = i < D.n_out ? w.master[o.b3 + i] : 0.f;
}

// ---- tensor-core tiles: mma.sync m16n8k8, TF32 operands, FP32 accumulators
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x = hi + lo + O(2^-22 |x|): hi the TF32 rounding of x, lo that of x - hi
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
// d += a b for a 16 x 8 (row-major) A, an 8 x 8 (column-major) B fragment
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp: c += sum_k A(m0 + i, k) B(k, n0 + j) over k < K (a multiple of
// 8) for the 16 x 8 output tile at (m0, n0).  Lane l holds (row l/4 [+ 8],
// columns 2 (l%4) [+ 1]) of c.  A is split (hi, lo) in every case; B too when
// kSplitB (an FP32 operand), else it must be exact in TF32 (FP16 weights).
template <bool kSplitB, class FA, class FB>
__device__ __forceinline__ void mma_tile(float (&c)[4], int m0, int n0, int K, FA A, FB B,
                                         int lane) {
  const int g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 8) {
    uint32_t ah[4], al[4], bh[2], bl[2];
    split_tf32(A(m0 + g, k0 + t), ah[0], al[0]);
    split_tf32(A(m0 + g + 8, k0 + t), ah[1], al[1]);
    split_tf32(A(m0 + g, k0 + t + 4), ah[2], al[2]);
    split_tf32(A(m0 + g + 8, k0 + t + 4), ah[3], al[3]);
    if constexpr (kSplitB) {
      split_tf32(B(k0 + t, n0 + g), bh[0], bl[0]);
      split_tf32(B(k0 + t + 4, n0 + g), bh[1], bl[1]);
    } else {
      bh[0] = to_tf32(B(k0 + t, n0 + g));
      bh[1] = to_tf32(B(k0 + t + 4, n0 + g));
    }
    mma_tf32(c, ah, bh);
    mma_tf32(c, al, bh);
    if constexpr (kSplitB) mma_tf32(c, ah, bl);
  }
}

// out[r][n] = act(sum_k in[r][k] W[k][n] + b[n]) for the kRows rows of a
// tile and n < n_out (K = pad8 of the input width; the padding of `in` and
// of W is zero).  Warp w owns column tiles w, w + 8, w + 16 (n_out <= 136:
// at most 17) for both 16-row halves, so every split A fragment it loads
// serves all of its column tiles.
template <bool kRelu>
__device__ __forceinline__ void dense_tile(const float* in, int in_pitch, int K, const __half* W,
                                           int w_pitch, const float* b, int n_out, float* out,
                                           int out_pitch, int tid) {
  constexpr int kNW = kThr / 32, kNT = (kMaxOut + 8 * kNW - 1) / (8 * kNW);
  static_assert(kRows == 32, "two 16-row halves per tile");
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const int n_tiles = (n_out + 7) >> 3;
  float c[2][kNT][4];
#pragma unroll
  for (int j = 0; j < kNT; ++j) {
    const int c0 = (warp + j * kNW) * 8 + 2 * t;
    const bool on = warp + j * kNW < n_tiles;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      c[h][j][0] = c[h][j][2] = on ? b[c0] : 0.f;
      c[h][j][1] = c[h][j][3] = on ? b[c0 + 1] : 0.f;
    }
  }
  for (int k0 = 0; k0 < K; k0 += 8) {
    uint32_t ah[2][4], al[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float* r0 = in + (h * 16 + g) * in_pitch + k0 + t;
      split_tf32(r0[0], ah[h][0], al[h][0]);
      split_tf32(r0[8 * in_pitch], ah[h][1], al[h][1]);
      split_tf32(r0[4], ah[h][2], al[h][2]);
      split_tf32(r0[8 * in_pitch + 4], ah[h][3], al[h][3]);
    }
#pragma unroll
    for (int j = 0; j < kNT; ++j) {
      const int nt = warp + j * kNW;
      if (nt < n_tiles) {
        const __half* wp = W + (k0 + t) * w_pitch + nt * 8 + g;
        const uint32_t bf[2] = {to_tf32(__half2float(wp[0])),
                                to_tf32(__half2float(wp[4 * w_pitch]))};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          mma_tf32(c[h][j], ah[h], bf);
          mma_tf32(c[h][j], al[h], bf);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kNT; ++j) {
    const int nt = warp + j * kNW;
    if (nt < n_tiles) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = h * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          if (n < n_out) out[r * out_pitch + n] = kRelu ? fmaxf(c[h][j][q], 0.0f) : c[h][j][q];
        }
    }
  }
}

// z1 = X W1 + b1, A1 = relu(z1); A2 = relu(A1 W2 + b2); Z = A2 W3 + b3,
// for the 32 rows of the tile (tensor cores, FP32 accumulation)
__device__ void forward_tile(const WSmem& w, const MlpDims& D, const float* X, float* A1,
                             float* A2, float* Z, int tid) {
  dense_tile<true>(X, kXP, pad8(D.n_in), w.W1, kP1, w.b1, kH, A1, kAP, tid);
  __syncthreads();
  dense_tile<true>(A1, kAP, kH, w.W2, kP2, w.b2, kH, A2, kAP, tid);
  __syncthreads();
  dense_tile<false>(A2, kAP, kH, w.W3, kP3, w.b3, D.n_out, Z, kZP, tid);
  __syncthreads();
}

// ----------------------------------------------------------------- features
struct FeatArgs {
  int64_t N, M, d;
  int a_max, r;
  const void* Y;  // held syndromes: rows 0..2a_m-1 consecutive, then random
  int64_t held_elems;
  const uint8_t* ak;
  const int2* queue;
  const int* qcount;     // entries filed from the front of the queue
  const int* qcount_hi;  // entries filed from the back (entry i at qcap - 1 - i)
  int64_t qcap;
  const int64_t* cs;
  OmegaTab om;
};

// queue position of the i-th voted bin (front entries first, then back)
__device__ __forceinline__ int queue_pos(const FeatArgs& g, int i) {
  const int n1 = *g.qcount;
  return i < n1 ? i : (int)(g.qcap - 1 - (i - n1));
}

// Features of queue entries e0 .. e0+nt-1 into X (rows beyond nt zero):
// m~_l = Y_l[k] omega^{-k sh_l} in FP64, rotated by conj(m~_0)/|m~_0| and
// scaled by 1/||m~||, interleaved (re, im) as floats.
template <class F>
__device__ void tile_features(const FeatArgs& g, int e0, int nt, FwdSmem& s, int tid) {
  typedef typename Store<F>::T T;
  const int nsyn = 2 * g.a_max + g.r;
  for (int it = tid; it < kRows * nsyn; it += kThr) {
    const int rr = it / nsyn, l = it - rr * nsyn;
    cdbl v = mk(0.0, 0.0);
    if (rr < nt) {
      const int2 q = g.queue[queue_pos(g, e0 + rr)];
      const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)q.x * g.held_elems;
      const cdbl y = Store<F>::to_d(Y[(int64_t)l * g.M + q.y]);
      const int64_t sh = l < 2 * g.a_max ? (int64_t)l : g.cs[l - 2 * g.a_max];
      v = y * conjd(omega_pow(g.om, (int64_t)q.y * sh));
    }
    s.MT[rr * kMaxSyn + l] = make_double2(v.x, v.y);
  }
  __syncthreads();
  if (tid < kRows) {
    const double2 m0 = s.MT[tid * kMaxSyn];
    const double a0 = sqrt(m0.x * m0.x + m0.y * m0.y);
    cdbl ph = a0 > 0.0 ? mk(m0.x / a0, -m0.y / a0) : mk(1.0, 0.0);
    double s2 = 0.0;
    for (int l = 0; l < nsyn; ++l) {
      const double2 v = s.MT[tid * kMaxSyn + l];
      s2 += v.x * v.x + v.y * v.y;
    }
    const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    s.SC[tid] = make_double2(ph.x * inv, ph.y * inv);
  }
  __syncthreads();
  for (int it = tid; it < kRows * kMaxIn; it += kThr) {
    const int rr = it / kMaxIn, c = it - rr * kMaxIn, l = c >> 1;
    float f = 0.0f;
    if (l < nsyn) {
      const double2 m = s.MT[rr * kMaxSyn + l], sc = s.SC[rr];
      f = (c & 1) ? (float)(m.x * sc.y + m.y * sc.x) : (float)(m.x * sc.x - m.y * sc.y);
    }
    s.X[rr * kXP + c] = f;
  }
  __syncthreads();
}

template <class F>
__global__ void __launch_bounds__(kThr) k_mlp_propose(FeatArgs g, MlpDims D, MlpW w,
                                                      int16_t* __restrict__ prop) {
  extern __shared__ __align__(16) char smem_raw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int tid = threadIdx.x;
  load_weights(s.w, D, w, tid);
  __syncthreads();
  const int n = *g.qcount + *g.qcount_hi;
  for (int e0 = blockIdx.x * kRows; e0 < n; e0 += gridDim.x * kRows) {
    const int nt = min(kRows, n - e0);
    tile_features<F>(g, e0, nt, s, tid);
    forward_tile(s.w, D, s.X, s.A1, s.A2, s.Z, tid);
    if (tid < nt) {
      const int pos = queue_pos(g, e0 + tid);
      const int2 q = g.queue[pos];
      const int a = g.ak[(int64_t)q.x * g.M + q.y];
      const int nk = (int)min((int64_t)min(2 * a, 8), g.d);
      float bv[8];
      int bt[8];
      int have = 0;
      const float* z = s.Z + tid * kZP;
      for (int t = 0; t < D.n_sup; ++t) {
        const float v = z[t];
        if (have < nk || v > bv[nk - 1]) {  // equal values keep the lower t
          int pos = have < nk ? have : nk - 1;
          while (pos > 0 && bv[pos - 1] < v) {
            bv[pos] = bv[pos - 1];
            bt[pos] = bt[pos - 1];
            --pos;
          }
          bv[pos] = v;
          bt[pos] = t;
          if (have < nk) ++have;
        }
      }
      for (int i = 1; i < have; ++i)
        for (int j = i; j > 0 && bt[j - 1] > bt[j]; --j) {
          const int tt = bt[j];
          bt[j] = bt[j - 1];
          bt[j - 1] = tt;
        }
      int16_t* o = prop + (int64_t)pos * 8;
      for (int u = 0; u < 8; ++u) o[u] = u < have ? (int16_t)bt[u] : (int16_t)-1;
    }
    __syncthreads();
  }
}

template <class F>
__global__ void __launch_bounds__(kThr) k_mlp_features(FeatArgs g, int n_in, int64_t cap,
                                                       float* __restrict__ feat,
                                                       int32_t* __restrict__ rows) {
  extern __shared__ __align__(16) char smem_raw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int n = (int)min((int64_t)*g.qcount + *g.qcount_hi, cap);
  for (int e0 = blockIdx.x * kRows; e0 < n; e0 += gridDim.x * kRows) {
    const int nt = min(kRows, n - e0);
    tile_features<F>(g, e0, nt, s, tid);
    for (int it = tid; it < nt * n_in; it += kThr) {
      const int rr = it / n_in, c = it - rr * n_in;
      feat[(int64_t)(e0 + rr) * n_in + c] = s.X[rr * kXP + c];
    }
    if (tid < nt) {
      const int2 q = g.queue[queue_pos(g, e0 + tid)];
      int32_t* o = rows + (int64_t)(e0 + tid) * 3;
      o[0] = q.x;
      o[1] = q.y;
      o[2] = g.ak[(int64_t)q.x * g.M + q.y];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThr) k_mlp_forward(MlpDims D, MlpW w, const float* __restrict__ feat,
                                                      int64_t n_rows, float* __restrict__ logits) {
  extern __shared__ __align__(16) char smem_raw[];
  FwdSmem& s = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int tid = threadIdx.x;
  load_weights(s.w, D, w, tid);
  __syncthreads();
  for (int64_t e0 = (int64_t)blockIdx.x * kRows; e0 < n_rows; e0 += (int64_t)gridDim.x * kRows) {
    const int nt = (int)min((int64_t)kRows, n_rows - e0);
    for (int it = tid; it < kRows * kMaxIn; it += kThr) {
      const int rr = it / kMaxIn, c = it - rr * kMaxIn;
      s.X[rr * kXP + c] = (rr < nt && c < D.n_in) ? feat[(e0 + rr) * D.n_in + c] : 0.0f;
    }
    __syncthreads();
    forward_tile(s.w, D, s.X, s.A1, s.A2, s.Z, tid);
    for (int it = tid; it < nt * D.n_out; it += kThr) {
      const int rr = it / D.n_out, c = it - rr * D.n_out;
      logits[(e0 + rr) * D.n_out + c] = s.Z[rr * kZP + c];
    }
    __syncthreads();
  }
}

// One tile of a minibatch: rows perm[b0 + blockIdx.x*32 + rr] (or
// b0 + ... without a permutation).  Loss per row = count cross-entropy +
// mean support binary cross-entropy; the deltas carry the 1/bs of the
// minibatch mean.  Gradients of the tile are summed in registers and added
// to `grad` atomically; loss_sum receives sum(rowloss) / bs.
__global__ void __launch_bounds__(kThr) k_mlp_train(MlpDims D, MlpW w, const float* __restrict__ feat,
                                                    const int32_t* __restrict__ cls,
                                                    const uint32_t* __restrict__ sup,
                                                    const uint32_t* __restrict__ perm, int64_t b0,
                                                    int bs, float* __restrict__ grad,
                                                    float* __restrict__ loss_sum) {
  extern __shared__ __align__(16) char smem_raw[];
  TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const MlpOffsets o = mlp_offsets(D);
  const int r0 = blockIdx.x * kRows;
  const int nt = min(kRows, bs - r0);
  const float inv_bs = 1.0f / (float)bs;
  load_weights(s.w, D, w, tid);
  for (int it = tid; it < kRows * kMaxIn; it += kThr) {
    const int rr = it / kMaxIn, c = it - rr * kMaxIn;
    float v = 0.0f;
    if (rr < nt && c < D.n_in) {
      const int64_t row = perm ? (int64_t)perm[b0 + r0 + rr] : b0 + r0 + rr;
      v = feat[row * D.n_in + c];
    }
    s.X[rr * kXP + c] = v;
  }
  if (tid < kRows) {
    int c = 0;
    uint32_t sw[4] = {0u, 0u, 0u, 0u};
    if (tid < nt) {
      const int64_t row = perm ? (int64_t)perm[b0 + r0 + tid] : b0 + r0 + tid;
      c = cls[row];
      for (int q = 0; q < 4; ++q) sw[q] = sup[row * 4 + q];
    }
    s.cls[tid] = c;
    for (int q = 0; q < 4; ++q) s.sup[tid * 4 + q] = sw[q];
  }
  __syncthreads();
  forward_tile(s.w, D, s.X, s.A1, s.A2, s.D3, tid);  // logits into D3
  // ---- output deltas and loss (one thread per row; Z row pitch is odd)
  if (tid < kRows) {
    float* z = s.D3 + tid * kZP;
    float rl = 0.0f;
    if (tid < nt) {
      const float scale_s = inv_bs / (float)D.n_sup;
      float bce = 0.0f;
      for (int t = 0; t < D.n_sup; ++t) {
        const float zt = z[t];
        const float y = (float)((s.sup[tid * 4 + (t >> 5)] >> (t & 31)) & 1u);
        // softplus(z) - y z, and d/dz = sigmoid(z) - y
        bce += fmaxf(zt, 0.0f) + log1pf(expf(-fabsf(zt))) - y * zt;
        z[t] = (1.0f / (1.0f + expf(-zt)) - y) * scale_s;
      }
      float zmax = -INFINITY;
      for (int j = 0; j < D.n_cls; ++j) zmax = fmaxf(zmax, z[D.n_sup + j]);
      float se = 0.0f;
      for (int j = 0; j < D.n_cls; ++j) se += expf(z[D.n_sup + j] - zmax);
      const float lse = zmax + logf(se);
      const int c = s.cls[tid];
      const float ce = lse - z[D.n_sup + c];
      for (int j = 0; j < D.n_cls; ++j) {
        const float p = expf(z[D.n_sup + j] - lse);
        z[D.n_sup + j] = (p - (j == c ? 1.0f : 0.0f)) * inv_bs;
      }
      rl = ce + bce / (float)D.n_sup;
    } else {
      for (int c = 0; c < D.n_out; ++c) z[c] = 0.0f;
    }
    s.rowloss[tid] = rl;
  }
  __syncthreads();
  if (tid < 32) {
    float v = s.rowloss[tid];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (tid == 0) atomicAdd(loss_sum, v * inv_bs);
  }
  // zero the delta columns between n_out and the next multiple of 8 (the
  // K padding of the product with W3)
  for (int it = tid; it < kRows * (pad8(D.n_out) - D.n_out); it += kThr) {
    const int np = pad8(D.n_out) - D.n_out;
    s.D3[(it / np) * kZP + D.n_out + it % np] = 0.0f;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  // gW[m][n] += sum_r P(r, m) Q(r, n) over the tile's rows, 16 x 8 tiles of
  // the m_n x n_n gradient block on the warps, added to grad[m * n_n + n]
  auto weight_grad = [&](int m_n, int n_n, float* gdst, auto P, auto Q) {
    const int mt = (m_n + 15) >> 4, nt = (n_n + 7) >> 3;
    for (int tile = warp; tile < mt * nt; tile += kThr / 32) {
      const int m0 = (tile % mt) * 16, n0 = (tile / mt) * 8;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tile<true>(c, m0, n0, kRows, [&](int m, int r) { return P(r, m); }, Q, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + g + (q >> 1) * 8, n = n0 + 2 * t4 + (q & 1);
        if (m < m_n && n < n_n) atomicAdd(gdst + (int64_t)m * n_n + n, c[q]);
      }
    }
  };
  // delta[r][n] = (sum_k Din[r][k] W[n][k]) * (act[r][n] > 0), n < 128:
  // the product with the transposed FP16 weights
  auto back_delta = [&](const float* Din, int din_pitch, int K, const __half* W, int w_pitch,
                        const float* act, float* dout) {
    for (int tile = warp; tile < (kH / 8) * (kRows / 16); tile += kThr / 32) {
      const int m0 = (tile & 1) * 16, n0 = (tile >> 1) * 8;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tile<false>(
          c, m0, n0, K, [&](int r, int k) { return Din[r * din_pitch + k]; },
          [&](int k, int n) { return __half2float(W[n * w_pitch + k]); }, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + g + (q >> 1) * 8, n = n0 + 2 * t4 + (q & 1);
        dout[r * kAP + n] = act[r * kAP + n] > 0.0f ? c[q] : 0.0f;
      }
    }
  };
  // ---- W3, b3: A2^T D3
  weight_grad(kH, D.n_out, grad + o.W3, [&](int r, int h) { return s.A2[r * kAP + h]; },
              [&](int r, int c) { return s.D3[r * kZP + c]; });
  for (int c = tid; c < D.n_out; c += kThr) {
    float acc = 0.0f;
    for (int rr = 0; rr < kRows; ++rr) acc += s.D3[rr * kZP + c];
    atomicAdd(grad + o.b3 + c, acc);
  }
  // ---- delta of the second hidden layer: (D3 W3^T) * (z2 > 0)
  back_delta(s.D3, kZP, pad8(D.n_out), s.w.W3, kP3, s.A2, s.D2);
  __syncthreads();
  // ---- W2, b2: A1^T D2
  weight_grad(kH, kH, grad + o.W2, [&](int r, int i) { return s.A1[r * kAP + i]; },
              [&](int r, int h) { return s.D2[r * kAP + h]; });
  if (tid < kH) {
    float acc = 0.0f;
    for (int rr = 0; rr < kRows; ++rr) acc += s.D2[rr * kAP + tid];
    atomicAdd(grad + o.b2 + tid, acc);
  }
  // ---- delta of the first hidden layer (into A2's space): (D2 W2^T) * (z1 > 0)
  back_delta(s.D2, kAP, kH, s.w.W2, kP2, s.A1, s.A2);
  __syncthreads();
  // ---- W1, b1: X^T D1
  weight_grad(D.n_in, kH, grad + o.W1, [&](int r, int i) { return s.X[r * kXP + i]; },
              [&](int r, int h) { return s.A2[r * kAP + h]; });
  if (tid < kH) {
    float acc = 0.0f;
    for (int rr = 0; rr < kRows; ++rr) acc += s.A2[rr * kAP + tid];
    atomicAdd(grad + o.b1 + tid, acc);
  }
}

// Adam on the FP32 master weights (bias-corrected moments), the FP16 copy
// of W1..W3 refreshed, the gradient cleared.
__global__ void k_mlp_adam(MlpDims D, float* __restrict__ master, float* __restrict__ m,
                           float* __restrict__ v, float* __restrict__ grad, __half* __restrict__ w16,
                           float lr, float b1, float b2, float eps, float c1, float c2) {
  const MlpOffsets o = mlp_offsets(D);
  const int64_t nW1 = (int64_t)D.n_in * kH, nW2 = (int64_t)kH * kH;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < o.n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float g = grad[p];
    const float mp = b1 * m[p] + (1.0f - b1) * g;
    const float vp = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mp;
    v[p] = vp;
    const float wv = master[p] - lr * (mp * c1) / (sqrtf(vp * c2) + eps);
    master[p] = wv;
    grad[p] = 0.0f;
    if (p < o.b1)
      w16[p] = __float2half_rn(wv);
    else if (p >= o.W2 && p < o.b2)
      w16[nW1 + (p - o.W2)] = __float2half_rn(wv);
    else if (p >= o.W3 && p < o.b3)
      w16[nW1 + nW2 + (p - o.W3)] = __float2half_rn(wv);
  }
}

// FP16 copy of W1..W3 from the master vector
__global__ void k_mlp_to_half(MlpDims D, const float* __restrict__ master, __half* __restrict__ w16) {
  const MlpOffsets o = mlp_offsets(D);
  const int64_t nW1 = (int64_t)D.n_in * kH, nW2 = (int64_t)kH * kH, nW3 = (int64_t)kH * D.n_out;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nW1 + nW2 + nW3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i < nW1 ? i : i < nW1 + nW2 ? o.W2 + (i - nW1) : o.W3 + (i - nW1 - nW2);
    w16[i] = __float2half_rn(master[p]);
  }
}

}  // namespace sft

// ------------------------------------------------------------------ host side
struct sft_mlp_s {
  sft_mlp_config cfg;
  sft::MlpDims D;
  int64_t n_params = 0;
  void* base = nullptr;  // master | m | v | grad | loss | w16
  float* master = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  float* loss = nullptr;
  __half* w16 = nullptr;
  uint32_t* perm = nullptr;
  int64_t perm_cap = 0;
  int64_t step = 0;
};

namespace {

using sft::kH;
using sft::kRows;
using sft::kThr;

// SplitMix64 (Steele, Lea, Flood 2014), output i of the stream of `seed`
uint64_t mix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

sft_status fail(sft_status st, const char* msg) {
  sft::set_error_detail(msg);
  return st;
}

sft_status cuda_fail(cudaError_t e) {
  sft::set_error_detail(cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
}

cudaError_t set_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(sft::k_mlp_propose<sft::F64>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(sft::FwdSmem));
  if (!e) e = cudaFuncSetAttribute(sft::k_mlp_propose<sft::FF>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(sft::FwdSmem));
  if (!e) e = cudaFuncSetAttribute(sft::k_mlp_features<sft::F64>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(sft::FwdSmem));
  if (!e) e = cudaFuncSetAttribute(sft::k_mlp_features<sft::FF>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(sft::FwdSmem));
  if (!e) e = cudaFuncSetAttribute(sft::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(sft::FwdSmem));
  if (!e) e = cudaFuncSetAttribute(sft::k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(sft::TrainSmem));
  return e;
}

int num_sms() {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

sft::MlpW weights_of(const sft_mlp_s* m) { return sft::MlpW{m->w16, m->master}; }

void refresh_half(sft_mlp_s* m, cudaStream_t st) {
  sft::k_mlp_to_half<<<64, 256, 0, st>>>(m->D, m->master, m->w16);
}

sft::FeatArgs feat_args(const sft_plan_s* P, int64_t B) {
  const sft::Workspace& W = P->ws;
  return sft::FeatArgs{P->p.N,        P->M0,     P->p.d,      P->p.a_max,
                       P->p.n_cs_shifts, W.held[0], W.held_elems, W.T[0],
                       W.queue[0],    W.qcount,  W.qcount + 2, B * P->M0, P->tab.cs_shifts,
                       sft::OmegaTab{P->tab.om_hi, P->tab.om_lo, P->tab.om_lo_bits, P->p.N - 1}};
}

}  // namespace

namespace sft {

void mlp_propose(sft_plan_s* P, int64_t B, int nsm, cudaStream_t st) {
  const sft_mlp_s* m = P->mlp;
  const int64_t maxq = B * P->M0;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((maxq + kRows - 1) / kRows, nsm));
  stage_begin(P, "mlp_propose", st);
  if (P->p.precision == SFT_FP64)
    k_mlp_propose<F64><<<grid, kThr, sizeof(FwdSmem), st>>>(feat_args(P, B), m->D, weights_of(m),
                                                             P->mlp_prop);
  else
    k_mlp_propose<FF><<<grid, kThr, sizeof(FwdSmem), st>>>(feat_args(P, B), m->D, weights_of(m),
                                                            P->mlp_prop);
  stage_end(P, st);
}

void mlp_features(sft_plan_s* P, int64_t B, int nsm, float* feat, int32_t* rows, int64_t cap_rows,
                  cudaStream_t st) {
  const int n_in = 2 * (2 * P->p.a_max + P->p.n_cs_shifts);
  const int64_t maxq = std::min<int64_t>(B * P->M0, cap_rows);
  if (maxq <= 0) return;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((maxq + kRows - 1) / kRows, nsm));
  if (P->p.precision == SFT_FP64)
    k_mlp_features<F64><<<grid, kThr, sizeof(FwdSmem), st>>>(feat_args(P, B), n_in, cap_rows, feat, rows);
  else
    k_mlp_features<FF><<<grid, kThr, sizeof(FwdSmem), st>>>(feat_args(P, B), n_in, cap_rows, feat, rows);
}

}  // namespace sft

extern "C" {

sft_status sft_mlp_config_for(const sft_params* p_in, sft_mlp_config* out) {
  if (!p_in || !out) return fail(SFT_EINVAL, "sft_mlp_config_for: NULL argument");
  sft_params p = *p_in;
  sft::normalize_params(&p);
  if (p.mode != SFT_GENERAL) return fail(SFT_EINVAL, "sft_mlp_config_for: mode is not SFT_GENERAL");
  const int n_in = 2 * (2 * p.a_max + p.n_cs_shifts);
  if (n_in > sft::kMaxIn)
    return fail(SFT_EUNSUPPORTED, "sft_mlp_config_for: 2 (2 a_max + n_cs_shifts) above 48");
  if (p.d > 128) return fail(SFT_EUNSUPPORTED, "sft_mlp_config_for: d above 128");
  sft_mlp_config c;
  std::memset(&c, 0, sizeof(c));
  c.n_in = n_in;
  c.n_hidden = kH;
  c.n_sup = (int32_t)p.d;
  c.n_cls = p.a_max + 2;
  c.seed = 0;
  c.lr = 2e-3f;
  c.beta1 = 0.9f;
  c.beta2 = 0.999f;
  c.eps = 1e-8f;
  *out = c;
  return SFT_OK;
}

sft_status sft_mlp_create(const sft_mlp_config* c, sft_mlp_t* out) {
  if (!c || !out) return fail(SFT_EINVAL, "sft_mlp_create: NULL argument");
  *out = nullptr;
  if (c->n_hidden != kH) return fail(SFT_EUNSUPPORTED, "sft_mlp_create: n_hidden must be 128");
  if (c->n_in < 2 || c->n_in > sft::kMaxIn || c->n_sup < 1 || c->n_sup > 128 || c->n_cls < 2 ||
      c->n_cls > 8 || c->n_sup + c->n_cls > sft::kMaxOut)
    return fail(SFT_EINVAL, "sft_mlp_create: n_in in [2, 48], n_sup in [1, 128], n_cls in [2, 8]");
  if (!(c->lr > 0.0f) || !(c->beta1 >= 0.0f && c->beta1 < 1.0f) ||
      !(c->beta2 >= 0.0f && c->beta2 < 1.0f) || !(c->eps > 0.0f))
    return fail(SFT_EINVAL, "sft_mlp_create: bad Adam settings");
  sft_mlp_s* m = new (std::nothrow) sft_mlp_s();
  if (!m) return SFT_ENOMEM;
  m->cfg = *c;
  m->D = sft::MlpDims{c->n_in, c->n_sup + c->n_cls, c->n_sup, c->n_cls};
  const sft::MlpOffsets o = sft::mlp_offsets(m->D);
  m->n_params = o.n;
  const int64_t n_half = (int64_t)c->n_in * kH + (int64_t)kH * kH + (int64_t)kH * m->D.n_out;
  const size_t fbytes = ((size_t)o.n * 4 * sizeof(float) + 256 + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&m->base, fbytes + (size_t)n_half * sizeof(__half));
  if (e) {
    delete m;
    return cuda_fail(e);
  }
  float* f = static_cast<float*>(m->base);
  m->master = f;
  m->m = f + o.n;
  m->v = f + 2 * o.n;
  m->grad = f + 3 * o.n;
  m->loss = f + 4 * o.n;
  m->w16 = reinterpret_cast<__half*>(static_cast<char*>(m->base) + fbytes);
  // He-uniform weights from SplitMix64(seed), zero biases
  std::vector<float> h((size_t)o.n, 0.0f);
  auto fill = [&](int64_t off, int64_t count, int fan_in) {
    const double lim = std::sqrt(6.0 / fan_in);
    for (int64_t i = 0; i < count; ++i) {
      const double u = (double)(mix64(c->seed, (uint64_t)(off + i)) >> 11) * 0x1.0p-53;
      h[(size_t)(off + i)] = (float)((2.0 * u - 1.0) * lim);
    }
  };
  fill(o.W1, (int64_t)c->n_in * kH, c->n_in);
  fill(o.W2, (int64_t)kH * kH, kH);
  fill(o.W3, (int64_t)kH * m->D.n_out, kH);
  e = set_smem_limits();
  if (!e) e = cudaMemcpy(m->master, h.data(), (size_t)o.n * sizeof(float), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(m->m, 0, (size_t)(3 * o.n + 1) * sizeof(float));
  if (!e) {
    refresh_half(m, 0);
    e = cudaDeviceSynchronize();
  }
  if (e) {
    cudaFree(m->base);
    delete m;
    return cuda_fail(e);
  }
  *out = m;
  return SFT_OK;
}

void sft_mlp_destroy(sft_mlp_t m) {
  if (!m) return;
  cudaDeviceSynchronize();
  if (m->perm) cudaFree(m->perm);
  if (m->base) cudaFree(m->base);
  delete m;
}

int64_t sft_mlp_param_count(sft_mlp_t m) { return m ? m->n_params : -1; }

sft_status sft_mlp_get_params(sft_mlp_t m, float* host_out) {
  if (!m || !host_out) return fail(SFT_EINVAL, "sft_mlp_get_params: NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (!e) e = cudaMemcpy(host_out, m->master, (size_t)m->n_params * sizeof(float), cudaMemcpyDeviceToHost);
  return e ? cuda_fail(e) : SFT_OK;
}

sft_status sft_mlp_set_params(sft_mlp_t m, const float* host_in) {
  if (!m || !host_in) return fail(SFT_EINVAL, "sft_mlp_set_params: NULL argument");
  cudaError_t e = cudaDeviceSynchronize();
  if (!e) e = cudaMemcpy(m->master, host_in, (size_t)m->n_params * sizeof(float), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemset(m->m, 0, (size_t)(3 * m->n_params + 1) * sizeof(float));
  if (!e) {
    refresh_half(m, 0);
    e = cudaDeviceSynchronize();
  }
  m->step = 0;
  return e ? cuda_fail(e) : SFT_OK;
}

sft_status sft_mlp_forward(sft_mlp_t m, const float* feat, int64_t n_rows, float* logits,
                           void* stream) {
  if (!m || (n_rows > 0 && (!feat || !logits)) || n_rows < 0)
    return fail(SFT_EINVAL, "sft_mlp_forward: NULL argument or n_rows < 0");
  if (n_rows == 0) return SFT_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)std::min<int64_t>((n_rows + kRows - 1) / kRows, num_sms());
  sft::k_mlp_forward<<<grid, kThr, sizeof(sft::FwdSmem), st>>>(m->D, weights_of(m), feat, n_rows,
                                                               logits);
  cudaError_t e = cudaGetLastError();
  return e ? cuda_fail(e) : SFT_OK;
}

static sft_status check_labels(sft_mlp_t m, const float* feat, const int32_t* cls,
                               const uint32_t* sup, int64_t n_rows, const char* who) {
  char msg[160];
  if (!m || !feat || !cls || !sup || n_rows < 1 || n_rows > (int64_t(1) << 30)) {
    std::snprintf(msg, sizeof(msg), "%s: NULL argument or n_rows outside [1, 2^30]", who);
    return fail(SFT_EINVAL, msg);
  }
  return SFT_OK;
}

sft_status sft_mlp_grad(sft_mlp_t m, const float* feat, const int32_t* cls, const uint32_t* sup,
                        int64_t n_rows, float* grad, float* loss, void* stream) {
  sft_status s = check_labels(m, feat, cls, sup, n_rows, "sft_mlp_grad");
  if (s != SFT_OK) return s;
  if (!grad || !loss) return fail(SFT_EINVAL, "sft_mlp_grad: NULL output");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(m->grad, 0, (size_t)(m->n_params + 1) * sizeof(float), st);
  if (!e) {
    sft::k_mlp_train<<<(unsigned)((n_rows + kRows - 1) / kRows), kThr, sizeof(sft::TrainSmem), st>>>(
        m->D, weights_of(m), feat, cls, sup, nullptr, 0, (int)n_rows, m->grad, m->loss);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(grad, m->grad, (size_t)m->n_params * sizeof(float),
                              cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (!e) e = cudaMemsetAsync(m->grad, 0, (size_t)(m->n_params + 1) * sizeof(float), st);
  return e ? cuda_fail(e) : SFT_OK;
}

sft_status sft_mlp_train(sft_mlp_t m, const float* feat, const int32_t* cls, const uint32_t* sup,
                         int64_t n_rows, int32_t epochs, int32_t batch, uint64_t shuffle_seed,
                         float* loss_out, void* stream) {
  sft_status s = check_labels(m, feat, cls, sup, n_rows, "sft_mlp_train");
  if (s != SFT_OK) return s;
  if (epochs < 1 || batch < 1 || batch > (1 << 20))
    return fail(SFT_EINVAL, "sft_mlp_train: epochs >= 1, batch in [1, 2^20]");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (m->perm_cap < n_rows) {
    if (m->perm) cudaFree(m->perm);
    m->perm = nullptr;
    m->perm_cap = 0;
    e = cudaMalloc(&m->perm, (size_t)n_rows * sizeof(uint32_t));
    if (e) return cuda_fail(e);
    m->perm_cap = n_rows;
  }
  std::vector<uint32_t> perm((size_t)n_rows);
  const int nsm = num_sms();
  const unsigned agrid = (unsigned)std::min<int64_t>((m->n_params + 255) / 256, 4 * nsm);
  e = cudaMemsetAsync(m->grad, 0, (size_t)(m->n_params + 1) * sizeof(float), st);
  for (int ep = 0; ep < epochs && !e; ++ep) {
    // Fisher-Yates shuffle driven by the SplitMix64 stream of this epoch
    const uint64_t es = mix64(shuffle_seed, (uint64_t)ep);
    for (int64_t i = 0; i < n_rows; ++i) perm[(size_t)i] = (uint32_t)i;
    for (int64_t i = 0; i + 1 < n_rows; ++i) {
      const int64_t j = i + (int64_t)(mix64(es, (uint64_t)i) % (uint64_t)(n_rows - i));
      std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    e = cudaMemcpyAsync(m->perm, perm.data(), (size_t)n_rows * sizeof(uint32_t),
                        cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemsetAsync(m->loss, 0, sizeof(float), st);
    int nb = 0;
    for (int64_t b0 = 0; b0 < n_rows && !e; b0 += batch, ++nb) {
      const int bs = (int)std::min<int64_t>(batch, n_rows - b0);
      sft::k_mlp_train<<<(unsigned)((bs + kRows - 1) / kRows), kThr, sizeof(sft::TrainSmem), st>>>(
          m->D, weights_of(m), feat, cls, sup, m->perm, b0, bs, m->grad, m->loss);
      ++m->step;
      const double c1 = 1.0 / (1.0 - std::pow((double)m->cfg.beta1, (double)m->step));
      const double c2 = 1.0 / (1.0 - std::pow((double)m->cfg.beta2, (double)m->step));
      sft::k_mlp_adam<<<agrid, 256, 0, st>>>(m->D, m->master, m->m, m->v, m->grad, m->w16,
                                             m->cfg.lr, m->cfg.beta1, m->cfg.beta2, m->cfg.eps,
                                             (float)c1, (float)c2);
      e = cudaGetLastError();
    }
    float l = 0.0f;
    if (!e) e = cudaMemcpyAsync(&l, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (!e && loss_out) loss_out[ep] = nb > 0 ? l / (float)nb : 0.0f;
  }
  if (!e) e = cudaStreamSynchronize(st);
  return e ? cuda_fail(e) : SFT_OK;
}

sft_status sft_plan_attach_mlp(sft_plan_t P, sft_mlp_t m) {
  if (!P) return fail(SFT_EINVAL, "sft_plan_attach_mlp: NULL plan");
  if (!m) {
    P->mlp = nullptr;
    return SFT_OK;
  }
  if (P->p.mode != SFT_GENERAL) return fail(SFT_EINVAL, "sft_plan_attach_mlp: plan is not SFT_GENERAL");
  if (m->D.n_in != 2 * (2 * P->p.a_max + P->p.n_cs_shifts) || m->D.n_sup != (int)P->p.d ||
      m->D.n_cls != P->p.a_max + 2)
    return fail(SFT_EINVAL, "sft_plan_attach_mlp: network dimensions do not match the plan");
  if (!P->mlp_prop) {
    cudaError_t e = cudaMalloc(&P->mlp_prop, (size_t)(P->max_signals * P->M0) * 8 * sizeof(int16_t));
    if (e) {
      P->mlp_prop = nullptr;
      return cuda_fail(e);
    }
  }
  P->mlp = m;
  return SFT_OK;
}

sft_status sft_mlp_features(sft_plan_t P, int64_t n, const void* x, int64_t x_stride, float* feat,
                            int32_t* rows, int64_t cap_rows, int64_t* n_rows, void* stream) {
  if (!P || !x || !n_rows || cap_rows < 0 || (cap_rows > 0 && (!feat || !rows)))
    return fail(SFT_EINVAL, "sft_mlp_features: NULL argument or cap_rows < 0");
  if (P->p.mode != SFT_GENERAL) return fail(SFT_EINVAL, "sft_mlp_features: plan is not SFT_GENERAL");
  if (n < 1 || n > P->max_signals) return fail(SFT_EINVAL, "sft_mlp_features: n_signals outside [1, max_signals]");
  if (x_stride < P->p.N) return fail(SFT_EINVAL, "sft_mlp_features: x_stride < N");
  if (2 * (2 * P->p.a_max + P->p.n_cs_shifts) > sft::kMaxIn)
    return fail(SFT_EUNSUPPORTED, "sft_mlp_features: more than 24 syndromes per bin");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = set_smem_limits();
  if (!e) e = cudaMemsetAsync(P->ws.zero_base, 0, P->ws.zero_bytes, st);
  if (!e) {
    sft::launch_general_features(P, n, x, x_stride, num_sms(), feat, rows, cap_rows, st);
    e = cudaGetLastError();
  }
  int q[3] = {0, 0, 0};  // voted bins: front (one alias), -, back (several)
  if (!e) e = cudaMemcpyAsync(q, P->ws.qcount, sizeof(q), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_fail(e);
  *n_rows = (int64_t)q[0] + q[2];
  return SFT_OK;
}

}  // extern "C"
