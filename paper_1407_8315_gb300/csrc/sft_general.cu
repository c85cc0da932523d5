// sft_general.cu -- generally K-sparse signals (Sec. III, Algorithm 2) for
// sm_103a.
//
// Per call, batched over B signals of one plan (M bins, d = N / M):
//   gather + FFT   the 2 a_m consecutive shifts 0 .. 2a_m-1 and the r random
//                  shifts n_l (Algorithm 2, Part 1)
//   k_gen_bound,   per bin a lower bound ||H||_F / sqrt(a_m) of the largest
//   k_gen_tau,     singular value, its K-th largest tau_L per signal, and
//   k_gen_prune    the bins whose upper bound ||H||_F reaches tau_L (the
//                  others cannot hold a vote) queued for
//   k_gen_svals    the a_m singular values of the a_m x a_m Hankel matrix of
//                  m_0 .. m_{2a_m-2} (Eq. (26)) by one-sided Jacobi in FP64
//                  (Algorithm 2, Part 2), grid-stride over the queue
//   k_gen_vote     one CTA per signal: the K largest singular values (radix
//                  select on their FP64 bit patterns, ties to the lower
//                  index) vote a_k per bin (Algorithm 2, Part 2); bins with a_k > 0
//                  are queued
//   k_gen_solve1,  per voted bin (one-alias bins, then the others): the a_k x a_k
//   _multi         Hankel locator, |P~| at all
//                  d candidates of U_k with the 2 a_k smallest kept (pruning
//                  Steps 2-3), Subspace Pursuit on the pruned sensing matrix
//                  Phi_p (Algorithm 2, Parts 3-4)
//   k_finalize     as for the exact transform
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "sft_decode.cuh"
#include "sft_device_util.cuh"
#include "sft_internal.h"

namespace sft {

struct GenArgs {
  int64_t N, M, d, K;
  int a_max, r, keep, sp_iters;
  const void* Y;  // rows 0..2a_m-1: consecutive shifts; 2a_m..2a_m+r-1: random
  int64_t held_elems;
  double* sv;   // [B][M a_m]
  uint8_t* ak;  // [B][M0] votes
  int2* queue;
  int* qcount;
  const int64_t* cs;  // the r random shifts n_l
  const int64_t* K_table;  // per-signal K (heterogeneous batches) or null
  uint8_t* slot_cnt;
  int64_t* slot_s;
  void* slot_p;
  int32_t* flags;
  OmegaTab om;
  const int16_t* prop;  // learned proposal: 8 candidates t per queue entry, or null
  double* tau_lo;       // per signal: pruning threshold tau_L
  double* lbound;       // [B][M]: per-bin lower bound of sigma_1
  int2* svq;            // bins whose singular values are computed
  int* svq_count;
  // voted bins: a_k = 1 filed from the front of `queue` (count *qcount),
  // a_k >= 2 from the back (count *qcount_hi, entry i at qcap - 1 - i)
  int* qcount_hi;
  int64_t qcap;
};

// One-sided Jacobi on the n x n Hankel H_ij = m_{i+j}: rotate column pairs
// until orthogonal (phase-align the inner product, then a real rotation with
// cot 2theta = (beta - alpha) / (2|gamma|)); singular values = column norms,
// returned descending.
template <int n>
__device__ void hankel_svals(const cdbl* m, double* sv) {
  cdbl A[n * n];
#pragma unroll
  for (int i = 0; i < n; ++i)
#pragma unroll
    for (int j = 0; j < n; ++j) A[i * n + j] = m[i + j];
  for (int sweep = 0; sweep < 30; ++sweep) {
    // a sweep that rotates no pair (every |gamma| <= 1e-15 sqrt(alpha beta),
    // compared squared) ends the iteration
    bool rotated = false;
#pragma unroll
    for (int p = 0; p < n; ++p) {
#pragma unroll
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0.0, beta = 0.0;
        cdbl gamma = mk(0.0, 0.0);
#pragma unroll
        for (int i = 0; i < n; ++i) {
          alpha += norm2(A[i * n + p]);
          beta += norm2(A[i * n + q]);
          gamma = gamma + conjd(A[i * n + p]) * A[i * n + q];
        }
        const double g2 = norm2(gamma), ab = alpha * beta;
        if (!(g2 > 0.0) || !(ab > 0.0)) continue;
        if (!(g2 > 1e-30 * ab)) continue;
        rotated = true;
        // 1/|gamma| and the rotation's cosine as reciprocal square roots,
        // tan by the reciprocal (fewer FP64 square roots and divisions)
        const double ig = rsqrt(g2);
        const cdbl phc = mk(gamma.x * ig, -gamma.y * ig);  // conj(gamma / |gamma|)
        const double zeta = (beta - alpha) * (0.5 * ig);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) * rcp_d(fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = rsqrt(1.0 + t * t), s = c * t;
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const cdbl ap = A[i * n + p], aq = A[i * n + q] * phc;
          A[i * n + p] = ap * c - aq * s;
          A[i * n + q] = ap * s + aq * c;
        }
      }
    }
    if (!rotated) break;
  }
#pragma unroll
  for (int j = 0; j < n; ++j) {
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) s2 += norm2(A[i * n + j]);
    sv[j] = sqrt(s2);
  }
#pragma unroll
  for (int i = 1; i < n; ++i)
#pragma unroll
    for (int j = n - 1; j >= 1; --j)
      if (j <= i && sv[j - 1] < sv[j]) {
        const double t = sv[j];
        sv[j] = sv[j - 1];
        sv[j - 1] = t;
      }
}

// ||H||_F^2 of the a_m x a_m Hankel matrix of m_0..m_{2a_m-2}: m_l appears
// min(l + 1, 2a_m - 1 - l) times
template <int AM>
__device__ __forceinline__ double hankel_frob2(const cdbl* m) {
  double f2 = 0.0;
#pragma unroll
  for (int l = 0; l < 2 * AM - 1; ++l) f2 += (double)min(l + 1, 2 * AM - 1 - l) * norm2(m[l]);
  return f2;
}

// Pruning bound, per bin: sigma_1 >= L_k = ||H v|| / ||v|| for any v; with
// v = conj of the first row of H (one power step) this is exact for a bin
// holding one alias (H = p z z^T is rank one).  Written to lbound[b M + k]
// for k_gen_tau.  The mixed path forms the bounds in FP32 from the
// float-float hi parts (relative error far below the pruning margin);
// FP64 serves the plain path and values outside the float range.
template <int AM, class C>
__device__ __forceinline__ void power_bound(const C* m, decltype(m[0].x)& v2, decltype(m[0].x)& hv2) {
  typedef decltype(m[0].x) R;
  v2 = R(0);
  hv2 = R(0);
#pragma unroll
  for (int j = 0; j < AM; ++j) v2 += m[j].x * m[j].x + m[j].y * m[j].y;
#pragma unroll
  for (int i = 0; i < AM; ++i) {
    R ax = R(0), ay = R(0);
#pragma unroll
    for (int j = 0; j < AM; ++j) {  // m_{i+j} conj(m_j)
      ax += m[i + j].x * m[j].x + m[i + j].y * m[j].y;
      ay += m[i + j].y * m[j].x - m[i + j].x * m[j].y;
    }
    hv2 += ax * ax + ay * ay;
  }
}

template <class F, int AM>
__device__ __forceinline__ double bin_lower_bound(const typename Store<F>::T* Y, int64_t M,
                                                  int64_t k) {
  if constexpr (std::is_same<F, FF>::value) {
    float2 mf[2 * AM - 1];
#pragma unroll
    for (int j = 0; j < 2 * AM - 1; ++j) {
      const float4 v = Y[j * M + k];
      mf[j] = make_float2(v.x, v.z);
    }
    float v2, hv2;
    power_bound<AM>(mf, v2, hv2);
    if (v2 > 1e-30f && hv2 < 1e37f) return (double)sqrtf(hv2 / v2);
  }
  cdbl m[2 * AM - 1];
#pragma unroll
  for (int j = 0; j < 2 * AM - 1; ++j) m[j] = Store<F>::to_d(Y[j * M + k]);
  double v2, hv2;
  power_bound<AM>(m, v2, hv2);
  return v2 > 0.0 ? sqrt(hv2 / v2) : 0.0;
}

// ||H||_F, the upper bound of every singular value of the bin: FP32 on the
// mixed path, FP64 on the plain path and outside the float range
template <class F, int AM>
__device__ __forceinline__ double bin_upper_bound(const typename Store<F>::T* Y, int64_t M,
                                                  int64_t k) {
  if constexpr (std::is_same<F, FF>::value) {
    float f2 = 0.0f;
#pragma unroll
    for (int l = 0; l < 2 * AM - 1; ++l) {
      const float4 v = Y[l * M + k];
      f2 += (float)min(l + 1, 2 * AM - 1 - l) * (v.x * v.x + v.z * v.z);
    }
    if (f2 < 1e37f) return (double)sqrtf(f2);
  }
  cdbl m[2 * AM - 1];
#pragma unroll
  for (int j = 0; j < 2 * AM - 1; ++j) m[j] = Store<F>::to_d(Y[j * M + k]);
  return sqrt(hankel_frob2<AM>(m));
}

// relative margin of the pruning test: FP32 bounds on the mixed path
template <class F>
__device__ __forceinline__ double prune_margin() {
  return std::is_same<F, FF>::value ? 4e-5 : 1e-12;
}

template <class F, int AM>
__global__ void __launch_bounds__(256) k_gen_bound(GenArgs g) {
  typedef typename Store<F>::T T;
  const int b = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (k >= g.M) return;
  const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
  g.lbound[(int64_t)b * g.M + k] = bin_lower_bound<F, AM>(Y, g.M, k);
}

// Bins that cannot hold a vote: ||H||_F bounds every singular value of the
// bin; if it is below tau_L, the K-th largest of the bins' lower bounds of
// sigma_1 (so tau_L <= the K-th largest singular value of the signal, up to
// the rounding the margin covers), the vote gives the bin nothing.  Every
// bin's singular values are cleared here; the others are queued for
// k_gen_svals (warp-aggregated).
template <class F, int AM>
__global__ void __launch_bounds__(256) k_gen_prune(GenArgs g) {
  typedef typename Store<F>::T T;
  const int b = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * 256 + threadIdx.x;
  bool keep = false;
  if (k < g.M) {
    double* o = g.sv + ((int64_t)b * g.M + k) * AM;
#pragma unroll
    for (int i = 0; i < AM; ++i) o[i] = 0.0;
    const double tau = g.tau_lo[b];
    // a bin whose lower bound already reaches tau_L needs no more reading
    keep = g.lbound[(int64_t)b * g.M + k] >= tau;
    if (!keep) {
      const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
      const double u = bin_upper_bound<F, AM>(Y, g.M, k);
      keep = u * (1.0 + prune_margin<F>()) >= tau && u > 0.0;
    }
  }
  queue_push(keep, b, (int)k, g.svq, g.svq_count);
}

// Singular values of the queued bins (grid-stride over the queue).
template <class F, int AM>
__global__ void __launch_bounds__(128) k_gen_svals(GenArgs g) {
  typedef typename Store<F>::T T;
  const int n = *g.svq_count;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 q = g.svq[e];
    const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)q.x * g.held_elems;
    cdbl m[2 * AM - 1];
#pragma unroll
    for (int j = 0; j < 2 * AM - 1; ++j) m[j] = Store<F>::to_d(Y[j * g.M + q.y]);
    double sv[AM];
    hankel_svals<AM>(m, sv);
    double* o = g.sv + ((int64_t)q.x * g.M + q.y) * AM;
#pragma unroll
    for (int i = 0; i < AM; ++i) o[i] = sv[i];
  }
}

// Block-wide exclusive scan of one int per thread.
__device__ __forceinline__ int gen_block_scan(int v, int* total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;
  }
  __syncthreads();
  const int before = (w > 0 ? wsum[w - 1] : 0) + x - v;
  *total = wsum[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// K-th largest of the n non-negative doubles `keys` (as bit patterns) of
// one signal: MSB-first radix select, 8 passes of 8 bits.  Returns the K-th
// largest key and, in *rem_out, how many of the keys equal to it are among
// the K largest (0 < K <= n).
//
// The signal is the work of one thread-block cluster (one CTA when the
// signals alone fill the GPU, up to eight when they are few): each CTA
// histograms a strided slice of the keys, and after a cluster barrier every
// CTA sums the cluster's histograms through distributed shared memory and
// takes the same digit.  The counts are integers, so the result does not
// depend on the cluster size.  The histogram counts are aggregated per warp
// (one shared atomic per distinct digit in a warp, not one per key), and
// once the keys still matching the selected prefix fit in shared memory
// (cluster-wide) each CTA copies its slice's there, so that the remaining
// passes read no global memory.  Every thread of every CTA of the cluster
// must call this.
constexpr int kSelCand = 4096;

__device__ __forceinline__ void hist_add(unsigned* hist, unsigned digit, bool pred) {
  const unsigned act = __activemask();
  const unsigned mm = __ballot_sync(act, pred);
  if (pred) {
    const unsigned peers = __match_any_sync(mm, digit);
    if ((int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[digit], (unsigned)__popc(peers));
  }
}

__device__ unsigned long long radix_select_desc(const unsigned long long* keys, int64_t n,
                                                long long K, long long* rem_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  __shared__ unsigned hist[256];
  __shared__ unsigned tot[256];
  __shared__ unsigned long long s_prefix;
  __shared__ long long s_rem;
  __shared__ unsigned s_sel_count;
  __shared__ int s_nc;
  __shared__ unsigned long long cand[kSelCand];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int64_t gtid = (int64_t)rank * nthr + tid, gstride = (int64_t)C * nthr;
  unsigned long long prefix = 0ull, mask = 0ull;
  long long rem = K;  // rank (from the top) still to find among keys matching prefix
  bool in_smem = false;
  int nc = 0;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    cl.sync();  // no CTA still reads this CTA's previous histogram
    for (int i = tid; i < 256; i += nthr) hist[i] = 0u;
    __syncthreads();
    if (in_smem) {
      for (int i = tid; i < nc; i += nthr) {
        const unsigned long long key = cand[i];
        hist_add(hist, (unsigned)((key >> shift) & 255ull), (key & mask) == prefix);
      }
    } else {
      for (int64_t i = gtid; i < n; i += gstride) {
        const unsigned long long key = keys[i];
        hist_add(hist, (unsigned)((key >> shift) & 255ull), (key & mask) == prefix);
      }
    }
    cl.sync();  // every CTA's histogram complete
    for (int i = tid; i < 256; i += nthr) {
      unsigned t = 0u;
      for (int r = 0; r < C; ++r) t += cl.map_shared_rank(hist, r)[i];
      tot[i] = t;
    }
    __syncthreads();
    if (tid == 0) {
      long long cum = 0;
      int sel = 0;
      for (int dg = 255; dg >= 0; --dg) {
        if (cum + (long long)tot[dg] >= rem) {
          sel = dg;
          break;
        }
        cum += tot[dg];
      }
      s_prefix = prefix | ((unsigned long long)sel << shift);
      s_rem = rem - cum;
      s_sel_count = tot[sel];
      s_nc = 0;
    }
    __syncthreads();
    prefix = s_prefix;
    rem = s_rem;
    mask |= 255ull << shift;
    // gather this CTA's keys matching the new prefix into shared memory once
    // the cluster's fit (this CTA's are a part of them)
    if (!in_smem && pass < 7 && s_sel_count <= (unsigned)kSelCand) {
      for (int64_t i = gtid; i < n; i += gstride) {
        const unsigned long long key = keys[i];
        if ((key & mask) == prefix) cand[atomicAdd(&s_nc, 1)] = key;
      }
      __syncthreads();
      nc = s_nc;
      in_smem = true;
    }
    __syncthreads();
  }
  cl.sync();  // the last histograms have been read: CTAs may go on (and exit)
  *rem_out = rem;
  return prefix;
}

// tau_L per signal: the K-th largest of the M bins' lower bounds (0 when K
// is 0 or not below M, which disables pruning)
// (one cluster per signal, launched by launch_per_signal)
__global__ void __launch_bounds__(1024, 1) k_gen_tau(GenArgs g) {
  namespace cg = cooperative_groups;
  const cg::cluster_group cl = cg::this_cluster();
  const int b = (int)(blockIdx.x / cl.num_blocks());
  const int64_t Kb = g.K_table != nullptr ? g.K_table[b] : g.K;
  double tau = 0.0;
  if (Kb > 0 && Kb < g.M) {
    long long rem = 0;
    const unsigned long long key = radix_select_desc(
        reinterpret_cast<const unsigned long long*>(g.lbound + (int64_t)b * g.M), g.M, Kb, &rem);
    tau = __longlong_as_double((long long)key);
  }
  if (threadIdx.x == 0 && cl.block_rank() == 0) g.tau_lo[b] = tau;
}

// Algorithm 2, the vote: the K largest of the M a_m singular values of one signal
// (radix select on their bit patterns); of the values equal to the K-th
// largest tau, those of lowest index are selected.
// One cluster per signal (launched by launch_per_signal): CTA rank r of C
// assigns the bins of the r-th of C consecutive chunks; the ties' order
// across CTAs comes from the lower ranks' tie counts (distributed shared
// memory).
__global__ void __launch_bounds__(1024, 1) k_gen_vote(GenArgs g) {
  namespace cg = cooperative_groups;
  const cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int b = (int)(blockIdx.x / C);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int am = g.a_max;
  const int64_t n = g.M * am;
  const unsigned long long* keys =
      reinterpret_cast<const unsigned long long*>(g.sv + (int64_t)b * n);
  uint8_t* ak = g.ak + (int64_t)b * g.M;
  const int64_t Kb = g.K_table != nullptr ? g.K_table[b] : g.K;
  const int64_t K = Kb < n ? Kb : n;
  unsigned long long prefix = 0ull;
  long long rem = 0;
  if (K > 0) prefix = radix_select_desc(keys, n, K, &rem);
  const unsigned long long tau = prefix;  // K-th largest key
  // this CTA's chunk of bins, then a per-thread chunk of it, in index order
  const int64_t cchunk = (g.M + C - 1) / C;
  const int64_t c_lo = min((int64_t)rank * cchunk, g.M), c_hi = min(c_lo + cchunk, g.M);
  const int64_t chunk = (c_hi - c_lo + nthr - 1) / nthr;
  const int64_t k_lo = min(c_lo + (int64_t)tid * chunk, c_hi), k_hi = min(k_lo + chunk, c_hi);
  int ties = 0;
  if (K > 0)
    for (int64_t i = k_lo * am; i < k_hi * am; ++i) ties += keys[i] == tau;
  int tie_total = 0;
  int tie_before = gen_block_scan(ties, &tie_total);
  // ties in the chunks of the lower ranks come first
  __shared__ int s_ties;
  if (tid == 0) s_ties = tie_total;
  cl.sync();
  int tie_lower = 0;
  for (int r = 0; r < rank; ++r) tie_lower += *cl.map_shared_rank(&s_ties, r);
  cl.sync();  // every CTA has read the counts it needs
  tie_before += tie_lower;
  for (int64_t k = k_lo; k < k_hi; ++k) {
    int a = 0;
    if (K > 0) {
      for (int j = 0; j < am; ++j) {
        const unsigned long long key = keys[k * am + j];
        if (key > tau) {
          ++a;
        } else if (key == tau) {
          if (tie_before < rem) ++a;
          ++tie_before;
        }
      }
    }
    ak[k] = (uint8_t)a;
    if (a == 1)
      g.queue[atomicAdd(g.qcount, 1)] = make_int2(b, (int)k);
    else if (a > 1)
      g.queue[g.qcap - 1 - atomicAdd(g.qcount_hi, 1)] = make_int2(b, (int)k);
  }
}

// One thread-block cluster of 1024-thread CTAs per signal: one CTA when the
// signals fill the GPU, else up to eight (a power of two), so that a few
// signals' selections still spread over the SMs.
static void launch_per_signal(void (*kernel)(GenArgs), int64_t B, int nsm, cudaStream_t st,
                              const GenArgs& g) {
  int C = 1;
  while (C < 8 && (int64_t)(2 * C) * B <= nsm) C *= 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(B * C), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, g);
}

// Subspace Pursuit on at most C = 2 a_k candidate columns and 16 rows; the
// arrays are sized by C so that a one-alias bin keeps a small frame.
//
// least squares on the columns T (ascending) of Phi (rows x cols, row-major
// in phi), normal equations by Gaussian elimination with partial pivoting;
// returns |y - Phi_T x|^2 or -1 when singular
template <int C>
__device__ __noinline__ double ls_cols(int rows, int cols, const cdbl* phi, const cdbl* y, const int* T, int nT,
                          cdbl* x, cdbl* res) {
  cdbl G[C * C], gv[C];
  for (int u = 0; u < nT; ++u) {
    gv[u] = mk(0.0, 0.0);
    for (int v = 0; v < nT; ++v) G[u * C + v] = mk(0.0, 0.0);
    for (int i = 0; i < rows; ++i) {
      const cdbl cu = conjd(phi[i * cols + T[u]]);
      gv[u] = gv[u] + cu * y[i];
      for (int v = 0; v < nT; ++v) G[u * C + v] = G[u * C + v] + cu * phi[i * cols + T[v]];
    }
  }
  // squared magnitudes compared on their bit patterns (integer pipes)
  long long amax_b = 0;
  for (int u = 0; u < nT; ++u)
    for (int v = 0; v < nT; ++v) amax_b = max(amax_b, ordbits(norm2(G[u * C + v])));
  const double amax2 = __longlong_as_double(amax_b);
  if (!(amax2 > 0.0)) return -1.0;
  cdbl inv[C];
  for (int c = 0; c < nT; ++c) {
    int piv = c;
    long long best_b = ordbits(norm2(G[c * C + c]));
    for (int rr = c + 1; rr < nT; ++rr) {
      const long long v = ordbits(norm2(G[rr * C + c]));
      if (v > best_b) {
        best_b = v;
        piv = rr;
      }
    }
    const double best = __longlong_as_double(best_b);
    if (!(best > 1e-28 * amax2)) return -1.0;
    if (piv != c) {
      for (int q = 0; q < nT; ++q) {
        const cdbl t = G[c * C + q];
        G[c * C + q] = G[piv * C + q];
        G[piv * C + q] = t;
      }
      const cdbl t = gv[c];
      gv[c] = gv[piv];
      gv[piv] = t;
    }
    inv[c] = conjd(G[c * C + c]) * rcp_d(best);  // 1 / pivot
    for (int rr = c + 1; rr < nT; ++rr) {
      const cdbl f = G[rr * C + c] * inv[c];
      for (int q = c + 1; q < nT; ++q) G[rr * C + q] = G[rr * C + q] - f * G[c * C + q];
      gv[rr] = gv[rr] - f * gv[c];
    }
  }
  for (int rr = nT - 1; rr >= 0; --rr) {
    cdbl acc = gv[rr];
    for (int q = rr + 1; q < nT; ++q) acc = acc - G[rr * C + q] * x[q];
    x[rr] = acc * inv[rr];
  }
  double rn = 0.0;
  for (int i = 0; i < rows; ++i) {
    cdbl f = mk(0.0, 0.0);
    for (int u = 0; u < nT; ++u) f = f + phi[i * cols + T[u]] * x[u];
    res[i] = y[i] - f;
    rn += norm2(res[i]);
  }
  return rn;
}

// indices (ascending) of the ks largest v[i] among allowed i (ties: lower i)
__device__ int top_ks(int n, const double* v, unsigned allowed, int ks, int* out) {
  unsigned taken = 0u;
  int cnt = 0;
  for (int r = 0; r < ks; ++r) {
    int best = -1;
    for (int i = 0; i < n; ++i)
      if (((allowed >> i) & 1u) && !((taken >> i) & 1u) && (best < 0 || v[i] > v[best])) best = i;
    if (best < 0) break;
    taken |= 1u << best;
    ++cnt;
  }
  int w = 0;
  for (int i = 0; i < n; ++i)
    if ((taken >> i) & 1u) out[w++] = i;
  return cnt;
}

// Subspace Pursuit (Dai and Dai 2009) on Phi (rows x cols, cols <= C),
// sparsity ks: T = ks columns most correlated with y; repeat: T' = T + the
// ks columns most correlated with the residual, least squares on T', keep
// its ks largest coefficients, least squares again; stop when the residual
// does not shrink.  Writes the support and the coefficients; returns |T|.
template <int C>
__device__ __noinline__ int subspace_pursuit(int rows, int cols, const cdbl* phi, const cdbl* y, int ks,
                                int iters, int* T, cdbl* x) {
  const unsigned all = (cols >= 32) ? 0xffffffffu : ((1u << cols) - 1u);
  double corr[C];
  cdbl res[16], xn[C], resn[16];
  if (ks > cols) ks = cols;
  for (int j = 0; j < cols; ++j) {
    cdbl c = mk(0.0, 0.0);
    for (int i = 0; i < rows; ++i) c = c + conjd(phi[i * cols + j]) * y[i];
    corr[j] = norm2(c);
  }
  int nT = top_ks(cols, corr, all, ks, T);
  double rn = ls_cols<C>(rows, cols, phi, y, T, nT, x, res);
  if (rn < 0.0) return 0;
  for (int it = 0; it < iters; ++it) {
    for (int j = 0; j < cols; ++j) {
      cdbl c = mk(0.0, 0.0);
      for (int i = 0; i < rows; ++i) c = c + conjd(phi[i * cols + j]) * res[i];
      corr[j] = norm2(c);
    }
    int add[C];
    const int na = top_ks(cols, corr, all, ks, add);
    unsigned in2 = 0u;
    for (int u = 0; u < nT; ++u) in2 |= 1u << T[u];
    for (int u = 0; u < na; ++u) in2 |= 1u << add[u];
    int T2[C], n2 = 0;
    for (int j = 0; j < cols; ++j)
      if ((in2 >> j) & 1u) T2[n2++] = j;
    cdbl x2[C], r2[16];
    if (ls_cols<C>(rows, cols, phi, y, T2, n2, x2, r2) < 0.0) break;
    double mag[C];
    for (int j = 0; j < cols; ++j) mag[j] = 0.0;
    for (int u = 0; u < n2; ++u) mag[T2[u]] = norm2(x2[u]);
    int Tn[C];
    const int nn = top_ks(cols, mag, in2, ks, Tn);
    const double rnn = ls_cols<C>(rows, cols, phi, y, Tn, nn, xn, resn);
    if (rnn < 0.0 || rnn >= rn) break;
    nT = nn;
    for (int u = 0; u < nT; ++u) {
      T[u] = Tn[u];
      x[u] = xn[u];
    }
    for (int i = 0; i < rows; ++i) res[i] = resn[i];
    rn = rnn;
  }
  return nT;
}

// squared residual of a bin's solution {(s_u, p_u)} over all its equations:
// the 2a_m consecutive syndromes and the r random-shift syndromes (Eq. (3))
template <class F>
__device__ double judge_res2(const GenArgs& g, const typename Store<F>::T* Y, int64_t k,
                             const int64_t* s, const cdbl* p, int n) {
  double acc = 0.0;
  const int nsyn = 2 * g.a_max + g.r;
  for (int l = 0; l < nsyn; ++l) {
    const int64_t sh = l < 2 * g.a_max ? (int64_t)l : g.cs[l - 2 * g.a_max];
    cdbl res = Store<F>::to_d(Y[(int64_t)l * g.M + k]);
    for (int u = 0; u < n; ++u) res = res - p[u] * omega_pow(g.om, s[u] * sh);
    acc += norm2(res);
  }
  return acc;
}

template <class F, int A>
__device__ void solve_bin(const GenArgs& g, int b, int64_t k, int e) {
  typedef typename Store<F>::T T;
  const int64_t M = g.M, d = g.d;
  const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
  const int r = g.r;
  cdbl y[16];
  for (int j = 0; j < r; ++j) y[j] = Store<F>::to_d(Y[(2 * g.a_max + j) * M + k]);
  int64_t s_out[2 * A];
  cdbl p_out[2 * A];
  int nout = 0;
  // the plain path's kept candidates (ascending), to recognise a proposal
  // that repeats them
  int kept_t[2 * A];
  int n_kept = -1;
  cdbl m[2 * A];
#pragma unroll
  for (int j = 0; j < 2 * A; ++j) m[j] = Store<F>::to_d(Y[j * M + k]);
  // Step 2 (a): the a x a Hankel system with the observed syndromes
  cdbl H[A * A], rhs[A], c[A];
#pragma unroll
  for (int i = 0; i < A; ++i) {
#pragma unroll
    for (int j = 0; j < A; ++j) H[i * A + j] = m[i + j];
    rhs[i] = -m[A + i];
  }
  if (solve_small<A>(H, rhs, c)) {
    // (b)-(c): |P~(z)| at every z = omega^{k + tM} of U_k; keep the smallest
    const int nk = (int)min((int64_t)min(g.keep * A, 2 * A), d);
    double bv[2 * A];
    int bt[2 * A];
    int have = 0;
    // one alias: |P~(z)|^2 = 1 + |c0|^2 - 2 |c0| cos(arg z - arg(-c0)) on the
    // unit circle, so the two smallest are the two candidates nearest the
    // root -c0 in angle, t = floor(u) and floor(u) + 1 with u the root's
    // fractional candidate index -- decided in FP32 unless u lies near an
    // integer (where the second place is a near tie: the full pass decides)
    int64_t t_hi = d;
    if constexpr (A == 1) {
      const float zx = (float)(-c[0].x), zy = (float)(-c[0].y);
      const float az = fabsf(zx) + fabsf(zy);
      if (nk == 2 && az > 1e-30f && az < 1e30f) {
        const float df = (float)d;
        const float u = fmaf(atan2f(zy, zx), df * 0.15915494309189533577f,
                             -(float)k / (float)M);
        const float fl = floorf(u), fr = u - fl;
        const float margin = fmaxf(1e-3f, 8e-7f * df);
        if (fr > margin && fr < 1.0f - margin) {
          // d is a power of two: the masks are the modulo, negatives too
          const int64_t t0 = (int64_t)((int)fl & (int)(d - 1));
          const int64_t t1 = (t0 + 1) & (d - 1);
          bt[0] = (int)min(t0, t1);
          bt[1] = (int)max(t0, t1);
          have = 2;
          t_hi = 0;  // no full pass
        }
      }
    }
    for (int64_t t = 0; t < t_hi; ++t) {
      const cdbl z = omega_pow(g.om, k + t * M);
      cdbl P = mk(1.0, 0.0);
#pragma unroll
      for (int j = A - 1; j >= 0; --j) P = P * z + c[j];
      const double v = norm2(P);
      if (have < nk || v < bv[nk - 1]) {
        int pos = have < nk ? have : nk - 1;
        while (pos > 0 && bv[pos - 1] > v) {  // stable: equal values keep lower t first
          bv[pos] = bv[pos - 1];
          bt[pos] = bt[pos - 1];
          --pos;
        }
        bv[pos] = v;
        bt[pos] = (int)t;
        if (have < nk) ++have;
      }
    }
    // Step 3: kept candidates in ascending t; Phi_p[j][u] = omega^{(k + t_u M) n_j}
    for (int i = 1; i < have; ++i)
      for (int j = i; j > 0 && bt[j - 1] > bt[j]; --j) {
        const int tt = bt[j];
        bt[j] = bt[j - 1];
        bt[j - 1] = tt;
      }
    cdbl phi[16 * 2 * A];
    for (int j = 0; j < r; ++j)
      for (int u = 0; u < have; ++u)
        phi[j * have + u] = omega_pow(g.om, (k + (int64_t)bt[u] * M) * g.cs[j]);
    n_kept = have;
    for (int u = 0; u < have; ++u) kept_t[u] = bt[u];
    int Tsup[2 * A];
    cdbl xs[2 * A];
    const int nz = subspace_pursuit<2 * A>(r, have, phi, y, A, g.sp_iters, Tsup, xs);
    for (int u = 0; u < nz; ++u) {
      if (xs[u].x == 0.0 && xs[u].y == 0.0) continue;
      s_out[nout] = k + (int64_t)bt[Tsup[u]] * M;
      p_out[nout] = xs[u];
      ++nout;
    }
  }
  // learned proposal: Subspace Pursuit on the network's candidates, kept
  // only when its residual over all equations is below (1 - 1e-6) times
  // the plain solution's
  if (g.prop != nullptr) {
    const int16_t* pr = g.prop + (int64_t)e * 8;
    int ct[2 * A];
    int nc = 0;
    for (int u = 0; u < 8 && nc < 2 * A; ++u)
      if (pr[u] >= 0) ct[nc++] = pr[u];
    // the same candidates in the same (ascending) order as the plain path:
    // Subspace Pursuit would repeat the plain solution exactly, and the
    // judge keeps the plain one on equal residuals -- nothing to do
    bool same = nc == n_kept;
    for (int u = 0; same && u < nc; ++u) same = ct[u] == kept_t[u];
    if (nc > 0 && !same) {
      cdbl phi2[16 * 2 * A];
      for (int j = 0; j < r; ++j)
        for (int u = 0; u < nc; ++u)
          phi2[j * nc + u] = omega_pow(g.om, (k + (int64_t)ct[u] * M) * g.cs[j]);
      int T2[2 * A];
      cdbl x2[2 * A];
      const int nz2 = subspace_pursuit<2 * A>(r, nc, phi2, y, A, g.sp_iters, T2, x2);
      int64_t s2[2 * A];
      cdbl p2[2 * A];
      int n2 = 0;
      for (int u = 0; u < nz2; ++u) {
        if (x2[u].x == 0.0 && x2[u].y == 0.0) continue;
        s2[n2] = k + (int64_t)ct[T2[u]] * M;
        p2[n2] = x2[u];
        ++n2;
      }
      if (n2 > 0) {
        const double rp = judge_res2<F>(g, Y, k, s_out, p_out, nout);
        const double rm = judge_res2<F>(g, Y, k, s2, p2, n2);
        if (rm < (1.0 - 1e-6) * rp) {
          for (int u = 0; u < n2; ++u) {
            s_out[u] = s2[u];
            p_out[u] = p2[u];
          }
          nout = n2;
        }
      }
    }
  }
  if (nout == 0) return;
  file_n<F>(nout, s_out, p_out, g.M, g.slot_cnt + (int64_t)b * g.M, g.slot_s + (int64_t)b * g.M * kSlots,
            reinterpret_cast<T*>(g.slot_p) + (int64_t)b * g.M * kSlots, g.flags + b);
}

// The one-alias bins (the front of the queue; every warp full and of one
// kind) and the bins with a_k >= 2 (the back of the queue), grid-stride.
template <class F>
__global__ void __launch_bounds__(128) k_gen_solve1(GenArgs g) {
  const int n = *g.qcount;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 q = g.queue[e];
    solve_bin<F, 1>(g, q.x, q.y, e);
  }
}

template <class F>
__global__ void __launch_bounds__(128) k_gen_solve_multi(GenArgs g) {
  const int n = *g.qcount_hi;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int e = (int)(g.qcap - 1 - i);
    const int2 q = g.queue[e];
    switch (g.ak[(int64_t)q.x * g.M + q.y]) {
      case 2: solve_bin<F, 2>(g, q.x, q.y, e); break;
      case 3: solve_bin<F, 3>(g, q.x, q.y, e); break;
      case 4: solve_bin<F, 4>(g, q.x, q.y, e); break;
      default: break;
    }
  }
}

// Part 1 and Part 2 (gather/FFT of every shift, singular values, vote);
// returns the arguments of the later stages
template <class F>
static GenArgs general_front(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride,
                             cudaStream_t st) {
  const Workspace& W = P->ws;
  const int am = P->p.a_max, r = P->p.n_cs_shifts;
  // Part 1: 2 a_m consecutive shifts (rows 0..2a_m-1), r random shifts after
  launch_gather_fft_any(P, B, x, x_stride, P->p.d, P->log2M0, 0, 2 * am, W.held[0], P->M0, 0,
                        false, st, nullptr, "gather_fft_consecutive");
  launch_gather_fft_any(P, B, x, x_stride, P->p.d, P->log2M0, 0, r, W.held[0], P->M0, 2 * am,
                        false, st, P->tab.cs_shifts, "gather_fft_random");
  // the bounds use the solution slots (filled only by k_gen_solve), the
  // pruned-bin queue the second queue and counter
  GenArgs g{P->p.N, P->M0, P->p.d, P->p.K, am, r, 2, 8, W.held[0], W.held_elems, W.sv, W.T[0],
            W.queue[0], W.qcount, P->tab.cs_shifts, P->K_table, W.slot_cnt, W.slot_s, W.slot_p,
            W.flags, OmegaTab{P->tab.om_hi, P->tab.om_lo, P->tab.om_lo_bits, P->p.N - 1},
            nullptr, reinterpret_cast<double*>(W.ymax2), reinterpret_cast<double*>(W.slot_s),
            W.queue[1], W.qcount + 1, W.qcount + 2, B * P->M0};
  dim3 sgrid((unsigned)((P->M0 + 255) / 256), (unsigned)B);
  stage_begin(P, "gen_bound", st);
  switch (am) {
    case 1: k_gen_bound<F, 1><<<sgrid, 256, 0, st>>>(g); break;
    case 2: k_gen_bound<F, 2><<<sgrid, 256, 0, st>>>(g); break;
    case 3: k_gen_bound<F, 3><<<sgrid, 256, 0, st>>>(g); break;
    default: k_gen_bound<F, 4><<<sgrid, 256, 0, st>>>(g); break;
  }
  stage_end(P, st);
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  stage_begin(P, "gen_tau", st);
  launch_per_signal(k_gen_tau, B, nsm, st, g);
  stage_end(P, st);
  stage_begin(P, "gen_prune", st);
  switch (am) {
    case 1: k_gen_prune<F, 1><<<sgrid, 256, 0, st>>>(g); break;
    case 2: k_gen_prune<F, 2><<<sgrid, 256, 0, st>>>(g); break;
    case 3: k_gen_prune<F, 3><<<sgrid, 256, 0, st>>>(g); break;
    default: k_gen_prune<F, 4><<<sgrid, 256, 0, st>>>(g); break;
  }
  stage_end(P, st);
  const unsigned vgrid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((B * P->M0 + 127) / 128, (int64_t)P->dec_ctas_per_sm * nsm));
  stage_begin(P, "gen_svals", st);
  switch (am) {
    case 1: k_gen_svals<F, 1><<<vgrid, 128, 0, st>>>(g); break;
    case 2: k_gen_svals<F, 2><<<vgrid, 128, 0, st>>>(g); break;
    case 3: k_gen_svals<F, 3><<<vgrid, 128, 0, st>>>(g); break;
    default: k_gen_svals<F, 4><<<vgrid, 128, 0, st>>>(g); break;
  }
  stage_end(P, st);
  stage_begin(P, "gen_vote", st);
  launch_per_signal(k_gen_vote, B, nsm, st, g);
  stage_end(P, st);
  return g;
}

// Parts 3-4: pruning and Subspace Pursuit per voted bin
template <class F>
static void general_solve(sft_plan_s* P, int64_t B, int nsm, cudaStream_t st, const GenArgs& g) {
  const int64_t maxq =
      B * (P->K_table != nullptr ? P->M0 : std::min<int64_t>(P->M0, std::max<int64_t>(P->p.K, 1)));
  const unsigned dgrid =
      (unsigned)std::max<int64_t>(1, std::min<int64_t>((maxq + 127) / 128, (int64_t)P->dec_ctas_per_sm * nsm));
  stage_begin(P, "gen_solve", st);
  k_gen_solve1<F><<<dgrid, 128, 0, st>>>(g);
  if (P->p.a_max >= 2) k_gen_solve_multi<F><<<dgrid, 128, 0, st>>>(g);
  stage_end(P, st);
}

// ------------------------------------------ the CS model without pruning
// Sec. III-B without the pruning strategy: per bin k the r random-shift
// syndromes y_j = Y_{n_j}[k] = sum_t b_t omega^{(k + tM) n_j} (Eq. (18))
// over all d candidates, solved by Subspace Pursuit at sparsity a_m, every
// non-zero coefficient kept.  As omega^{(k + tM) n_j} = omega^{k n_j}
// e^{2 pi i t n_j / d}, the bin's rows are rotated once (y~_j =
// omega^{-k n_j} y_j, with the same solution b) and every column entry is
// read from a shared-memory table of the d-th roots of unity,
// Phi~[j][t] = E[(t n_j) mod d].  One warp per bin: the lanes stride the d
// candidates for the correlations and merge their top-a lists; lane 0
// solves the least-squares problems (at most 2 a_m columns) and shares the
// residual through shared memory.
constexpr int kUnprWarps = 8;

struct UnprWarp {
  cdbl yr[16];   // rotated syndromes y~
  cdbl res[16];  // current residual (rotated frame)
  int go;        // lane 0's verdict: continue with this bin
};

// The ks largest |sum_j conj(E[(t n_j) mod d]) v_j|^2 over t < d (ties: the
// smaller t), returned ascending in T; every lane returns the same list.
__device__ int unpr_top(const cdbl* E, int64_t d, const int* nj, int r, const cdbl* v, int ks,
                        int* T) {
  const int lane = threadIdx.x & 31;
  double bv[4];
  int bt[4];
  int have = 0;
  for (int64_t t = lane; t < d; t += 32) {
    cdbl c = mk(0.0, 0.0);
    for (int j = 0; j < r; ++j) c = c + conjd(E[((int64_t)nj[j] * t) & (d - 1)]) * v[j];
    const double val = norm2(c);
    if (have < ks || val > bv[ks - 1]) {  // lane order visits t ascending: ties keep the first
      int pos = have < ks ? have : ks - 1;
      while (pos > 0 && bv[pos - 1] < val) {
        bv[pos] = bv[pos - 1];
        bt[pos] = bt[pos - 1];
        --pos;
      }
      bv[pos] = val;
      bt[pos] = (int)t;
      if (have < ks) ++have;
    }
  }
  int head = 0, n = 0;
  int out[4];
  for (int round = 0; round < ks; ++round) {
    double v0 = head < have ? bv[head] : -1.0;
    int t0 = head < have ? bt[head] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v1 = __shfl_xor_sync(0xffffffffu, v0, o);
      const int t1 = __shfl_xor_sync(0xffffffffu, t0, o);
      if (v1 > v0 || (v1 == v0 && t1 < t0)) {
        v0 = v1;
        t0 = t1;
      }
    }
    if (v0 < 0.0) break;
    if (head < have && bt[head] == t0) ++head;
    out[n++] = t0;
  }
  for (int i = 1; i < n; ++i)  // ascending candidates
    for (int j = i; j > 0 && out[j - 1] > out[j]; --j) {
      const int tt = out[j];
      out[j] = out[j - 1];
      out[j - 1] = tt;
    }
  for (int i = 0; i < n; ++i) T[i] = out[i];
  return n;
}

// least squares of the rotated syndromes on the candidates T (lane 0)
__device__ double unpr_ls(const cdbl* E, int64_t d, const int* nj, int r, const cdbl* yr,
                          const int* T, int n, cdbl* x, cdbl* res) {
  cdbl phi[16 * 8];
  int id[8];
  for (int u = 0; u < n; ++u) id[u] = u;
  for (int j = 0; j < r; ++j)
    for (int u = 0; u < n; ++u) phi[j * n + u] = E[((int64_t)nj[j] * T[u]) & (d - 1)];
  return ls_cols<8>(r, n, phi, yr, id, n, x, res);
}

template <class F>
__global__ void __launch_bounds__(32 * kUnprWarps) k_gen_unpruned(GenArgs g, int64_t B) {
  typedef typename Store<F>::T T;
  extern __shared__ __align__(16) char smem_u[];
  const int64_t d = g.d, M = g.M;
  const int r = g.r, ks = g.a_max;
  cdbl* E = reinterpret_cast<cdbl*>(smem_u);
  UnprWarp* w = reinterpret_cast<UnprWarp*>(E + d) + (threadIdx.x >> 5);
  int nj[16];
  for (int j = 0; j < r; ++j) nj[j] = (int)g.cs[j];
  for (int64_t t = threadIdx.x; t < d; t += blockDim.x) E[t] = omega_pow(g.om, t * M);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * kUnprWarps;
  for (int64_t e = (int64_t)blockIdx.x * kUnprWarps + (threadIdx.x >> 5); e < B * M; e += nw) {
    const int b = (int)(e / M);
    const int64_t k = e - (int64_t)b * M;
    const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
    if (lane < r)
      w->yr[lane] = conjd(omega_pow(g.om, k * g.cs[lane])) *
                    Store<F>::to_d(Y[(2 * g.a_max + lane) * M + k]);
    __syncwarp();
    // initial selection and its least squares
    int Tc[8], nT = unpr_top(E, d, nj, r, w->yr, ks, Tc);
    cdbl x[8];
    double rn = -1.0;
    if (lane == 0) {
      rn = unpr_ls(E, d, nj, r, w->yr, Tc, nT, x, w->res);
      w->go = rn >= 0.0;
    }
    __syncwarp();
    if (!w->go) continue;
    for (int it = 0; it < g.sp_iters; ++it) {
      int add[8];
      const int na = unpr_top(E, d, nj, r, w->res, ks, add);
      if (lane == 0) {
        // union, least squares on it, its ks largest coefficients, again
        int U[8], nu = 0, i = 0, j = 0;
        while (i < nT || j < na) {
          const int v = (j >= na || (i < nT && Tc[i] <= add[j])) ? Tc[i] : add[j];
          if (i < nT && Tc[i] == v) ++i;
          if (j < na && add[j] == v) ++j;
          U[nu++] = v;
        }
        cdbl xu[8], ru[16];
        bool ok = unpr_ls(E, d, nj, r, w->yr, U, nu, xu, ru) >= 0.0;
        if (ok) {
          double mag[8];
          for (int u = 0; u < nu; ++u) mag[u] = norm2(xu[u]);
          int sel[8];
          const int nn = top_ks(nu, mag, nu >= 32 ? 0xffffffffu : ((1u << nu) - 1u), ks, sel);
          int Tn[8];
          for (int u = 0; u < nn; ++u) Tn[u] = U[sel[u]];
          cdbl xn[8], rsn[16];
          const double rnn = unpr_ls(E, d, nj, r, w->yr, Tn, nn, xn, rsn);
          ok = rnn >= 0.0 && rnn < rn;
          if (ok) {
            nT = nn;
            for (int u = 0; u < nn; ++u) {
              Tc[u] = Tn[u];
              x[u] = xn[u];
            }
            for (int q = 0; q < r; ++q) w->res[q] = rsn[q];
            rn = rnn;
          }
        }
        w->go = ok;
      }
      __syncwarp();
      if (!w->go) break;  // (only lane 0's selection and coefficients are used)
    }
    if (lane == 0) {
      int64_t s_out[8];
      cdbl p_out[8];
      int nout = 0;
      for (int u = 0; u < nT; ++u) {
        if (x[u].x == 0.0 && x[u].y == 0.0) continue;
        s_out[nout] = k + (int64_t)Tc[u] * M;
        p_out[nout] = x[u];
        ++nout;
      }
      if (nout > 0)
        file_n<F>(nout, s_out, p_out, M, g.slot_cnt + (int64_t)b * M, g.slot_s + (int64_t)b * M * kSlots,
                  reinterpret_cast<T*>(g.slot_p) + (int64_t)b * M * kSlots, g.flags + b);
    }
    __syncwarp();
  }
}

static size_t unpruned_smem(int64_t d) { return (size_t)d * sizeof(cdbl) + kUnprWarps * sizeof(UnprWarp); }

template <class F>
static void launch_unpruned_t(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                              cudaStream_t st) {
  const Workspace& W = P->ws;
  const int am = P->p.a_max, r = P->p.n_cs_shifts;
  // only the r random shifts (rows 2a_m .. 2a_m + r - 1 of the general layout)
  launch_gather_fft_any(P, B, x, x_stride, P->p.d, P->log2M0, 0, r, W.held[0], P->M0, 2 * am,
                        false, st, P->tab.cs_shifts, "gather_fft_random");
  GenArgs g{P->p.N, P->M0, P->p.d, P->p.K, am, r, 2, 8, W.held[0], W.held_elems, nullptr,
            nullptr, nullptr, nullptr, P->tab.cs_shifts, nullptr, W.slot_cnt, W.slot_s,
            W.slot_p, W.flags,
            OmegaTab{P->tab.om_hi, P->tab.om_lo, P->tab.om_lo_bits, P->p.N - 1}};
  const size_t smem = unpruned_smem(P->p.d);
  // the attribute is set to the largest table (d = 4096) so that no plan
  // lowers it under another's captured launches
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gen_unpruned<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)unpruned_smem(4096));
    attr_set = true;
  }
  const int64_t warps = B * P->M0;
  const int64_t ctas = std::min<int64_t>((warps + kUnprWarps - 1) / kUnprWarps, (int64_t)nsm * 8);
  stage_begin(P, "gen_unpruned_sp", st);
  k_gen_unpruned<F><<<(unsigned)ctas, 32 * kUnprWarps, smem, st>>>(g, B);
  stage_end(P, st);
}

template <class F>
static void launch_general_t(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                             cudaStream_t st) {
  if (P->p.mode == SFT_GENERAL_UNPRUNED) {
    launch_unpruned_t<F>(P, B, x, x_stride, nsm, st);
    return;
  }
  GenArgs g = general_front<F>(P, B, x, x_stride, st);
  if (P->mlp != nullptr && P->mlp_prop != nullptr) {
    mlp_propose(P, B, nsm, st);
    g.prop = P->mlp_prop;
  }
  general_solve<F>(P, B, nsm, st, g);
}

void launch_general(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                    cudaStream_t st) {
  if (P->p.precision == SFT_FP64)
    launch_general_t<F64>(P, B, x, x_stride, nsm, st);
  else
    launch_general_t<FF>(P, B, x, x_stride, nsm, st);
}

void launch_general_features(sft_plan_s* P, int64_t B, const void* x, int64_t x_stride, int nsm,
                             float* feat, int32_t* rows, int64_t cap_rows, cudaStream_t st) {
  if (P->p.precision == SFT_FP64)
    general_front<F64>(P, B, x, x_stride, st);
  else
    general_front<FF>(P, B, x, x_stride, st);
  mlp_features(P, B, nsm, feat, rows, cap_rows, st);
}

}  // namespace sft
