// sft_wide.cu -- bins with more than four aliases (a = 5..8) on the exact
// paths, and the instances of the per-bin kernels that a_max > 4 needs.
// Sec. II-B: above four aliases the locator still comes from a quadratic-cost
// recurrence (Berlekamp-Massey), but the roots have no closed form; the
// candidates of the bin are known, so they are searched.
//
// One warp per queued bin:
//   (i)   Berlekamp-Massey on m_0..m_{2a-1} (lane 0): the shortest linear
//         recurrence; the locator exists when its length is a, and then
//         c_j = C_{a-j} solves Eq. (4)-(5);
//   (ii)  the candidate search: |P(omega^{k+tM})|^2 at every t < d (lanes
//         stride the candidates, per-lane lists of the a smallest are
//         merged; ties to the smaller t), the a smallest kept, each at most
//         root_tol (1 + sum |c_j|) in magnitude;
//   (iii) the values by least squares over all nm equations of Eq. (3): the
//         normal matrix entries sum_i omega^{(s_v - s_u) i} and the
//         right-hand side (lanes per entry), solved on lane 0; then every
//         value above theta and the residual over all equations within
//         res_tol (lanes per equation).
// The same steps as the FP64 oracle's decoder for a > 4, in FP64.
#include <algorithm>
#include <type_traits>

#include "sft_internal.h"
#include "sft_levels.cuh"

namespace sft {
namespace {

constexpr int kWideWarps = 4;  // warps (bins in flight) per CTA

struct WideWarp {
  cdbl m[16];  // syndromes
  cdbl G[64];  // normal matrix
  cdbl g[8];   // right-hand side
  cdbl p[8];   // values
  cdbl r[16];  // residual
  int ok;
};

// Berlekamp-Massey (Massey 1969) over the 2a syndromes; c_j = C_{a-j} when
// the recurrence has length a.  A discrepancy is zero only when exactly zero.
template <int A>
__device__ bool bm_locator(const cdbl* m, cdbl* c) {
  cdbl C[2 * A + 1], Bp[2 * A + 1];
#pragma unroll
  for (int i = 0; i <= 2 * A; ++i) {
    C[i] = mk(0.0, 0.0);
    Bp[i] = mk(0.0, 0.0);
  }
  C[0] = mk(1.0, 0.0);
  Bp[0] = mk(1.0, 0.0);
  int L = 0, shift = 1;
  cdbl bd = mk(1.0, 0.0);
  for (int n = 0; n < 2 * A; ++n) {
    cdbl delta = m[n];
    for (int i = 1; i <= L; ++i) delta = delta + C[i] * m[n - i];
    if (delta.x == 0.0 && delta.y == 0.0) {
      ++shift;
      continue;
    }
    const cdbl f = cdivd(delta, bd);
    if (2 * L <= n) {
      cdbl T[2 * A + 1];
#pragma unroll
      for (int i = 0; i <= 2 * A; ++i) T[i] = C[i];
      for (int i = 0; i + shift <= 2 * A; ++i) C[i + shift] = C[i + shift] - f * Bp[i];
      L = n + 1 - L;
#pragma unroll
      for (int i = 0; i <= 2 * A; ++i) Bp[i] = T[i];
      bd = delta;
      shift = 1;
    } else {
      for (int i = 0; i + shift <= 2 * A; ++i) C[i + shift] = C[i + shift] - f * Bp[i];
      ++shift;
    }
  }
  if (L != A) return false;
#pragma unroll
  for (int j = 0; j < A; ++j) c[j] = C[A - j];
  return true;
}

// Decodes bin k (syndromes in w->m, nm of them) with A aliases; every lane
// calls it and every lane returns the same verdict.  On success s (all
// lanes) and w->p, w->r (the residual) hold the solution.
template <int A>
__device__ bool decode_wide(WideWarp* w, int nm, int64_t k, int64_t M, int64_t d,
                            const OmegaTab& om, const Tol2& tol, int64_t* s) {
  const int lane = threadIdx.x & 31;
  // (i) the locator, on lane 0
  cdbl c[A];
  if (lane == 0) w->ok = bm_locator<A>(w->m, c);
  __syncwarp();
  if (!w->ok) return false;
#pragma unroll
  for (int j = 0; j < A; ++j) {
    c[j].x = __shfl_sync(0xffffffffu, c[j].x, 0);
    c[j].y = __shfl_sync(0xffffffffu, c[j].y, 0);
  }
  double bound = 1.0;
#pragma unroll
  for (int j = 0; j < A; ++j) bound += absd(c[j]);
  bound *= sqrt(tol.root2);
  // (ii) the a smallest |P| over the candidates: per-lane lists, then merge
  double bv[A];
  int bt[A];
  int have = 0;
  for (int64_t t = lane; t < d; t += 32) {
    const cdbl z = omega_pow(om, k + t * M);
    cdbl P = mk(1.0, 0.0);
#pragma unroll
    for (int j = A - 1; j >= 0; --j) P = P * z + c[j];
    const double v = norm2(P);
    if (have < A || v < bv[A - 1]) {  // t ascending per lane: ties keep the first
      int pos = have < A ? have : A - 1;
      while (pos > 0 && bv[pos - 1] > v) {
        bv[pos] = bv[pos - 1];
        bt[pos] = bt[pos - 1];
        --pos;
      }
      bv[pos] = v;
      bt[pos] = (int)t;
      if (have < A) ++have;
    }
  }
  int head = 0;
  double vlast = 0.0;
  int tsel[A];
#pragma unroll
  for (int j = 0; j < A; ++j) {
    double v0 = head < have ? bv[head] : INFINITY;
    int t0 = head < have ? bt[head] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double v1 = __shfl_xor_sync(0xffffffffu, v0, o);
      const int t1 = __shfl_xor_sync(0xffffffffu, t0, o);
      if (v1 < v0 || (v1 == v0 && t1 < t0)) {
        v0 = v1;
        t0 = t1;
      }
    }
    if (head < have && bt[head] == t0) ++head;
    tsel[j] = t0;
    vlast = v0;
  }
  if (!(vlast <= bound * bound)) return false;  // also fails when d < A (infinite)
  // ascending locations
#pragma unroll
  for (int i = 1; i < A; ++i)
    for (int j = i; j > 0 && tsel[j - 1] > tsel[j]; --j) {
      const int tt = tsel[j];
      tsel[j] = tsel[j - 1];
      tsel[j - 1] = tt;
    }
#pragma unroll
  for (int j = 0; j < A; ++j) s[j] = k + (int64_t)tsel[j] * M;
  // (iii) normal equations: G_uv = sum_i omega^{(s_v - s_u) i}, g_u =
  // sum_i omega^{-s_u i} m_i (lanes per entry), solved on lane 0
  for (int e = lane; e < A * A + A; e += 32) {
    cdbl acc = mk(0.0, 0.0);
    if (e < A * A) {
      const int u = e / A, v = e % A;
      const int64_t ds = s[v] - s[u];
      for (int i = 0; i < nm; ++i) acc = acc + omega_pow(om, ds * i);
      w->G[e] = acc;
    } else {
      const int u = e - A * A;
      for (int i = 0; i < nm; ++i) acc = acc + conjd(omega_pow(om, s[u] * i)) * w->m[i];
      w->g[u] = acc;
    }
  }
  __syncwarp();
  if (lane == 0) {
    cdbl G[A * A], g[A], p[A];
#pragma unroll
    for (int i = 0; i < A * A; ++i) G[i] = w->G[i];
#pragma unroll
    for (int i = 0; i < A; ++i) g[i] = w->g[i];
    bool ok = solve_small<A>(G, g, p);
#pragma unroll
    for (int j = 0; j < A; ++j) {
      ok = ok && norm2(p[j]) > tol.theta2;
      w->p[j] = p[j];
    }
    w->ok = ok;
  }
  __syncwarp();
  if (!w->ok) return false;
  // the residual over all equations (lanes per equation)
  double mm2 = 0.0, rr2 = 0.0;
  if (lane < nm) {
    cdbl fit = mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < A; ++j) fit = fit + w->p[j] * omega_pow(om, s[j] * lane);
    const cdbl r = w->m[lane] - fit;
    w->r[lane] = r;
    mm2 = norm2(w->m[lane]);
    rr2 = norm2(r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mm2 = fmax(mm2, __shfl_xor_sync(0xffffffffu, mm2, o));
    rr2 = fmax(rr2, __shfl_xor_sync(0xffffffffu, rr2, o));
  }
  __syncwarp();
  return rr2 <= tol.res2 * mm2;
}

// ITER level l = A - 1 >= 4: one warp per queued bin
template <class F, int A>
__global__ void __launch_bounds__(32 * kWideWarps) k_iter_decode_wide(LevelArgs g,
                                                                     const int2* queue,
                                                                     const int* qcount) {
  typedef typename Store<F>::T T;
  constexpr int nm = 2 * A;
  __shared__ WideWarp ws[kWideWarps];
  WideWarp* w = ws + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int n = *qcount;
  const int64_t M = g.M, M0 = g.M0;
  for (int e = blockIdx.x * kWideWarps + (threadIdx.x >> 5); e < n; e += gridDim.x * kWideWarps) {
    const int2 q = queue[e];
    const int b = q.x;
    const int64_t k = q.y;
    T* cur = reinterpret_cast<T*>(g.cur) + (int64_t)b * g.held_elems;
    const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)g.ymax2[b]),
                   g.root_tol * g.root_tol, g.res_tol * g.res_tol};
    if (lane < nm) w->m[lane] = Store<F>::to_d(cur[lane * M + k]);
    __syncwarp();
    int64_t s[A];
    const bool ok = decode_wide<A>(w, nm, k, M, g.d, g.om, tol, s);
    if (ok) {
      if (lane == 0) {
        cdbl p[A];
#pragma unroll
        for (int j = 0; j < A; ++j) p[j] = w->p[j];
        file_solution<F, A>(s, p, M0, g.slot_cnt + (int64_t)b * M0,
                            g.slot_s + (int64_t)b * M0 * kSlots,
                            reinterpret_cast<T*>(g.slot_p) + (int64_t)b * M0 * kSlots,
                            g.flags + b);
      }
      // the recovered terms leave every syndrome held for this bin
      if (lane < nm) cur[lane * M + k] = Store<F>::from_d_small(w->r[lane]);
    }
    if (lane == 0) g.Tcur[(int64_t)b * M0 + k] = ok ? 0 : 1;
    __syncwarp();
  }
}

// FIXED round a = A >= 5 over the bins no smaller a solved: one warp per bin
template <class F, int A>
__global__ void __launch_bounds__(32 * kWideWarps) k_fixed_round_wide(FixedArgs g,
                                                                     const int2* qin,
                                                                     const int* nin, int2* qout,
                                                                     int* nout) {
  typedef typename Store<F>::T T;
  __shared__ WideWarp ws[kWideWarps];
  WideWarp* w = ws + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int n = *nin;
  const int nm = 2 * g.a_max;
  const int64_t M = g.M;
  for (int e = blockIdx.x * kWideWarps + (threadIdx.x >> 5); e < n; e += gridDim.x * kWideWarps) {
    const int2 q = qin[e];
    const int b = q.x;
    const int64_t k = q.y;
    const T* Y = reinterpret_cast<const T*>(g.Y) + (int64_t)b * g.held_elems;
    const Tol2 tol{g.zero_tol * g.zero_tol * __longlong_as_double((long long)g.ymax2[b]),
                   g.root_tol * g.root_tol, g.res_tol * g.res_tol};
    if (lane < nm) w->m[lane] = Store<F>::to_d(Y[lane * M + k]);
    __syncwarp();
    int64_t s[A];
    const bool ok = decode_wide<A>(w, nm, k, M, g.d, g.om, tol, s);
    if (lane == 0) {
      if (ok) {
        cdbl p[A];
#pragma unroll
        for (int j = 0; j < A; ++j) p[j] = w->p[j];
        file_solution<F, A>(s, p, M, g.slot_cnt + (int64_t)b * M, g.slot_s + (int64_t)b * M * kSlots,
                            reinterpret_cast<T*>(g.slot_p) + (int64_t)b * M * kSlots, g.flags + b);
      } else if (qout == nullptr) {
        g.T[(int64_t)b * M + k] = 1;
      } else {
        qout[atomicAdd(nout, 1)] = make_int2(b, (int)k);
      }
    }
    __syncwarp();
  }
}

unsigned wide_grid(int64_t maxq, int nsm) {
  return (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((maxq + kWideWarps - 1) / kWideWarps, (int64_t)nsm * 16));
}

template <class F, int A>
void level_wide_a(sft_plan_s* P, const LevelArgs& g, int2* q, int* c, dim3 fgrid, unsigned wg,
                  cudaStream_t st, const char* fold_name, const char* dec_name) {
  stage_begin(P, fold_name, st);
  k_iter_fold<F, A><<<fgrid, kFoldThreads, 0, st>>>(g, q, c, 0);
  stage_end(P, st);
  stage_begin(P, dec_name, st);
  k_iter_decode_wide<F, A><<<wg, 32 * kWideWarps, 0, st>>>(g, q, c);
  stage_end(P, st);
}

template <class F>
void level_wide_t(sft_plan_s* P, int A, const LevelArgs& g, int2* q, int* c, dim3 fgrid,
                  unsigned wg, cudaStream_t st, const char* fn, const char* dn) {
  switch (A) {
    case 5: level_wide_a<F, 5>(P, g, q, c, fgrid, wg, st, fn, dn); break;
    case 6: level_wide_a<F, 6>(P, g, q, c, fgrid, wg, st, fn, dn); break;
    case 7: level_wide_a<F, 7>(P, g, q, c, fgrid, wg, st, fn, dn); break;
    default: level_wide_a<F, 8>(P, g, q, c, fgrid, wg, st, fn, dn); break;
  }
}

template <class F>
void fixed_rounds_t(const FixedArgs& g, int2* q0, int2* q1, int* c, dim3 sgrid, unsigned dgrid,
                    unsigned wgrid, sft_plan_s* P, cudaStream_t st) {
  static const char* rnames[] = {"decode_fixed_a1", "decode_fixed_a2", "decode_fixed_a3",
                                 "decode_fixed_a4", "decode_fixed_a5", "decode_fixed_a6",
                                 "decode_fixed_a7", "decode_fixed_a8"};
  const int am = g.a_max;
  stage_begin(P, "decode_fixed_scan", st);
  k_fixed_scan<F, 16><<<sgrid, kFoldThreads, 0, st>>>(g, q0, c);
  stage_end(P, st);
  // round a reads queue (a-1)&1 / counter a-1, writes queue a&1 / counter a
  auto in_q = [&](int a) { return (a & 1) ? q0 : q1; };
  auto out_q = [&](int a) { return a == am ? nullptr : ((a & 1) ? q1 : q0); };
  auto out_c = [&](int a) { return a == am ? nullptr : c + a; };
  stage_begin(P, rnames[0], st);
  k_fixed_round<F, 1, 16><<<dgrid, kDecThreads, 0, st>>>(g, in_q(1), c, out_q(1), out_c(1));
  stage_end(P, st);
  stage_begin(P, rnames[1], st);
  k_fixed_round<F, 2, 16><<<dgrid, kDecThreads, 0, st>>>(g, in_q(2), c + 1, out_q(2), out_c(2));
  stage_end(P, st);
  stage_begin(P, rnames[2], st);
  k_fixed_round<F, 3, 16><<<dgrid, kDecThreads, 0, st>>>(g, in_q(3), c + 2, out_q(3), out_c(3));
  stage_end(P, st);
  stage_begin(P, rnames[3], st);
  k_fixed_round<F, 4, 16><<<dgrid, kDecThreads, 0, st>>>(g, in_q(4), c + 3, out_q(4), out_c(4));
  stage_end(P, st);
  const unsigned T = 32 * kWideWarps;
  stage_begin(P, rnames[4], st);
  k_fixed_round_wide<F, 5><<<wgrid, T, 0, st>>>(g, in_q(5), c + 4, out_q(5), out_c(5));
  stage_end(P, st);
  stage_begin(P, rnames[5], st);
  k_fixed_round_wide<F, 6><<<wgrid, T, 0, st>>>(g, in_q(6), c + 5, out_q(6), out_c(6));
  stage_end(P, st);
  stage_begin(P, rnames[6], st);
  k_fixed_round_wide<F, 7><<<wgrid, T, 0, st>>>(g, in_q(7), c + 6, out_q(7), out_c(7));
  stage_end(P, st);
  stage_begin(P, rnames[7], st);
  k_fixed_round_wide<F, 8><<<wgrid, T, 0, st>>>(g, in_q(8), c + 7, out_q(8), out_c(8));
  stage_end(P, st);
}

}  // namespace

void launch_level_wide(sft_plan_s* P, int A, const LevelArgs& g, int2* q, int* c, dim3 fgrid,
                       int64_t maxq, int nsm, cudaStream_t st, const char* fold_name,
                       const char* dec_name) {
  const unsigned wg = wide_grid(maxq, nsm);
  if (P->p.precision == SFT_FP64)
    level_wide_t<F64>(P, A, g, q, c, fgrid, wg, st, fold_name, dec_name);
  else
    level_wide_t<FF>(P, A, g, q, c, fgrid, wg, st, fold_name, dec_name);
}

void launch_fixed_wide(sft_plan_s* P, int64_t B, const FixedArgs& g, int nsm, cudaStream_t st) {
  const Workspace& W = P->ws;
  dim3 sgrid((unsigned)((P->M0 + kFoldThreads - 1) / kFoldThreads), (unsigned)B);
  const int64_t maxq = B * P->M0;
  const unsigned dgrid = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((maxq + kDecThreads - 1) / kDecThreads,
                           (int64_t)P->dec_ctas_per_sm * nsm));
  if (P->p.precision == SFT_FP64)
    fixed_rounds_t<F64>(g, W.queue[0], W.queue[1], W.qcount, sgrid, dgrid, wide_grid(maxq, nsm),
                        P, st);
  else
    fixed_rounds_t<FF>(g, W.queue[0], W.queue[1], W.qcount, sgrid, dgrid, wide_grid(maxq, nsm), P,
                       st);
}

}  // namespace sft
