// sft_quad.cuh -- SynDec of one bin with a = 3 or 4 aliases (Sec. II-B
// steps (i)-(iii)) on a group of four lanes, eight bins per warp.
//
// The one-lane decoder (decode_bin) walks a serial chain of about 1 700 FP64
// instructions per bin at a = 4.  An FP64 warp instruction occupies its SM
// sub-partition for the same time whatever the number of active lanes, so
// the chain, not the number of bins, sets the time of the last levels.  Here
// the four lanes of a group share one bin:
//   (i)   the Hankel solve for the locator c by row-per-lane elimination
//         (the arithmetic of solve_small: the pivot search, the row exchange
//         and the pivot row's broadcast done by shuffles), the roots of the
//         locator on every lane;
//   (ii)  one root per lane: its snap to S_k and the root_tol test;
//   (iii) the Gram matrix Z^H Z (one or two of its off-diagonal sums per
//         lane) and Z^H m (one entry per lane), the normal equations by
//         row-per-lane elimination, and the validation residual with each
//         lane taking every fourth equation.
// Decisions are taken on the group's reduced values, so all four lanes
// follow the same path and every shuffle names exactly the group's lanes.
#pragma once

#include "sft_decode.cuh"

namespace sft {

struct Quad {
  unsigned mask;  // the group's four lanes
  int q;          // this lane's place in the group (0..3)
  __device__ __forceinline__ double sh(double v, int src) const {
    return __shfl_sync(mask, v, src, 4);
  }
  __device__ __forceinline__ cdbl sh(cdbl v, int src) const { return cdbl{sh(v.x, src), sh(v.y, src)}; }
  __device__ __forceinline__ int64_t sh(int64_t v, int src) const {
    return (int64_t)__shfl_sync(mask, (long long)v, src, 4);
  }
  __device__ __forceinline__ double max4(double v) const {
    v = fmax(v, __shfl_xor_sync(mask, v, 1, 4));
    return fmax(v, __shfl_xor_sync(mask, v, 2, 4));
  }
  __device__ __forceinline__ float max4(float v) const {
    v = fmaxf(v, __shfl_xor_sync(mask, v, 1, 4));
    return fmaxf(v, __shfl_xor_sync(mask, v, 2, 4));
  }
  __device__ __forceinline__ bool all4(bool p) const {
    return (__ballot_sync(mask, p) & mask) == mask;
  }
  // the first lane of the group (0..3) with p, or -1
  __device__ __forceinline__ int first4(bool p) const {
    const unsigned b = __ballot_sync(mask, p) & mask;
    return b != 0u ? ((__ffs((int)b) - 1) & 3) : -1;
  }
};

// v[q] for a lane-dependent q in 0..3 from statically indexed values
template <class V>
__device__ __forceinline__ V pick4(int q, const V& v0, const V& v1, const V& v2, const V& v3) {
  return q == 0 ? v0 : (q == 1 ? v1 : (q == 2 ? v2 : v3));
}

// Gaussian elimination with partial pivoting on an n x n system, lane q of
// the group holding row q of A (Ar) and of b (br); lanes q >= n hold
// nothing.  Pivot choice (the first row of largest |A_rc|^2), the failure
// rule (a pivot below 1e-14 of max |A|) and the elimination arithmetic are
// those of solve_small; the back substitution accumulates the known
// unknowns as they arrive (last first).  Returns false on every lane where
// solve_small fails; on success every lane holds x[0..n).
template <int n>
__device__ __forceinline__ bool solve_rows(const Quad& G, cdbl* Ar, cdbl br, cdbl* x) {
  const int q = G.q;
  const bool mine = q < n;
  double am = 0.0;
  if (mine) {
#pragma unroll
    for (int c = 0; c < n; ++c) am = fmax(am, norm2(Ar[c]));
  }
  const double amax2 = G.max4(am);
  if (!(amax2 > 0.0)) return false;
  cdbl inv_mine = mk(0.0, 0.0);
#pragma unroll
  for (int col = 0; col < n; ++col) {
    const bool cand = mine && q >= col;
    const double v = cand ? norm2(Ar[col]) : -1.0;
    const double best = G.max4(v);
    const int piv = G.first4(cand && v == best);
    if (piv < 0 || !(best > 1e-28 * amax2)) return false;
    // exchange rows col and piv (columns before col are not read again)
    const int src = q == col ? piv : (q == piv ? col : q);
#pragma unroll
    for (int c = col; c < n; ++c) Ar[c] = G.sh(Ar[c], src);
    br = G.sh(br, src);
    cdbl P[n];
#pragma unroll
    for (int c = col; c < n; ++c) P[c] = G.sh(Ar[c], col);
    const cdbl Pb = G.sh(br, col);
    const cdbl inv = crcp(P[col]);
    if (q == col) inv_mine = inv;
    if (mine && q > col) {
      const cdbl f = Ar[col] * inv;
#pragma unroll
      for (int c = col + 1; c < n; ++c) Ar[c] = Ar[c] - f * P[c];
      br = br - f * Pb;
    }
  }
  cdbl acc = br;
#pragma unroll
  for (int r = n - 1; r >= 0; --r) {
    const cdbl xr = G.sh(acc * inv_mine, r);
    x[r] = xr;
    if (mine && q < r) acc = acc - Ar[r] * xr;
  }
  return true;
}

// the off-diagonal Gram entries (u, v), u < v, in the order
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) for a = 4 and (0,1) (0,2) (1,2) for
// a = 3; entry e is summed by lane e mod 4
template <int a>
struct GramPairs {
  static constexpr int n = a * (a - 1) / 2;
  __device__ static constexpr int u(int e) {
    return a == 4 ? (e < 3 ? 0 : (e < 5 ? 1 : 2)) : (e < 2 ? 0 : 1);
  }
  __device__ static constexpr int v(int e) {
    return a == 4 ? (e < 3 ? e + 1 : (e < 5 ? e - 1 : 3)) : (e < 2 ? e + 1 : 2);
  }
  // index of the pair (u, v), u < v
  __device__ static constexpr int index(int uu, int vv) {
    return a == 4 ? (uu == 0 ? vv - 1 : (uu == 1 ? vv + 1 : 5)) : (uu == 0 ? vv - 1 : 2);
  }
};

// sum_{i < nm} (conj(wu) wv)^i, as the one-lane decoder forms it
template <int nm>
__device__ __forceinline__ cdbl geo_sum(cdbl wu, cdbl wv) {
  const cdbl qv = conjd(wu) * wv;
  cdbl acc = mk(1.0, 0.0), qp = qv;
#pragma unroll
  for (int i = 1; i < nm; ++i) {
    acc = acc + qp;
    if (i + 1 < nm) qp = qp * qv;
  }
  return acc;
}

// SynDec with a in {3, 4} aliases of bin k from the float-float syndromes
// Y[i M + k], i < nm.  On success (true on every lane) s[0..a) ascending and
// p[0..a) are on every lane and, when `out` is not null, the residual
// m - Z p is written to out[i M + k]; on failure nothing is written.
template <int a, int nm>
__device__ __forceinline__ bool decode_quad(const Quad& G, const float4* Y, float4* out, int64_t M,
                                            int64_t k, const BinGeom& g, const Tol2& tol,
                                            const OmegaTabFF& omff, int64_t* s, cdbl* p) {
  static_assert(a == 3 || a == 4, "four-lane decoder for three or four aliases");
  static_assert(nm >= 2 * a && nm <= 8, "2a <= nm <= 8 syndromes");
  const int q = G.q;
  cdbl m[nm];
#pragma unroll
  for (int i = 0; i < nm; ++i) m[i] = Store<FF>::to_d(Y[(int64_t)i * M + k]);

  // (i) locator: H c = -m_{a..2a-1}, H_ij = m_{i+j}, row q on lane q
  const int qr = q < a ? q : a - 1;
  cdbl Ar[a];
#pragma unroll
  for (int c = 0; c < a; ++c) Ar[c] = pick4(qr, m[c], m[c + 1], m[c + 2], m[(c + 3) % nm]);
  const cdbl br = -pick4(qr, m[a], m[a + 1], m[a + 2], m[(a + 3) % nm]);
  cdbl c[a];
  if (!solve_rows<a>(G, Ar, br, c)) return false;
  cdbl z[4];
  if constexpr (a == 3)
    cubic_roots(c[2], c[1], c[0], z);
  else
    quartic_roots(c[3], c[2], c[1], c[0], z);

  // (ii) root q on lane q: snap to S_k, root_tol
  int64_t s_mine = 0;
  cdbl w_mine = mk(1.0, 0.0);
  bool ok = true;
  if (q < a) {
    const cdbl zq = pick4(q, z[0], z[1], z[2], z[3]);
    if (!(isfinite(zq.x) && isfinite(zq.y)) || (zq.x == 0.0 && zq.y == 0.0)) {
      ok = false;
    } else {
      s_mine = snap_root(zq, k, g);
      w_mine = omega_pow(g.om, s_mine);
      ok = norm2(zq - w_mine) <= tol.root2;
    }
  }
  if (!G.all4(ok)) return false;
  cdbl w[a];
#pragma unroll
  for (int j = 0; j < a; ++j) {
    s[j] = G.sh(s_mine, j);
    w[j] = G.sh(w_mine, j);
  }
  // ascending locations (the one-lane decoder's sorting network), distinct
  auto cswap = [&](int u, int v) {
    if (s[u] > s[v]) {
      const int64_t ts = s[u];
      s[u] = s[v];
      s[v] = ts;
      const cdbl tw = w[u];
      w[u] = w[v];
      w[v] = tw;
    }
  };
  if constexpr (a == 3) {
    cswap(0, 1);
    cswap(1, 2);
    cswap(0, 1);
  } else {
    cswap(0, 1);
    cswap(2, 3);
    cswap(0, 2);
    cswap(1, 3);
    cswap(1, 2);
  }
#pragma unroll
  for (int j = 1; j < a; ++j)
    if (s[j] == s[j - 1]) return false;

  // (iii) normal equations (Z^H Z) p = Z^H m, Z_ij = w_j^i
  typedef GramPairs<a> GP;
  constexpr int kPer = (GP::n + 3) / 4;
  cdbl pv[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int e = q + 4 * t;
    pv[t] = mk(0.0, 0.0);
    if (e < GP::n) {
      // the pair (u, v) of entry e, picked from the statically known pairs
      cdbl wu = w[0], wv = w[1];
#pragma unroll
      for (int f = 0; f < GP::n; ++f)
        if (f == e) {
          wu = w[GP::u(f)];
          wv = w[GP::v(f)];
        }
      pv[t] = geo_sum<nm>(wu, wv);
    }
  }
  cdbl pall[GP::n];
#pragma unroll
  for (int f = 0; f < GP::n; ++f) pall[f] = G.sh(pv[f / 4], f % 4);
  // row qr of Z^H Z: nm on the diagonal, the pair sums above, conjugates below
  cdbl Gr[a];
#pragma unroll
  for (int cc = 0; cc < a; ++cc) {
    cdbl r4[4];
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      if (rr >= a || rr == cc)
        r4[rr] = mk((double)nm, 0.0);
      else if (rr < cc)
        r4[rr] = pall[GP::index(rr, cc)];
      else
        r4[rr] = conjd(pall[GP::index(cc, rr)]);
    }
    Gr[cc] = pick4(qr, r4[0], r4[1], r4[2], r4[3]);
  }
  // entry qr of Z^H m
  const cdbl wq = pick4(qr, w[0], w[1], w[2 < a ? 2 : 0], w[3 < a ? 3 : 0]);
  cdbl gr = m[0], wp = wq;
#pragma unroll
  for (int i = 1; i < nm; ++i) {
    gr = gr + conjd(wp) * m[i];
    if (i + 1 < nm) wp = wp * wq;
  }
  if (!solve_rows<a>(G, Gr, gr, p)) return false;
#pragma unroll
  for (int j = 0; j < a; ++j)
    if (!(norm2(p[j]) > tol.theta2)) return false;

  // validation (iii): residual r_i = m_i - sum_j p_j w_j^i, equations
  // i = q, q + 4 on lane q, in float-float (FP64 when the float range is left)
  constexpr int kEq = (nm + 3) / 4;
  FF::V pf[a];
#pragma unroll
  for (int j = 0; j < a; ++j) pf[j] = FF::from4(Store<FF>::from_d(p[j]));
  FF::V r[kEq];
  float mm = 0.0f, rm = 0.0f;
#pragma unroll
  for (int t = 0; t < kEq; ++t) {
    const int i = q + 4 * t;
    r[t] = FF::V{0.0f, 0.0f, 0.0f, 0.0f};
    if (i < nm) {
      const FF::V mi = FF::from4(Y[(int64_t)i * M + k]);
      FF::V fit = FF::mulv(pf[0], omega_ff(omff, s[0] * i));
#pragma unroll
      for (int j = 1; j < a; ++j) fit = FF::add(fit, FF::mulv(pf[j], omega_ff(omff, s[j] * i)));
      r[t] = FF::sub(mi, fit);
      const float mx = __fadd_rn(mi.rh, mi.rl), my = __fadd_rn(mi.ih, mi.il);
      const float rx = __fadd_rn(r[t].rh, r[t].rl), ry = __fadd_rn(r[t].ih, r[t].il);
      mm = fmaxf(mm, mx * mx + my * my);
      rm = fmaxf(rm, rx * rx + ry * ry);
    }
  }
  const float mmax2 = G.max4(mm), rmax2 = G.max4(rm);
  if (mmax2 < 1e36f && rmax2 < 1e36f) {
    if (!((double)rmax2 <= tol.res2 * (double)mmax2)) return false;
    if (out != nullptr) {
#pragma unroll
      for (int t = 0; t < kEq; ++t) {
        const int i = q + 4 * t;
        if (i < nm) out[(int64_t)i * M + k] = FF::to4(r[t]);
      }
    }
    return true;
  }
  // FP64 residual
  cdbl rd[kEq];
  double md = 0.0, rdm = 0.0;
#pragma unroll
  for (int t = 0; t < kEq; ++t) {
    const int i = q + 4 * t;
    rd[t] = mk(0.0, 0.0);
    if (i < nm) {
      const cdbl mi = Store<FF>::to_d(Y[(int64_t)i * M + k]);
      cdbl fit = mk(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < a; ++j) fit = fit + p[j] * omega_pow(g.om, s[j] * i);
      rd[t] = mi - fit;
      md = fmax(md, norm2(mi));
      rdm = fmax(rdm, norm2(rd[t]));
    }
  }
  const double mmax2d = G.max4(md), rmax2d = G.max4(rdm);
  if (!(rmax2d <= tol.res2 * mmax2d)) return false;
  if (out != nullptr) {
#pragma unroll
    for (int t = 0; t < kEq; ++t) {
      const int i = q + 4 * t;
      if (i < nm) out[(int64_t)i * M + k] = Store<FF>::from_d_small(rd[t]);
    }
  }
  return true;
}

}  // namespace sft
