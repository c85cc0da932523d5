// sft_decode.cuh -- per-bin syndrome decoding in FP64 (Sec. II-B, the SynDec
// function of Algorithm 1), run by one thread per bin.
//
// Given n_m >= 2a syndromes m_i = sum_j p_j z_j^i of bin k (Eq. (3)):
//  (i)   solve the a x a Hankel system sum_j c_j m_{i+j} = -m_{a+i}
//        (Eq. (4)-(5)) by Gaussian elimination with partial pivoting;
//  (ii)  take the roots of P(z) = z^a + c_{a-1} z^{a-1} + ... + c_0 by the
//        analytical solutions for a <= 4 (quadratic, Cardano, Ferrari);
//        each root gives the location s_j = ln(z_j) N / (i 2 pi), taken as
//        the member k + tM of S_k nearest to it (Alg. 1 lines 29-30);
//  (iii) solve all n_m equations of Eq. (3) for the values p_j in the least
//        squares sense (normal equations).
// Accept iff every root lies within root_tol of omega^{s_j}, the s_j are
// distinct, every |p_j| > theta and ||m - Z p||_inf <= res_tol ||m||_inf.
#pragma once

#include "sft_common.cuh"

namespace sft {

// Gaussian elimination with partial pivoting on an n x n system (n <= 4).
// A is row-major and destroyed.  Fails on a pivot below 1e-14 of max |A|.
template <int n>
__device__ __forceinline__ bool solve_small(cdbl* A, cdbl* b, cdbl* x) {
  double amax2 = 0.0;
#pragma unroll
  for (int i = 0; i < n * n; ++i) amax2 = fmax(amax2, norm2(A[i]));
  if (!(amax2 > 0.0)) return false;
#pragma unroll
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = norm2(A[col * n + col]);
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      double v = norm2(A[r * n + col]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (!(best > 1e-28 * amax2)) return false;
    // swap rows col and piv (predicated moves keep the indexing static)
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      if (r == piv) {
#pragma unroll
        for (int c = 0; c < n; ++c) {
          cdbl t = A[col * n + c];
          A[col * n + c] = A[r * n + c];
          A[r * n + c] = t;
        }
        cdbl t = b[col];
        b[col] = b[r];
        b[r] = t;
      }
    }
    const cdbl dv = A[col * n + col];
#pragma unroll
    for (int r = col + 1; r < n; ++r) {
      cdbl f = cdivd(A[r * n + col], dv);
#pragma unroll
      for (int c = col; c < n; ++c) A[r * n + c] = A[r * n + c] - f * A[col * n + c];
      b[r] = b[r] - f * b[col];
    }
  }
#pragma unroll
  for (int r = n - 1; r >= 0; --r) {
    cdbl acc = b[r];
#pragma unroll
    for (int c = r + 1; c < n; ++c) acc = acc - A[r * n + c] * x[c];
    x[r] = cdivd(acc, A[r * n + r]);
  }
  return true;
}

// z^2 + b z + c = 0 in the cancellation-free form q = -(b + sgn sqrt(D))/2,
// roots q and c/q.
__device__ __forceinline__ void quad_roots(cdbl b, cdbl c, cdbl* z) {
  cdbl sq = csqrtd(b * b - c * 4.0);
  cdbl qp = b + sq, qm = b - sq;
  cdbl q = (norm2(qp) >= norm2(qm) ? qp : qm) * -0.5;
  if (q.x == 0.0 && q.y == 0.0) {
    z[0] = z[1] = mk(0.0, 0.0);
    return;
  }
  z[0] = q;
  z[1] = cdivd(c, q);
}

// z^3 + c2 z^2 + c1 z + c0 = 0: shift z = y - c2/3 to y^3 + p y + q = 0;
// y = u + v, u^3 = -q/2 +- sqrt((q/2)^2 + (p/3)^3) (the larger), u v = -p/3,
// u over its three cube-root branches.
__device__ __forceinline__ void cubic_roots(cdbl c2, cdbl c1, cdbl c0, cdbl* z) {
  const cdbl sh = c2 * (1.0 / 3.0);
  const cdbl p = c1 - c2 * c2 * (1.0 / 3.0);
  const cdbl q = c2 * c2 * c2 * (2.0 / 27.0) - c2 * c1 * (1.0 / 3.0) + c0;
  const cdbl sD = csqrtd(q * q * 0.25 + p * p * p * (1.0 / 27.0));
  const cdbl w1 = q * -0.5 + sD, w2 = q * -0.5 - sD;
  const cdbl u = ccbrtd(norm2(w1) >= norm2(w2) ? w1 : w2);
  const cdbl br[3] = {mk(1.0, 0.0), mk(-0.5, 0.86602540378443864676), mk(-0.5, -0.86602540378443864676)};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    cdbl uj = u * br[j];
    cdbl vj = (uj.x == 0.0 && uj.y == 0.0) ? mk(0.0, 0.0) : cdivd(-p, uj * 3.0);
    z[j] = uj + vj - sh;
  }
}

// z^4 + c3 z^3 + c2 z^2 + c1 z + c0 = 0: shift z = y - c3/4 to
// y^4 + p y^2 + q y + r; m = largest root of 8m^3 + 8p m^2 + (2p^2 - 8r) m - q^2;
// with s^2 = 2m the quartic splits into y^2 -+ s y + p/2 + m +- q/(2s).
__device__ __forceinline__ void quartic_roots(cdbl c3, cdbl c2, cdbl c1, cdbl c0, cdbl* z) {
  const cdbl sh = c3 * 0.25;
  const cdbl c3s = c3 * c3;
  const cdbl p = c2 - c3s * (3.0 / 8.0);
  const cdbl q = c3s * c3 * (1.0 / 8.0) - c3 * c2 * 0.5 + c1;
  const cdbl r = c3s * c3s * (-3.0 / 256.0) + c3s * c2 * (1.0 / 16.0) - c3 * c1 * 0.25 + c0;
  cdbl mr[3];
  cubic_roots(p, (p * p * 2.0 - r * 8.0) * (1.0 / 8.0), q * q * (-1.0 / 8.0), mr);
  int best = 0;
  if (norm2(mr[1]) > norm2(mr[best])) best = 1;
  if (norm2(mr[2]) > norm2(mr[best])) best = 2;
  const cdbl m = mr[best];
  cdbl y[4];
  if (m.x == 0.0 && m.y == 0.0) {
    cdbl w[2];
    quad_roots(p, r, w);
    y[0] = csqrtd(w[0]);
    y[1] = -y[0];
    y[2] = csqrtd(w[1]);
    y[3] = -y[2];
  } else {
    const cdbl s = csqrtd(m * 2.0);
    const cdbl qs = cdivd(q, s * 2.0);
    quad_roots(-s, p * 0.5 + m + qs, y);
    quad_roots(s, p * 0.5 + m - qs, y + 2);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = y[j] - sh;
}

struct BinGeom {
  int64_t N, M, d;  // signal length, bins at this level, N / M
  OmegaTab om;
};

struct Tol {
  double theta, root_tol, res_tol;
};

// Decode bin k with `a` aliases from m[0..nm).  On success fills s[0..a)
// (ascending), p[0..a) and returns true.
template <int a>
__device__ __forceinline__ bool decode_bin(const cdbl* m, int nm, int64_t k, const BinGeom& g,
                                           const Tol& tol, int64_t* s, cdbl* p) {
  cdbl H[a * a], rhs[a], c[a];
#pragma unroll
  for (int i = 0; i < a; ++i) {
#pragma unroll
    for (int j = 0; j < a; ++j) H[i * a + j] = m[i + j];
    rhs[i] = -m[a + i];
  }
  if (!solve_small<a>(H, rhs, c)) return false;

  cdbl z[4];
  if constexpr (a == 1) {
    z[0] = -c[0];
  } else if constexpr (a == 2) {
    quad_roots(c[1], c[0], z);
  } else if constexpr (a == 3) {
    cubic_roots(c[2], c[1], c[0], z);
  } else {
    quartic_roots(c[3], c[2], c[1], c[0], z);
  }

  const double inv2pi = 0.15915494309189533577;  // 1 / (2 pi)
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < a) {
      if (!(isfinite(z[j].x) && isfinite(z[j].y)) || (z[j].x == 0.0 && z[j].y == 0.0)) return false;
      const double pos = atan2(z[j].y, z[j].x) * inv2pi * (double)g.N;
      const double tf = rint((pos - (double)k) / (double)g.M);
      int64_t t = ((int64_t)tf) % g.d;
      if (t < 0) t += g.d;
      s[j] = k + t * g.M;
      const cdbl w = omega_pow(g.om, s[j]);
      if (!(absd(z[j] - w) <= tol.root_tol)) return false;
    }
  }
  // ascending (4-input sorting network; unused slots sort last), distinct
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j >= a) s[j] = INT64_MAX;
  auto cswap = [](int64_t& u, int64_t& v) {
    if (u > v) {
      int64_t t = u;
      u = v;
      v = t;
    }
  };
  cswap(s[0], s[1]);
  cswap(s[2], s[3]);
  cswap(s[0], s[2]);
  cswap(s[1], s[3]);
  cswap(s[1], s[2]);
#pragma unroll
  for (int j = 1; j < 4; ++j)
    if (j < a && s[j] == s[j - 1]) return false;

  // normal equations (Z^H Z) p = Z^H m over all nm equations, Z_ij = omega^{s_j i}
  cdbl G[16], gr[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    gr[u] = mk(0.0, 0.0);
#pragma unroll
    for (int v = 0; v < 4; ++v) G[u * 4 + v] = mk(0.0, 0.0);
  }
  for (int i = 0; i < nm; ++i) {
    cdbl zi[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < a) zi[j] = omega_pow(g.om, s[j] * (int64_t)i);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (u < a) {
        gr[u] = gr[u] + conjd(zi[u]) * m[i];
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (v < a) G[u * 4 + v] = G[u * 4 + v] + conjd(zi[u]) * zi[v];
      }
    }
  }
  cdbl Gs[a * a];
#pragma unroll
  for (int u = 0; u < a; ++u)
#pragma unroll
    for (int v = 0; v < a; ++v) Gs[u * a + v] = G[u * 4 + v];
  if (!solve_small<a>(Gs, gr, p)) return false;

#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (j < a && !(absd(p[j]) > tol.theta)) return false;
  double mmax = 0.0, rmax = 0.0;
  for (int i = 0; i < nm; ++i) {
    cdbl fit = mk(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < a) fit = fit + p[j] * omega_pow(g.om, s[j] * (int64_t)i);
    mmax = fmax(mmax, absd(m[i]));
    rmax = fmax(rmax, absd(m[i] - fit));
  }
  return rmax <= tol.res_tol * mmax;
}

}  // namespace sft
