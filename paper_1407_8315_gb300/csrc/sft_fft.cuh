// sft_fft.cuh -- CTA-wide FFT of one length-M sequence held in shared memory.
//
// Stockham autosort formulation, forward (e^{-2 pi i k n / M}), natural order
// in and out.  M = 2^m is factored into radix-16 passes plus one radix-2/4/8
// pass.  In every pass each thread loads its R inputs (stride M/R) into
// registers, applies the inter-pass twiddles, runs an R-point DFT in
// registers (radix-2 decimation in frequency, constant twiddles), and stores
// the R outputs.  All loads of a pass complete before any store (barrier),
// so one M-point buffer suffices.
//
// Pass with radix R after sub-transforms of length Ns (Ns = product of the
// earlier radices): group j (0 <= j < M/R), kk = j mod Ns,
//   v[r] = buf[j + r M/R] * e^{-2 pi i r kk / (Ns R)}
//   V    = DFT_R(v)
//   buf[(j - kk) R + kk + r Ns] = V[r]
// The inter-pass twiddles come from a table of e^{-2 pi i q / Mt} (Mt >= M,
// Mt a power of two), indexed at q = r kk (Mt / (Ns R)).
#pragma once

#include "sft_common.cuh"

namespace sft {

// In-register DFT of R = 2, 4, 8 or 16 points: radix-2 DIF stages, then the
// bit-reversal permutation (compile-time register renaming).
template <class F, int R>
__device__ __forceinline__ void dft_reg(typename F::V* v) {
#pragma unroll
  for (int h = R / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int blk = 0; blk < R; blk += 2 * h) {
#pragma unroll
      for (int j = 0; j < h; ++j) {
        typename F::V a = v[blk + j], b = v[blk + j + h];
        v[blk + j] = F::add(a, b);
        typename F::V t = F::sub(a, b);
        const int m = j * (8 / h);  // e^{-2 pi i j / (2h)} = e^{-2 pi i m / 16}
        if (m == 0) {
          v[blk + j + h] = t;
        } else if (m == 4) {
          v[blk + j + h] = F::mul_mi(t);
        } else {
          v[blk + j + h] = F::mul_c16(t, m);
        }
      }
    }
  }
  // bit reversal of the R outputs
  constexpr int LOG = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < LOG; ++b) r |= ((i >> b) & 1) << (LOG - 1 - b);
    if (r > i) {
      typename F::V t = v[i];
      v[i] = v[r];
      v[r] = t;
    }
  }
}

// One Stockham pass of radix R over buf[0..M).  Each thread owns up to
// G = PTS / R groups (group j = tid + g * nthr): PTS points per thread.
template <class F, int R, int PTS = 16>
__device__ __forceinline__ void stockham_pass(char* buf, int M, int Ns, int log2Mt,
                                              const typename F::Tw* __restrict__ tw, int tid,
                                              int nthr) {
  constexpr int G = PTS / R;
  const int groups = M / R;
  typename F::V v[G][R];
  const int twstep_log = log2Mt - (31 - __clz(Ns * R));  // log2(Mt / (Ns R))
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tid + g * nthr;
    if (j < groups) {
      const int kk = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        v[g][r] = F::ld(buf, M, j + r * groups);
        if (r > 0 && Ns > 1) v[g][r] = F::mul_tw(v[g][r], __ldg(tw + ((r * kk) << twstep_log)));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tid + g * nthr;
    if (j < groups) {
      const int kk = j & (Ns - 1);
      dft_reg<F, R>(v[g]);
      const int base = (j - kk) * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) F::st(buf, M, base + r * Ns, v[g][r]);
    }
  }
  __syncthreads();
}

// The last Stockham pass with its outputs handed to out(index, value)
// instead of stored back: the transform's result goes straight to its
// destination (one shared-memory round trip and two barriers fewer).
// Every value is computed exactly as by stockham_pass.
template <class F, int R, int PTS, class Out>
__device__ __forceinline__ void stockham_pass_out(char* buf, int M, int Ns, int log2Mt,
                                                  const typename F::Tw* __restrict__ tw, int tid,
                                                  int nthr, Out&& out) {
  constexpr int G = PTS / R;
  const int groups = M / R;
  const int twstep_log = log2Mt - (31 - __clz(Ns * R));
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tid + g * nthr;
    if (j < groups) {
      const int kk = j & (Ns - 1);
      typename F::V v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        v[r] = F::ld(buf, M, j + r * groups);
        if (r > 0 && Ns > 1) v[r] = F::mul_tw(v[r], __ldg(tw + ((r * kk) << twstep_log)));
      }
      dft_reg<F, R>(v);
      const int base = (j - kk) * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) out(base + r * Ns, v[r]);
    }
  }
}

// stockham_pass whose stores go through st(index, value) (which must store
// into buf, e.g. after a per-point multiply): loads, barrier, st, barrier.
template <class F, int R, int PTS, class St>
__device__ __forceinline__ void stockham_pass_st(char* buf, int M, int Ns, int log2Mt,
                                                 const typename F::Tw* __restrict__ tw, int tid,
                                                 int nthr, St&& st) {
  constexpr int G = PTS / R;
  const int groups = M / R;
  typename F::V v[G][R];
  const int twstep_log = log2Mt - (31 - __clz(Ns * R));
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tid + g * nthr;
    if (j < groups) {
      const int kk = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        v[g][r] = F::ld(buf, M, j + r * groups);
        if (r > 0 && Ns > 1) v[g][r] = F::mul_tw(v[g][r], __ldg(tw + ((r * kk) << twstep_log)));
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int j = tid + g * nthr;
    if (j < groups) {
      const int kk = j & (Ns - 1);
      dft_reg<F, R>(v[g]);
      const int base = (j - kk) * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) st(base + r * Ns, v[g][r]);
    }
  }
  __syncthreads();
}

// The first radix-PTS pass (Ns = 1: no inter-pass twiddles) straight from
// registers: with nthr = M / PTS, the inputs of thread tid's group are the
// samples tid + r nthr, r < PTS, which are exactly the ones it gathered, so
// they need not round-trip through shared memory.  Stores the pass's
// outputs; the caller synchronises and continues with cta_fft from Ns = PTS.
template <class F, int PTS>
__device__ __forceinline__ void first_pass_regs(char* buf, int M, const typename F::In* in,
                                                int tid) {
  typename F::V v[PTS];
#pragma unroll
  for (int r = 0; r < PTS; ++r) v[r] = F::from_in(in[r]);
  dft_reg<F, PTS>(v);
#pragma unroll
  for (int r = 0; r < PTS; ++r) F::st(buf, M, tid * PTS + r, v[r]);
}

// Forward FFT of buf[0..M), M = 2^log2M (1 <= log2M <= 13 here), executed by
// nthr threads holding PTS = 16 or 8 points each (nthr * PTS >= M): radix-PTS
// passes and one radix-2/4/8 pass for the remaining factor, starting after
// the first `done` radix-PTS passes (0, or 1 after first_pass_regs).  Caller
// synchronises before the call.
template <class F, int PTS = 16>
__device__ void cta_fft(char* buf, int log2M, int log2Mt, const typename F::Tw* __restrict__ tw,
                        int tid, int nthr, int done = 0) {
  static_assert(PTS == 16 || PTS == 8, "16 or 8 points per thread");
  constexpr int LP = PTS == 16 ? 4 : 3;
  const int M = 1 << log2M;
  int Ns = 1 << (LP * done);
  int rem = log2M - LP * done;
  while (rem >= LP) {
    stockham_pass<F, PTS, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
    Ns <<= LP;
    rem -= LP;
  }
  if constexpr (PTS == 16) {
    if (rem == 3) stockham_pass<F, 8, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
  }
  if (rem == 2) stockham_pass<F, 4, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
  if (rem == 1) stockham_pass<F, 2, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
}

// cta_fft whose last pass stores through st(index, value) (into buf); false,
// having run no pass, when no pass is left after the first `done`.
template <class F, int PTS, class St>
__device__ bool cta_fft_st(char* buf, int log2M, int log2Mt, const typename F::Tw* __restrict__ tw,
                           int tid, int nthr, int done, St&& st) {
  static_assert(PTS == 16 || PTS == 8, "16 or 8 points per thread");
  constexpr int LP = PTS == 16 ? 4 : 3;
  const int M = 1 << log2M;
  int Ns = 1 << (LP * done);
  int rem = log2M - LP * done;
  if (rem <= 0) return false;
  while (rem > LP) {
    stockham_pass<F, PTS, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
    Ns <<= LP;
    rem -= LP;
  }
  if (rem == LP) {
    if constexpr (PTS == 16)
      stockham_pass_st<F, 16, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, st);
    else
      stockham_pass_st<F, 8, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, st);
  } else if (rem == 3) {
    stockham_pass_st<F, 8, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, st);
  } else if (rem == 2) {
    stockham_pass_st<F, 4, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, st);
  } else {
    stockham_pass_st<F, 2, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, st);
  }
  return true;
}

// cta_fft whose last pass hands each output to out(index, value) instead of
// storing it (the same pass sequence and arithmetic).  Returns false, having
// run no pass, when no pass is left after the first `done` (the transform is
// then already in buf).
template <class F, int PTS, class Out>
__device__ bool cta_fft_out(char* buf, int log2M, int log2Mt, const typename F::Tw* __restrict__ tw,
                            int tid, int nthr, int done, Out&& out) {
  static_assert(PTS == 16 || PTS == 8, "16 or 8 points per thread");
  constexpr int LP = PTS == 16 ? 4 : 3;
  const int M = 1 << log2M;
  int Ns = 1 << (LP * done);
  int rem = log2M - LP * done;
  if (rem <= 0) return false;
  while (rem > LP) {
    stockham_pass<F, PTS, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr);
    Ns <<= LP;
    rem -= LP;
  }
  // rem = LP, or the remainder pass; with PTS = 16 a remainder of 3 is one
  // radix-8 pass
  if (rem == LP) {
    if constexpr (PTS == 16)
      stockham_pass_out<F, 16, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, out);
    else
      stockham_pass_out<F, 8, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, out);
  } else if (rem == 3) {
    stockham_pass_out<F, 8, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, out);
  } else if (rem == 2) {
    stockham_pass_out<F, 4, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, out);
  } else {
    stockham_pass_out<F, 2, PTS>(buf, M, Ns, log2Mt, tw, tid, nthr, out);
  }
  return true;
}

}  // namespace sft
