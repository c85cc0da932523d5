/*
 * sft.h -- C ABI of the GB300 (sm_103a) sparse FFT by downsampling in time
 * (sFFT-DT, Hsieh, Lu and Pei).
 *
 * Problem (Sec. II-A, Eq. (1)-(2)).  Given x in C^N, recover the K-sparse
 * spectrum X[s] = sum_n x[n] e^{-2 pi i s n / N} (unnormalised DFT; x is its
 * inverse with 1/N).  The signal is downsampled in time, x_{d,l}[n] =
 * x[n d + l], and each length-M = N/d FFT, scaled by d, gives per bin k the
 * syndromes m_l = Y_{d,l}[k] = sum_{s in S_k} X[s] omega^{s l} with
 * omega = e^{2 pi i / N} and S_k = {k + tM : 0 <= t < d} (Eq. (3)).  A bin
 * holding a <= 4 non-zero frequencies is decoded from 2a syndromes
 * (Sec. II-B): Hankel locator solve (Eq. (4)-(5)), roots of the locator
 * polynomial snapped to the candidate set S_k, least-squares value solve.
 *
 * Modes.
 *   SFT_EXACT_ITER   Algorithm 1: level l = 0..max_iters-1 works at
 *                    d_l = 2^l d with M_l = M / 2^l bins, computes the two
 *                    new shifts 2l, 2l+1, folds the syndromes held from
 *                    earlier levels (Y_{2d,j}[k] = Y_{d,j}[k] + Y_{d,j}[k+M/2]),
 *                    removes the frequencies already solved (SubFreq) and
 *                    decodes every active bin with a = l + 1.
 *   SFT_EXACT_FIXED  the non-iterative method (Fig. 1(b)): all 2 a_max shifts
 *                    at d, each active bin decoded once with the smallest
 *                    a <= a_max that validates.
 *   SFT_GENERAL      generally K-sparse signals, Algorithm 2 (Sec. III): the
 *                    2 a_max consecutive shifts and r = n_cs_shifts random
 *                    shifts n_l (drawn from `seed`); per bin the singular
 *                    values of the a_max x a_max Hankel matrix of
 *                    m_0..m_{2a_max-2} (Eq. (26)); the K largest over all
 *                    bins give each bin its count a_k; per bin with a_k > 0
 *                    the a_k-term locator is evaluated at all d candidates,
 *                    the 2 a_k smallest |P~| are kept (pruning Steps 2-3)
 *                    and Subspace Pursuit on the pruned sensing matrix
 *                    Phi_p[j][t] = omega^{(k + tM) n_j} (Eq. (22)) returns
 *                    a_k values.
 *   SFT_GENERAL_UNPRUNED  the CS model of Sec. III-B without the pruning
 *                    strategy (the "without pruning" rows of Tables III-V):
 *                    only the r random shifts; every bin solved by Subspace
 *                    Pursuit at sparsity a_max on the full sensing matrix
 *                    Phi[j][t] = omega^{(k + tM) n_j}, t < d (Eq. (18)),
 *                    and every non-zero coefficient returned (up to
 *                    a_max N/d entries per signal; K is not used).  d <= 4096.
 *
 * Precision.
 *   SFT_FP64   input complex128 (interleaved re, im doubles); FFTs, folds,
 *              peels and solves in FP64.
 *   SFT_MIXED  input complex64 (interleaved re, im floats); the FFTs run on
 *              the FP32 pipes in compensated (float-float) arithmetic, which
 *              keeps FP64-grade syndromes; the held syndromes, folds, peels
 *              and activity tests stay in float-float on the FP32 pipes, and
 *              the per-bin Hankel / root / value solves run in FP64.
 *
 * Conventions of every entry point.
 *   - Pointers marked "device" must be CUDA device (or managed) memory on
 *     the current device; "host" pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Device entry points are asynchronous on that stream; errors of the
 *     launch itself are returned, errors of the kernels surface on the
 *     stream (check with cudaStreamSynchronize).
 *   - A plan is not thread-safe: calls on one plan must not overlap on the
 *     GPU (they share its workspace).  Use one plan per concurrent stream.
 *   - No C++ exception crosses this boundary.
 */
#ifndef SFT_H
#define SFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFT_OK = 0,
  SFT_EINVAL = 1,       /* bad argument: sizes, pointers, parameters      */
  SFT_ENOMEM = 2,       /* device or host allocation failed               */
  SFT_ECUDA = 3,        /* a CUDA call failed (see sft_last_cuda_error)   */
  SFT_ETIMEOUT = 4,     /* a bounded device wait gave up                  */
  SFT_EUNSUPPORTED = 5  /* valid request this build does not implement    */
} sft_status;

typedef enum {
  SFT_EXACT_ITER = 0,
  SFT_EXACT_FIXED = 1,
  SFT_GENERAL = 2,
  SFT_GENERAL_UNPRUNED = 3
} sft_mode;
typedef enum { SFT_FP64 = 0, SFT_MIXED = 1 } sft_precision;

/* Parameters as the paper states the problem (Algorithm 1 inputs: x, K;
 * initialisation d, a_m). */
typedef struct {
  int64_t N;           /* signal length; power of two, 2^3 .. 2^30            */
  int64_t K;           /* sparsity; the result capacity must be >= K         */
  int64_t d;           /* (initial) downsampling factor; d | N, M = N/d a     */
                       /* power of two, M <= 2^26 (M > 8192: four-step FFT)  */
  int32_t a_max;       /* largest alias count: ITER 1..8, FIXED 1..4 or 8,   */
                       /* general 1..4 (0 -> 4 exact, 3 general); above 4    */
                       /* the locator is found by Berlekamp-Massey and the   */
                       /* roots by a search over the d candidates of the bin */
  int32_t max_iters;   /* ITER: number of levels, 1..a_max (0 -> a_max);     */
                       /* M / 2^(max_iters-1) must be >= 1; more than four   */
                       /* levels only with SFT_FP64 (complex128 input): on   */
                       /* complex64 input the decisions of levels 4..7 are   */
                       /* set by the input's rounding (SFT_EUNSUPPORTED)     */
  int32_t mode;        /* sft_mode                                           */
  int32_t precision;   /* sft_precision                                      */
  int32_t n_cs_shifts; /* general modes: random shifts r, 1..16, r <= d (0 -> 3 a_max) */
  int32_t reserved_;   /* must be 0                                          */
  uint64_t seed;       /* general modes only: draws the random shifts        */
  double zero_tol;     /* bin active iff |m| > zero_tol * max_k |Y_{d,0}[k]| */
  double root_tol;     /* a root must lie within root_tol of its candidate    */
  double res_tol;      /* accept iff ||m - Z p||_inf <= res_tol ||m||_inf     */
} sft_params;

/* Fills *p with the paper's defaults for (N, K, d, mode, precision):
 * a_max = 4 (3 for SFT_GENERAL, with r = 9 random shifts), max_iters =
 * a_max, seed 0, and tolerances keyed to the input precision
 * (FP64: zero 1e-10, root 0.1, residual 1e-9; MIXED: 1e-6, 0.1, 1e-6).
 * Returns SFT_EINVAL for a NULL pointer, SFT_OK otherwise (validation of
 * the sizes happens in sft_plan_create). */
sft_status sft_params_default(sft_params* p, int64_t N, int64_t K, int64_t d, int32_t mode,
                              int32_t precision);

/* Result buffers, owned by the caller.  For n_signals signals:
 *   idx        device int64  [n_signals * cap]   recovered locations s
 *   val        device double [n_signals * cap * 2] recovered X[s] (re, im)
 *   count      device int64  [n_signals]         entries written per signal
 *                                                 (<= cap; see `overflow`)
 *   unresolved device int32  [n_signals]         bins left unsolved
 *   overflow   device int32  [n_signals]         1 if more than cap entries
 *                                                 were recovered (extra dropped)
 * Entries of one signal are ordered by bin s mod (N/d), then by s. */
typedef struct {
  int64_t cap;
  int64_t* idx;
  double* val;
  int64_t* count;
  int32_t* unresolved;
  int32_t* overflow;
} sft_result;

typedef struct sft_plan_s* sft_plan_t;

/* Validates *p and creates a plan for batches of up to max_signals signals
 * of that shape: uploads the twiddle / omega tables and allocates the
 * workspace (plan-owned device memory, see sft_plan_workspace_bytes).
 * Must be called with the target device current.  Returns SFT_EINVAL,
 * SFT_EUNSUPPORTED (e.g. M > 2^26), SFT_ENOMEM or SFT_ECUDA. */
sft_status sft_plan_create(const sft_params* p, int64_t max_signals, sft_plan_t* out);

/* Frees the plan and its device memory (synchronises the device). */
void sft_plan_destroy(sft_plan_t plan);

/* Copies the plan's parameters, with every default filled in as
 * sft_plan_create applied them, into *out (host).  Lets a caller check an
 * input against the plan (element type by precision, row length N) before
 * a call.  SFT_EINVAL for a NULL plan or pointer. */
sft_status sft_plan_get_params(sft_plan_t plan, sft_params* out);

/* Device bytes the plan holds (tables + workspace). */
size_t sft_plan_workspace_bytes(sft_plan_t plan);

/* Exactly K-sparse transform of n_signals signals (Algorithm 1, or the
 * non-iterative variant), all on the GPU.
 *   x         device, n_signals signals of N complex values each (complex128
 *             for SFT_FP64, complex64 for SFT_MIXED); signal b starts at
 *             element b * x_stride (x_stride >= N, in complex elements)
 *   r         result buffers (device pointers inside), cap >= K
 * Asynchronous on `stream`.  1 <= n_signals <= max_signals of the plan. */
sft_status sft_exact(sft_plan_t plan, int64_t n_signals, const void* x, int64_t x_stride,
                     const sft_result* r, void* stream);

/* Same transform from and to HOST memory (`x_host` and the arrays of
 * `r_host`, same layout as sft_result, are host pointers); synchronises
 * `stream` before returning.
 *   - If x_host is page-locked (cudaHostAlloc, cudaHostRegister, torch
 *     pin_memory) the kernels read the samples in place over the host link:
 *     only the samples of the shifts cross it, a small fraction of each
 *     signal.  Otherwise the inputs are first copied whole into a
 *     plan-owned device staging buffer.
 *   - If every result array is page-locked the kernels write the results in
 *     place; otherwise they are staged on the device and copied back. */
sft_status sft_exact_host(sft_plan_t plan, int64_t n_signals, const void* x_host,
                          int64_t x_stride, const sft_result* r_host, void* stream);

/* Generally K-sparse transform (Algorithm 2) of n_signals signals; the plan
 * must have mode SFT_GENERAL (at most K entries per signal, the sum of the
 * votes a_k) or SFT_GENERAL_UNPRUNED (at most a_max N/d entries; a result
 * capacity below that count sets `overflow` and keeps the first cap
 * entries in the documented order).  Arguments, layout and behaviour as for sft_exact; the
 * `unresolved` count is 0 (the method has no unsolved-bin notion). */
sft_status sft_general(sft_plan_t plan, int64_t n_signals, const void* x, int64_t x_stride,
                       const sft_result* r, void* stream);

/* Host-memory variant of sft_general (as sft_exact_host). */
sft_status sft_general_host(sft_plan_t plan, int64_t n_signals, const void* x_host,
                            int64_t x_stride, const sft_result* r_host, void* stream);

/* The random shifts n_l of a general-mode plan: r distinct values in
 * [0, d), a partial Fisher-Yates shuffle of 0..d-1 whose draw i exchanges
 * positions i and i + (u_i mod (d - i)), u_i the i-th output of SplitMix64
 * (Steele, Lea, Flood 2014) seeded with params.seed.  Writes up to `cap`
 * into out (host) and returns r (0 for exact plans, -1 for a NULL plan). */
int32_t sft_plan_cs_shifts(sft_plan_t plan, int64_t* out, int32_t cap);

/* ---- heterogeneous batches ---------------------------------------------
 * Many signals of uneven N, K and kind (exactly or generally sparse) in one
 * call.  A batch context groups the signals by shape (everything except K
 * that fixes the launch sequence), keeps one internal plan per shape, reads
 * every signal's input pointer, result buffers and K from device tables
 * (no copies of the signals), captures the launches of the whole call into
 * one CUDA graph and replays it while the composition of the batch (the
 * shapes and how many signals of each) stays the same.  Exactly sparse
 * signals that fit one CTA run in one persistent kernel
 * (sft_batch_set_persistent).  On the first call of a shape class (log2
 * N/d, a_max, mode, precision) an autotuner times the group's launch
 * sequence for every combination of FFT points per thread (8 or 16) and
 * decoder CTAs per SM (2, 4, 8, 16) on that call's data and keeps the
 * fastest for every later group of the class; the FFT points change the
 * rounding of the FFT, so values may differ from a single-signal call in
 * the last bits.  Not thread-safe; calls on one context must not overlap on
 * the GPU. */
typedef struct sft_batch_s* sft_batch_t;

sft_status sft_batch_create(sft_batch_t* out);
/* Frees the context, its plans and its graph (synchronises the device). */
void sft_batch_destroy(sft_batch_t ctx);
/* use_graph: capture and replay (default 1); autotune: tune new shapes
 * (default 1). */
sft_status sft_batch_set_options(sft_batch_t ctx, int32_t use_graph, int32_t autotune);
/* Transforms n_signals signals.  Host arrays of n_signals entries:
 *   params   the parameters of each signal (mode SFT_EXACT_ITER,
 *            SFT_EXACT_FIXED or SFT_GENERAL; as for sft_plan_create)
 *   x        the address of each signal as the GPU sees it (complex64 for
 *            SFT_MIXED, complex128 for SFT_FP64): device memory, or
 *            page-locked host memory, which the kernels read in place
 *   results  each signal's own result buffers (device or page-locked host
 *            memory; count, unresolved and overflow point at one value
 *            each; cap >= K)
 * Asynchronous on `stream`; the first call of a new composition builds
 * plans (allocates) and captures the graph. */
sft_status sft_batch(sft_batch_t ctx, int64_t n_signals, const sft_params* params,
                     const void* const* x, const sft_result* results, void* stream);
/* Groups of the last call, nodes of the current graph, shape classes
 * (log2 N/d, a_max, mode, precision) in the autotuner's table. */
int32_t sft_batch_info(sft_batch_t ctx, int32_t* n_groups, int64_t* n_graph_nodes,
                       int32_t* n_tuned);
/* The persistent kernel of a batch (not in the paper; Algorithm 1 per
 * signal, unchanged).  With enable != 0 (the default) every exactly sparse
 * signal that fits one CTA -- SFT_EXACT_ITER, SFT_MIXED, a_max <= 4,
 * N/d <= 4096 -- is one item of a device work queue that a single launch of
 * resident CTAs drains, largest signals first; each CTA runs the whole of
 * Algorithm 1 for the signal it claimed (gather, FFTs, folds, SubFreq,
 * decodes, compaction of the result) with the arithmetic of the per-shape
 * launch sequence, so that results equal those of sft_exact on one signal.
 * No CTA waits on another: the queue head is the only shared state.  ctas
 * is the launch's CTA count (0: chosen by the autotuner on the first call
 * that has such signals).  SFT_EINVAL for a NULL context or ctas < 0. */
sft_status sft_batch_set_persistent(sft_batch_t ctx, int32_t enable, int32_t ctas);
/* Signals of the last call that ran in the persistent kernel, and the CTAs
 * of its launch. */
int32_t sft_batch_persistent_info(sft_batch_t ctx, int64_t* n_signals, int32_t* ctas);

/* Allocation-free variant of sft_exact (the paper has no counterpart: this
 * is a deployment interface).  Some callers cannot allocate device memory
 * when they need a transform -- code inside another framework's memory
 * manager that owns every device byte, latency-critical loops that cannot
 * absorb cudaFree's implicit device synchronisation or an allocation failure
 * mid-run, fixed-budget embedded deployments -- and so cannot create a plan.
 * This entry point takes the parameters directly and keeps its tables and
 * workspace in one static device array of SFT_NOALLOC_SCRATCH_BYTES that the
 * library holds on every device that loads it, until the process exits.  It
 * calls no allocation routine.
 *   p, n_signals, x, x_stride, r   as for sft_plan_create + sft_exact
 *                                  (x and the arrays of r are device memory)
 * Returns SFT_EINVAL (with the required and the maximum size in
 * sft_last_cuda_error) when n_signals signals of this shape do not fit the
 * array: per signal 275 * N/d + 16 bytes for SFT_EXACT_ITER (338 * N/d + 16
 * for SFT_EXACT_FIXED with a_max = 4), plus 16 * (N/d + 2 * (2^ceil(log2(N)/2)
 * + 2^floor(log2(N)/2))) bytes of tables, 256 bytes of counters and 256-byte
 * alignment of each array (at N = 2^22, N/d = 2^13: 7 signals per call).
 *
 * Set-up.  The library's module is loaded lazily, so the first call on each
 * device is where the array's memory is committed on that device and where
 * the call looks up the array's device address there.  Make that first call
 * at start-up, before any stream capture and before another memory manager
 * reserves the device; when the device has no room for the array it returns
 * SFT_ECUDA with "scratch set-up: out of memory" in sft_last_cuda_error.  A
 * call that finds a different current context on the device than the one
 * the address was looked up in (after cudaDeviceReset, for instance) repeats
 * the look-up and the set-up, so it too should come outside any capture.
 *
 * Differences from the plan path: the gather reads each shift's samples
 * straight from x (no compact extraction pass, which would need the array's
 * room for a copy of the samples), and the omega and twiddle tables are
 * computed on the device in FP64 (the plan path computes them on the host in
 * long double); both round to within an ulp, so results agree with
 * sft_exact's to rounding.  All calls share the array and it keeps the last
 * call's contents; each call rebuilds what it needs, but calls that overlap
 * on the GPU race and must be serialised by the caller.  Asynchronous on
 * `stream` like sft_exact. */
#define SFT_NOALLOC_SCRATCH_BYTES (16u << 20)
sft_status sft_exact_noalloc(const sft_params* p, int64_t n_signals, const void* x,
                             int64_t x_stride, const sft_result* r, void* stream);

/* ---- learned support proposal (generally K-sparse path) ----------------
 *
 * Not in the paper: a small network proposes, for every bin that Algorithm 2
 * votes a_k > 0 aliases, the candidates t of S_k = {k + tM} that pruning
 * Step 2 would otherwise take from the a_k-term locator; Subspace Pursuit
 * runs on them as in Step 3, and the paper's own residual judges the
 * result: over all 2a_m + r equations of Eq. (3) the network's solution
 * replaces the plain one only when its squared residual is below
 * (1 - 1e-6) times the plain solution's.  The plain decoder is therefore
 * the fallback and the judge of every prediction.
 *
 * Features of a voted bin k (2 (2a_m + r) floats): the syndromes of its
 * 2a_m consecutive and r random shifts sh_l, de-rotated by omega^{-k sh_l}
 * (which leaves sum_j p_j e^{2 pi i t_j sh_l / d}), rotated so that the
 * first is real and non-negative, scaled to unit 2-norm, interleaved
 * (re, im).  Network: n_in -> 128 -> 128 -> n_sup + n_cls, ReLU, FP16
 * weights with FP32 accumulation (FP32 master copy, Adam).  Outputs:
 * support logits over t = 0..d-1 and count logits over 0..a_m+1 aliases.
 * Loss per row: count cross-entropy + mean support binary cross-entropy.
 *
 * Parameters are one FP32 vector, in order: W1 [n_in][128], b1 [128],
 * W2 [128][128], b2 [128], W3 [128][n_out], b3 [n_out], n_out = n_sup +
 * n_cls (support logits first).  Not thread-safe; calls that share an
 * sft_mlp_t must not overlap on the GPU. */
typedef struct sft_mlp_s* sft_mlp_t;
typedef struct {
  int32_t n_in;      /* 2 (2 a_max + n_cs_shifts), at most 48             */
  int32_t n_hidden;  /* 128 (the only width built)                        */
  int32_t n_sup;     /* support logits: d, at most 128                    */
  int32_t n_cls;     /* count classes: a_max + 2                          */
  uint64_t seed;     /* initial weights: He-uniform from SplitMix64(seed) */
  float lr, beta1, beta2, eps;  /* Adam                                    */
} sft_mlp_config;

/* Dimensions matching a SFT_GENERAL parameter set (and the default Adam
 * settings lr 2e-3, 0.9, 0.999, 1e-8).  SFT_EUNSUPPORTED when d > 128 or
 * the feature count exceeds 48. */
sft_status sft_mlp_config_for(const sft_params* p, sft_mlp_config* out);
sft_status sft_mlp_create(const sft_mlp_config* c, sft_mlp_t* out);
void sft_mlp_destroy(sft_mlp_t mlp);
int64_t sft_mlp_param_count(sft_mlp_t mlp);
/* Host copies of the FP32 parameters (layout above).  Setting them resets
 * the Adam moments and step count. */
sft_status sft_mlp_get_params(sft_mlp_t mlp, float* host_out);
sft_status sft_mlp_set_params(sft_mlp_t mlp, const float* host_in);

/* Features of the bins a SFT_GENERAL plan votes, for training data: runs
 * the gather/FFT, singular-value and vote stages of sft_general on
 * n_signals signals (x as for sft_general) and writes, for up to cap_rows
 * voted bins, feat (device, [cap_rows][n_in] floats) and rows (device,
 * [cap_rows][3] int32: signal, bin, a_k).  Row order is unspecified.
 * Synchronises `stream`; *n_rows (host) receives the number of voted bins
 * (rows beyond cap_rows are not written). */
sft_status sft_mlp_features(sft_plan_t plan, int64_t n_signals, const void* x, int64_t x_stride,
                            float* feat, int32_t* rows, int64_t cap_rows, int64_t* n_rows,
                            void* stream);
/* Logits of n_rows feature rows (device [n_rows][n_in] -> device
 * [n_rows][n_out] floats).  Asynchronous. */
sft_status sft_mlp_forward(sft_mlp_t mlp, const float* feat, int64_t n_rows, float* logits,
                           void* stream);
/* Mean loss and its gradient over n_rows labelled rows, without updating
 * the parameters: feat (device [n_rows][n_in]), cls (device int32
 * [n_rows], 0..n_cls-1), sup (device uint32 [n_rows][4], bit t of word
 * t/32 set when t is in the bin's support); grad (device, param_count
 * floats, overwritten), loss (device, one float, overwritten).
 * Asynchronous. */
sft_status sft_mlp_grad(sft_mlp_t mlp, const float* feat, const int32_t* cls, const uint32_t* sup,
                        int64_t n_rows, float* grad, float* loss, void* stream);
/* Trains in place with Adam for `epochs` passes over the rows in
 * minibatches of `batch` (a fresh SplitMix64-driven shuffle per epoch from
 * shuffle_seed); the forward and backward passes and the update run in
 * this library's kernels.  loss_out (host, `epochs` floats, may be NULL)
 * receives each epoch's mean loss.  Synchronises `stream`. */
sft_status sft_mlp_train(sft_mlp_t mlp, const float* feat, const int32_t* cls, const uint32_t* sup,
                         int64_t n_rows, int32_t epochs, int32_t batch, uint64_t shuffle_seed,
                         float* loss_out, void* stream);
/* Attach the network to a SFT_GENERAL plan (its dimensions must match the
 * plan: n_in = 2 (2 a_max + n_cs_shifts), n_sup = d, n_cls = a_max + 2);
 * sft_general on that plan then proposes and judges as described above.
 * NULL detaches.  The plan does not own the network; keep it alive while
 * attached. */
sft_status sft_plan_attach_mlp(sft_plan_t plan, sft_mlp_t mlp);

/* Unknown K (Sec. II-E, the bottom-up strategy): each signal is transformed
 * with d = N / M_start, then with d halved (M doubled) while its run leaves
 * a bin unsolved or a level-0 bin overflowed, up to M_max (0: N).
 *   p        N, a_max, mode (SFT_EXACT_ITER or SFT_EXACT_FIXED), precision,
 *            tolerances; K, d and max_iters are ignored (ITER runs
 *            min(a_max, log2(M) + 1) levels at each M)
 *   x        device, n_signals rows of N complex values, row pitch x_stride
 *   r        device result arrays laid out as for sft_exact (cap per
 *            signal); each signal's row holds its last run
 *   m_out    host, n_signals entries (may be NULL): the M each signal
 *            stopped at (its last M when it never solved every bin)
 * Creates and destroys one plan per M tried (synchronous; allocates).
 * SFT_EINVAL on bad arguments, SFT_EUNSUPPORTED when M_max > 2^26. */
sft_status sft_exact_auto(const sft_params* p, int64_t n_signals, const void* x, int64_t x_stride,
                          int64_t M_start, int64_t M_max, const sft_result* r, int64_t* m_out,
                          void* stream);

/* Collision counts (Sec. II-C, Lemma 2 and Fig. 2): for n_sets support sets
 * of K locations each, the number of bins k < M holding exactly a of a
 * set's locations (k = s mod M), summed over the sets.
 *   supports  device int64 [n_sets][K]; any values (only s mod M is used);
 *             may be NULL when n_sets or K is 0
 *   M         number of bins, a power of two <= 2^15
 *   n_cells   2..33: hist[a] for a < n_cells - 1, hist[n_cells - 1] counts
 *             the bins holding n_cells - 1 or more
 *   hist      device int64 [n_cells], overwritten
 * Asynchronous on `stream`.  SFT_EINVAL on NULL pointers or bad sizes,
 * SFT_EUNSUPPORTED for M > 2^15. */
sft_status sft_alias_histogram(const int64_t* supports, int64_t n_sets, int64_t K, int64_t M,
                               int32_t n_cells, int64_t* hist, void* stream);

/* Number of kernel launches one call of this plan on max_signals signals
 * issues (sft_exact / sft_general). */
int32_t sft_plan_launches_per_call(sft_plan_t plan);

/* Work counts of the plan's last call, for throughput models, summed over
 * the call's signals and sub-batches: the number of (signal, bin) pairs
 * queued for decoding at each level of SFT_EXACT_ITER (Algorithm 1's active
 * or unsolved bins, decoded with a = l + 1), or entering each round
 * a = 1..a_max of SFT_EXACT_FIXED; for SFT_GENERAL three counts: the bins
 * whose Hankel singular values are computed (those the pruning bounds leave
 * open), the voted bins with a_k = 1, the voted bins with a_k >= 2.
 * Synchronises the device; writes up to `cap` entries to out (host) and
 * returns their number (0 for SFT_GENERAL_UNPRUNED, -1 for a NULL plan or
 * a CUDA error). */
int32_t sft_plan_queue_lengths(sft_plan_t plan, int64_t* out, int32_t cap);

/* Sub-batching.  A call on n signals may be split into S sub-batches of
 * consecutive signals (sizes differ by at most one), each enqueued on its
 * own stream forked from and joined back into the call's stream, so that
 * the latency-bound stages of one overlap the throughput-bound stages of
 * another.  Results are identical for every S.  n = 0 (the default)
 * chooses S = min(4, n_signals / 32) (at least 1); 1..4
 * fixes it (capped at the call's signal count).  The plan creates its
 * three extra streams when it is created.  sft_plan_sub_batches returns the S a
 * call of n_signals signals would use.  SFT_EINVAL for n outside 0..4. */
sft_status sft_plan_set_sub_batches(sft_plan_t plan, int32_t n);
int32_t sft_plan_sub_batches(sft_plan_t plan, int64_t n_signals);

/* Four-lane decoders (exact paths, mixed precision; off by default).  SynDec
 * of a bin with a = 3 or 4 aliases (Sec. II-B steps (i)-(iii)) is a serial
 * chain of FP64 operations, so on few signals the last levels of ITER and
 * the last rounds of FIXED take the time of one bin's chain.  With
 * enable != 0, a call that runs as one sub-batch decodes a queue of at most
 * 64 bins per SM with four lanes per bin: both small solves by row-per-lane
 * elimination, one root, one or two Gram sums and one right-hand side per
 * lane, the validation residual split by equation.  That shortens the chain
 * but spends about twice the FP64 issue slots per bin, so longer queues and
 * calls split into sub-batches keep the one-lane decoder.  The supports are
 * those of the one-lane decoder; the values agree to float-float rounding
 * (~1e-13), not bit for bit, with calls that use the one-lane decoder (other
 * sub-batch counts, batches).  SFT_EINVAL on a NULL plan. */
sft_status sft_plan_set_quad_decoders(sft_plan_t plan, int32_t enable);

/* Per-stage timing.  With profiling enabled, every launch of an sft_exact
 * call on this plan is bracketed by CUDA events recorded on the call's
 * stream.  sft_plan_stage_times synchronises the device, sums the elapsed
 * times per stage name since the previous read (or since profiling was
 * enabled), writes up to `cap` entries (names are static strings, ms is the
 * total, launches the number of launches summed) and resets the record.
 * *n receives the number of stages.  Profiling adds one event pair per launch. */
sft_status sft_plan_set_profiling(sft_plan_t plan, int32_t enable);
sft_status sft_plan_stage_times(sft_plan_t plan, int32_t cap, const char** names, double* ms,
                                int64_t* launches, int32_t* n);

/* The same records as a timeline: one entry per profiled launch since the
 * previous read, in enqueue order.  names[i] is the stage (static string),
 * sub[i] the sub-batch whose stream ran it (0 for a call that is not split),
 * t0_ms[i] / t1_ms[i] its start and end in ms after the start of the first
 * record.  Synchronises the device, writes up to `cap` entries (host
 * arrays, owned by the caller), *n receives the number of records, and the
 * record is reset (like sft_plan_stage_times).  Shows how the sub-batches'
 * stages overlap, e.g. the host-link extraction of one against the compute
 * of another.  SFT_EINVAL on a NULL plan or n, or cap > 0 with a NULL
 * array; SFT_ECUDA if the synchronisation fails. */
sft_status sft_plan_stage_timeline(sft_plan_t plan, int32_t cap, const char** names, int32_t* sub,
                                   double* t0_ms, double* t1_ms, int32_t* n);

/* The device arithmetic the FP64 decoders build on, evaluated elementwise,
 * so that it can be checked against correctly rounded references.  x and
 * out are device arrays of n doubles (which = 0, 1) or n complex values as
 * (re, im) pairs, 2n doubles (which = 2), owned by the caller; the call is
 * enqueued on `stream` (NULL: the default stream) and returns without
 * waiting.
 *   which = 0: the reciprocal 1/x (an FP32 seed whose operand is x
 *              truncated to float and whose result is widened back, both
 *              by moving bits, then two Newton steps r <- r + r (1 - x r);
 *              an FP64 division for |x| outside [2^-123, 2^124));
 *   which = 1: the float nearest x widened back to double by moving bits
 *              (exact);
 *   which = 2: the principal complex square root of the closed-form roots
 *              (cancellation-free form, the reciprocal above for its
 *              quotient), for values whose squared magnitude is a normal
 *              double.
 * SFT_EINVAL on n < 0, which outside 0..2, or NULL arrays with n > 0;
 * SFT_ECUDA if the launch fails. */
sft_status sft_device_math_check(const double* x, int64_t n, double* out, int32_t which,
                                 void* stream);

/* Human-readable name of a status code (static storage). */
const char* sft_strerror(sft_status s);

/* Detail of the last error this library reported in the calling thread: the
 * CUDA error text for SFT_ECUDA, the offending argument for SFT_EINVAL
 * (static per-thread storage; "" if none). */
const char* sft_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFT_H */
