// sft_batch.cu -- many signals of uneven N, K and kind in one call.
//
// Signals are grouped by shape (everything that fixes the launch sequence:
// N, d, mode, precision, a_max, levels, random shifts, tolerances; K is
// per signal).  Each group owns an internal plan (tables and workspace).
//
// Two ways to run a group:
//  - the persistent kernel (sft_persist.cu): every exactly sparse signal of
//    the batch that fits one CTA (ITER, mixed precision, a_max <= 4,
//    N/d <= 4096) becomes one item of a device work queue, and a single
//    launch of resident CTAs drains it, largest signals first;
//  - the group's own launch sequence (the plan path), reading every
//    signal's input pointer, result buffers and K from device tables, so
//    that any set of buffers is batched without copies.
// The whole call -- the persistent launch and the groups' sequences, spread
// over capture lanes -- is captured once into a CUDA graph and replayed
// while the batch composition stays the same; only the tables are
// refreshed per call.
//
// Autotuning.  The first time a shape class (log2 N/d, a_max, mode,
// precision) is seen, its group is timed on the call's own data for every
// combination of FFT points per thread (8 or 16) and decoder CTAs per SM
// (2, 4, 8, 16), and the fastest is kept in a table that every later group
// of that class uses.  The persistent kernel's CTA count is tuned the same
// way (a quarter, half or all of the SMs' resident CTAs) on the first call
// that has persistent signals.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

#include "sft_internal.h"

namespace {

struct ShapeKey {
  int64_t N, d;
  int32_t a_max, max_iters, mode, precision, n_cs;
  uint64_t seed;
  double zt, rt, et;
  auto tie() const {
    return std::tie(N, d, a_max, max_iters, mode, precision, n_cs, seed, zt, rt, et);
  }
  bool operator<(const ShapeKey& o) const { return tie() < o.tie(); }
};

ShapeKey key_of(const sft_params& p) {
  return ShapeKey{p.N,         p.d,       p.a_max,    p.mode == SFT_EXACT_ITER ? p.max_iters : 0,
                  p.mode,      p.precision, sft::is_general_mode(p.mode) ? p.n_cs_shifts : 0,
                  sft::is_general_mode(p.mode) ? p.seed : 0, p.zero_tol, p.root_tol, p.res_tol};
}

struct Group {
  sft_plan_t plan = nullptr;
  int64_t capacity = 0;
  std::vector<int64_t> members;  // signal indices of the current call
  int64_t off = 0;               // first table entry of the group
  bool tuned = false;
  bool persist = false;          // its signals run in the persistent kernel
};

// Shape class of the autotuner's table and the launch shape picked for it.
struct TuneKey {
  int log2M, a_max, mode, precision;
  bool operator<(const TuneKey& o) const {
    return std::tie(log2M, a_max, mode, precision) <
           std::tie(o.log2M, o.a_max, o.mode, o.precision);
  }
};
struct TunePick {
  int dec_ctas_per_sm, fft_pts;
};

int ilog2i(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// A signal the persistent kernel takes: one CTA holds its FFT and its queue.
bool persistent_fits(const sft_params& p) {
  return p.mode == SFT_EXACT_ITER && p.precision == SFT_MIXED && p.a_max <= 4 &&
         p.max_iters <= 4 && p.N / p.d <= sft::kPersistMaxM;
}

}  // namespace

struct sft_batch_s {
  std::map<ShapeKey, Group> groups;
  int64_t tab_cap = 0;
  void** x_tab = nullptr;  // device tables
  sft_result* r_tab = nullptr;
  int64_t* k_tab = nullptr;
  void** hx = nullptr;  // pinned host staging
  sft_result* hr = nullptr;
  int64_t* hk = nullptr;
  cudaEvent_t staged = nullptr;  // last table upload done
  cudaStream_t cap_stream = nullptr;
  // independent groups run concurrently inside the graph: forked onto
  // kLanes capture streams, joined back at the end
  static constexpr int kLanes = 8;
  cudaStream_t lane[kLanes] = {};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[kLanes] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> comp;  // composition the graph was captured for
  int use_graph = 1, autotune = 1;
  int32_t last_groups = 0, tuned = 0;
  size_t graph_nodes = 0;
  std::map<TuneKey, TunePick> table;  // autotuned launch shapes per shape class
  // persistent kernel: signal descriptors and their order (device and
  // page-locked staging), the queue head, the CTA count
  int use_persistent = 1;
  int persist_ctas = 0;        // set by the caller (0: tuned)
  int persist_pick = 0;        // tuned CTA count
  int64_t p_cap = 0;
  sft::PSig* psig = nullptr;
  int* porder = nullptr;
  int* phead = nullptr;
  sft::PSig* hpsig = nullptr;
  int* hporder = nullptr;
  int64_t last_persist = 0;    // signals of the last call in the persistent kernel
  int32_t last_persist_ctas = 0;
};

namespace {

void free_tables(sft_batch_s* B) {
  if (B->x_tab) cudaFree(B->x_tab);
  if (B->r_tab) cudaFree(B->r_tab);
  if (B->k_tab) cudaFree(B->k_tab);
  if (B->hx) cudaFreeHost(B->hx);
  if (B->hr) cudaFreeHost(B->hr);
  if (B->hk) cudaFreeHost(B->hk);
  B->x_tab = nullptr;
  B->r_tab = nullptr;
  B->k_tab = nullptr;
  B->hx = nullptr;
  B->hr = nullptr;
  B->hk = nullptr;
  B->tab_cap = 0;
}

void free_persist(sft_batch_s* B) {
  if (B->psig) cudaFree(B->psig);
  if (B->porder) cudaFree(B->porder);
  if (B->phead) cudaFree(B->phead);
  if (B->hpsig) cudaFreeHost(B->hpsig);
  if (B->hporder) cudaFreeHost(B->hporder);
  B->psig = nullptr;
  B->porder = nullptr;
  B->phead = nullptr;
  B->hpsig = nullptr;
  B->hporder = nullptr;
  B->p_cap = 0;
}

void drop_graph(sft_batch_s* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
  B->comp.clear();
}

cudaError_t grow_tables(sft_batch_s* B, int64_t n) {
  if (B->tab_cap >= n) return cudaSuccess;
  drop_graph(B);
  free_tables(B);
  const int64_t cap = n + n / 2 + 16;
  cudaError_t e;
  if ((e = cudaMalloc(&B->x_tab, cap * sizeof(void*)))) return e;
  if ((e = cudaMalloc(&B->r_tab, cap * sizeof(sft_result)))) return e;
  if ((e = cudaMalloc(&B->k_tab, cap * sizeof(int64_t)))) return e;
  if ((e = cudaMallocHost(&B->hx, cap * sizeof(void*)))) return e;
  if ((e = cudaMallocHost(&B->hr, cap * sizeof(sft_result)))) return e;
  if ((e = cudaMallocHost(&B->hk, cap * sizeof(int64_t)))) return e;
  B->tab_cap = cap;
  return cudaSuccess;
}

cudaError_t grow_persist(sft_batch_s* B, int64_t n) {
  if (B->p_cap >= n) return cudaSuccess;
  drop_graph(B);
  free_persist(B);
  const int64_t cap = n + n / 2 + 16;
  cudaError_t e;
  if ((e = cudaMalloc(&B->psig, cap * sizeof(sft::PSig)))) return e;
  if ((e = cudaMalloc(&B->porder, cap * sizeof(int)))) return e;
  if ((e = cudaMalloc(&B->phead, sizeof(int)))) return e;
  if ((e = cudaMallocHost(&B->hpsig, cap * sizeof(sft::PSig)))) return e;
  if ((e = cudaMallocHost(&B->hporder, cap * sizeof(int)))) return e;
  B->p_cap = cap;
  return cudaSuccess;
}

// The persistent kernel's descriptor of member j (signal i) of group g.
sft::PSig persist_desc(const Group& g, int64_t j, const void* x, const sft_result& r) {
  const sft_plan_s* P = g.plan;
  const sft::Workspace& W = P->ws;
  sft::PSig d{};
  d.x = static_cast<const float2*>(x);
  d.N = P->p.N;
  d.d0 = P->p.d;
  d.M0 = P->M0;
  d.levels = P->levels;
  d.log2M0 = P->log2M0;
  d.zero_tol = P->p.zero_tol;
  d.root_tol = P->p.root_tol;
  d.res_tol = P->p.res_tol;
  d.tw = static_cast<const float4*>(P->tab.tw);
  d.om_hi = P->tab.om_hi;
  d.om_lo = P->tab.om_lo;
  d.om_hi_ff = P->tab.om_hi_ff;
  d.om_lo_ff = P->tab.om_lo_ff;
  d.om_lo_bits = P->tab.om_lo_bits;
  for (int i = 0; i < 2; ++i) {
    d.held[i] = static_cast<char*>(W.held[i]) + j * W.held_elems * 16;
    d.T[i] = W.T[i] + j * P->M0;
  }
  d.held_elems = W.held_elems;
  d.slot_cnt = W.slot_cnt + j * P->M0;
  d.slot_s = W.slot_s + j * P->M0 * sft::kSlots;
  d.slot_p = static_cast<float4*>(W.slot_p) + j * P->M0 * sft::kSlots;
  d.ymax2 = W.ymax2 + j;
  d.flags = W.flags + j;
  d.r = r;
  return d;
}

int sm_count() {
  int dev = 0, nsm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}

// Enqueue one group's transform on stream s (tables already on the device).
cudaError_t enqueue_group(sft_batch_s* B, Group& g, cudaStream_t s) {
  sft_plan_s* P = g.plan;
  const int64_t n = (int64_t)g.members.size();
  P->x_table = reinterpret_cast<const void* const*>(B->x_tab + g.off);
  P->r_table = B->r_tab + g.off;
  P->K_table = B->k_tab + g.off;
  sft_result dummy{};
  cudaError_t e = cudaMemsetAsync(P->ws.zero_base, 0, P->ws.zero_bytes, s);
  if (e == cudaSuccess) e = sft::launch_exact(P, n, nullptr, P->p.N, &dummy, s);
  P->x_table = nullptr;
  P->r_table = nullptr;
  P->K_table = nullptr;
  return e;
}

// Picks the group's launch shape: from the table when its shape class was
// tuned before, else by timing the group on this call's data for every
// (FFT points per thread, decoder CTAs per SM) and recording the fastest.
cudaError_t tune_group(sft_batch_s* B, Group& g, cudaStream_t s) {
  sft_plan_s* P = g.plan;
  const TuneKey key{P->log2M0, P->p.a_max, P->p.mode, P->p.precision};
  auto it = B->table.find(key);
  if (it != B->table.end()) {
    P->dec_ctas_per_sm = it->second.dec_ctas_per_sm;
    P->fft_pts = it->second.fft_pts;
    g.tuned = true;
    return cudaSuccess;
  }
  const int ctas[4] = {2, 4, 8, 16};
  const int pts[2] = {8, 16};
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  TunePick pick{8, 8};
  cudaError_t e = cudaSuccess;
  for (int pp : pts) {
    for (int c : ctas) {
      P->fft_pts = pp;
      P->dec_ctas_per_sm = c;
      e = enqueue_group(B, g, s);  // warm
      if (e == cudaSuccess) e = cudaEventRecord(t0, s);
      if (e == cudaSuccess) e = enqueue_group(B, g, s);
      if (e == cudaSuccess) e = cudaEventRecord(t1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      if (e != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (ms < best) {
        best = ms;
        pick = TunePick{c, pp};
      }
    }
    if (e != cudaSuccess) break;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  P->dec_ctas_per_sm = pick.dec_ctas_per_sm;
  P->fft_pts = pick.fft_pts;
  if (e == cudaSuccess) B->table[key] = pick;
  g.tuned = true;
  return e;
}

// The persistent kernel's CTA count: a quarter, half or all of its resident
// CTAs, timed on this call's signals (descriptors already on the device).
cudaError_t tune_persist(sft_batch_s* B, int n, cudaStream_t s) {
  const int full = sm_count() * std::max(1, sft::persistent_ctas_per_sm());
  const int cands[3] = {std::max(1, full / 4), std::max(1, full / 2), full};
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  int pick = full;
  cudaError_t e = cudaSuccess;
  for (int c : cands) {
    e = sft::launch_exact_persistent(B->psig, B->porder, n, B->phead, c, s);
    if (e == cudaSuccess) e = cudaEventRecord(t0, s);
    if (e == cudaSuccess) e = sft::launch_exact_persistent(B->psig, B->porder, n, B->phead, c, s);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  B->persist_pick = pick;
  return e;
}

}  // namespace

extern "C" {

sft_status sft_batch_create(sft_batch_t* out) {
  if (!out) return SFT_EINVAL;
  sft_batch_s* B = new (std::nothrow) sft_batch_s();
  if (!B) return SFT_ENOMEM;
  bool ok = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->staged, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&B->fork_ev, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < sft_batch_s::kLanes; ++i)
    ok = cudaStreamCreateWithFlags(&B->lane[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&B->join_ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    sft::set_error_detail("sft_batch_create: stream or event creation failed");
    delete B;
    return SFT_ECUDA;
  }
  *out = B;
  return SFT_OK;
}

void sft_batch_destroy(sft_batch_t B) {
  if (!B) return;
  cudaDeviceSynchronize();
  drop_graph(B);
  for (auto& kv : B->groups)
    if (kv.second.plan) sft_plan_destroy(kv.second.plan);
  free_tables(B);
  free_persist(B);
  if (B->staged) cudaEventDestroy(B->staged);
  if (B->fork_ev) cudaEventDestroy(B->fork_ev);
  for (int i = 0; i < sft_batch_s::kLanes; ++i) {
    if (B->lane[i]) cudaStreamDestroy(B->lane[i]);
    if (B->join_ev[i]) cudaEventDestroy(B->join_ev[i]);
  }
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  delete B;
}

sft_status sft_batch_set_options(sft_batch_t B, int32_t use_graph, int32_t autotune) {
  if (!B) return SFT_EINVAL;
  if ((use_graph != 0) != (B->use_graph != 0)) drop_graph(B);
  B->use_graph = use_graph != 0;
  B->autotune = autotune != 0;
  return SFT_OK;
}

sft_status sft_batch_set_persistent(sft_batch_t B, int32_t enable, int32_t ctas) {
  if (!B || ctas < 0) return SFT_EINVAL;
  if ((enable != 0) != (B->use_persistent != 0) || ctas != B->persist_ctas) drop_graph(B);
  B->use_persistent = enable != 0;
  B->persist_ctas = ctas;
  return SFT_OK;
}

int32_t sft_batch_persistent_info(sft_batch_t B, int64_t* n_signals, int32_t* ctas) {
  if (!B) return -1;
  if (n_signals) *n_signals = B->last_persist;
  if (ctas) *ctas = B->last_persist_ctas;
  return 0;
}

int32_t sft_batch_info(sft_batch_t B, int32_t* n_groups, int64_t* n_graph_nodes, int32_t* n_tuned) {
  if (!B) return -1;
  if (n_groups) *n_groups = B->last_groups;
  if (n_graph_nodes) *n_graph_nodes = (int64_t)B->graph_nodes;
  if (n_tuned) *n_tuned = (int32_t)B->table.size();
  return 0;
}

sft_status sft_batch(sft_batch_t B, int64_t n, const sft_params* ps, const void* const* x,
                     const sft_result* rs, void* stream) {
  if (!B || n < 1 || !ps || !x || !rs) {
    sft::set_error_detail("sft_batch: NULL context, params, inputs or results, or n < 1");
    return SFT_EINVAL;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (auto& kv : B->groups) kv.second.members.clear();
  // 1. normalise, validate and group the signals
  std::vector<sft_params> norm((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    sft_params p = ps[i];
    sft::normalize_params(&p);
    sft_status v = sft::validate_params(p);
    char msg[256];
    if (v != SFT_OK) {
      std::snprintf(msg, sizeof(msg), "sft_batch: signal %lld: invalid parameters", (long long)i);
      sft::set_error_detail(msg);
      return v;
    }
    const sft_result& r = rs[i];
    if (!x[i] || r.cap < p.K || r.cap < 1 || !r.idx || !r.val || !r.count || !r.unresolved ||
        !r.overflow) {
      std::snprintf(msg, sizeof(msg), "sft_batch: signal %lld: NULL buffer or cap < K",
                    (long long)i);
      sft::set_error_detail(msg);
      return SFT_EINVAL;
    }
    norm[(size_t)i] = p;
    B->groups[key_of(p)].members.push_back(i);
  }
  // 2. a plan with enough capacity for every group in use (a persistent
  // group's plan holds its tables and workspace; its launch sequence is
  // not used)
  int32_t ngroups = 0;
  int64_t off = 0, n_p = 0;
  for (auto& kv : B->groups) {
    Group& g = kv.second;
    if (g.members.empty()) continue;
    ++ngroups;
    const int64_t size = (int64_t)g.members.size();
    if (!g.plan || g.capacity < size) {
      drop_graph(B);
      if (g.plan) sft_plan_destroy(g.plan);
      g.plan = nullptr;
      sft_params p = norm[(size_t)g.members[0]];
      p.K = 0;  // K is per signal (tables)
      sft_status cs = sft_plan_create(&p, size, &g.plan);
      if (cs != SFT_OK) return cs;
      g.capacity = size;
      g.tuned = false;
    }
    g.persist = B->use_persistent && persistent_fits(g.plan->p);
    if (g.persist) n_p += size;
    g.off = off;
    off += size;
  }
  // 3. per-signal tables (pinned staging -> device, ordered before the launches)
  cudaError_t e = grow_tables(B, n);
  if (e == cudaSuccess && n_p > 0) e = grow_persist(B, n_p);
  if (e == cudaSuccess) e = cudaEventSynchronize(B->staged);  // staging free again
  if (e != cudaSuccess) {
    sft::set_error_detail(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
  }
  std::vector<std::pair<std::pair<int64_t, int64_t>, int>> porder;
  int64_t ip = 0;
  for (auto& kv : B->groups) {
    Group& g = kv.second;
    for (size_t j = 0; j < g.members.size(); ++j) {
      const int64_t i = g.members[j];
      B->hx[g.off + (int64_t)j] = const_cast<void*>(x[i]);
      B->hr[g.off + (int64_t)j] = rs[i];
      B->hk[g.off + (int64_t)j] = norm[(size_t)i].K;
      if (g.persist) {
        B->hpsig[ip] = persist_desc(g, (int64_t)j, x[i], rs[i]);
        // largest first: bins, then signal length
        porder.push_back({{-g.plan->M0, -g.plan->p.N}, (int)ip});
        ++ip;
      }
    }
  }
  std::stable_sort(porder.begin(), porder.end(),
                   [](const std::pair<std::pair<int64_t, int64_t>, int>& a,
                      const std::pair<std::pair<int64_t, int64_t>, int>& b) {
                     return a.first < b.first;
                   });
  for (int64_t k = 0; k < n_p; ++k) B->hporder[k] = porder[(size_t)k].second;
  e = cudaMemcpyAsync(B->x_tab, B->hx, n * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->r_tab, B->hr, n * sizeof(sft_result), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->k_tab, B->hk, n * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_p > 0)
    e = cudaMemcpyAsync(B->psig, B->hpsig, n_p * sizeof(sft::PSig), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n_p > 0)
    e = cudaMemcpyAsync(B->porder, B->hporder, n_p * sizeof(int), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(B->staged, st);
  // 4. autotune shape classes seen for the first time, and the persistent
  // kernel's CTA count on the first call with persistent signals
  if (e == cudaSuccess && B->autotune) {
    for (auto& kv : B->groups) {
      Group& g = kv.second;
      if (!g.members.empty() && !g.persist && !g.tuned) {
        drop_graph(B);
        e = tune_group(B, g, st);
        if (e != cudaSuccess) break;
      }
    }
    if (e == cudaSuccess && n_p > 0 && B->persist_ctas == 0 && B->persist_pick == 0 &&
        sft::persistent_ctas_per_sm() > 0) {
      drop_graph(B);
      e = tune_persist(B, (int)n_p, st);
    }
  }
  // (sets the kernel's shared-memory limit before any launch of it)
  const int per_sm = n_p > 0 ? std::max(1, sft::persistent_ctas_per_sm()) : 1;
  int pctas = B->persist_ctas;
  if (pctas <= 0) pctas = B->persist_pick;
  if (pctas <= 0) pctas = sm_count() * per_sm;
  // 5. replay the captured graph, or capture one for this composition
  std::vector<int64_t> comp;
  comp.push_back(n);
  comp.push_back(n_p);
  comp.push_back(n_p > 0 ? pctas : 0);
  for (auto& kv : B->groups) {
    const Group& g = kv.second;
    if (g.members.empty()) continue;
    comp.push_back(reinterpret_cast<int64_t>(g.plan));
    comp.push_back((int64_t)g.members.size());
    comp.push_back(g.off);
    comp.push_back(g.persist ? -1 : g.plan->dec_ctas_per_sm);
    comp.push_back(g.persist ? -1 : g.plan->fft_pts);
  }
  if (e == cudaSuccess && B->use_graph) {
    if (!B->exec || comp != B->comp) {
      drop_graph(B);
      // the graph is captured on a private stream and launched on `st`; the
      // persistent launch and the groups (independent plans and
      // workspaces) are spread over the lanes, largest first onto the
      // least-loaded lane, so that small groups run side by side
      e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = cudaEventRecord(B->fork_ev, B->cap_stream);
      for (int i = 0; e == cudaSuccess && i < sft_batch_s::kLanes; ++i)
        e = cudaStreamWaitEvent(B->lane[i], B->fork_ev, 0);
      double load[sft_batch_s::kLanes] = {};
      if (e == cudaSuccess && n_p > 0) {
        e = sft::launch_exact_persistent(B->psig, B->porder, (int)n_p, B->phead, pctas,
                                         B->lane[0]);
        for (auto& kv : B->groups)
          if (kv.second.persist && !kv.second.members.empty())
            load[0] += (double)kv.second.members.size() * (double)kv.second.plan->p.N;
      }
      std::vector<std::pair<double, Group*>> order;
      for (auto& kv : B->groups)
        if (!kv.second.members.empty() && !kv.second.persist)
          order.push_back({(double)kv.second.members.size() * (double)kv.second.plan->p.N,
                           &kv.second});
      std::sort(order.begin(), order.end(),
                [](const std::pair<double, Group*>& a, const std::pair<double, Group*>& b) {
                  return a.first > b.first;
                });
      for (auto& og : order) {
        if (e != cudaSuccess) break;
        int li = 0;
        for (int i = 1; i < sft_batch_s::kLanes; ++i)
          if (load[i] < load[li]) li = i;
        load[li] += og.first;
        e = enqueue_group(B, *og.second, B->lane[li]);
      }
      for (int i = 0; e == cudaSuccess && i < sft_batch_s::kLanes; ++i) {
        e = cudaEventRecord(B->join_ev[i], B->lane[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap_stream, B->join_ev[i], 0);
      }
      cudaGraph_t gph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(B->cap_stream, &gph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, gph, 0);
      if (e == cudaSuccess) {
        B->graph = gph;
        B->comp = comp;
        size_t nn = 0;
        cudaGraphGetNodes(gph, nullptr, &nn);
        B->graph_nodes = nn;
      } else if (gph) {
        cudaGraphDestroy(gph);
      }
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(B->exec, st);
  } else if (e == cudaSuccess) {
    if (n_p > 0)
      e = sft::launch_exact_persistent(B->psig, B->porder, (int)n_p, B->phead, pctas, st);
    for (auto& kv : B->groups)
      if (e == cudaSuccess && !kv.second.members.empty() && !kv.second.persist)
        e = enqueue_group(B, kv.second, st);
  }
  B->last_persist = n_p;
  B->last_persist_ctas = n_p > 0 ? std::min<int>(pctas, (int)n_p) : 0;
  B->last_groups = ngroups;
  if (e != cudaSuccess) {
    sft::set_error_detail(cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

}  // extern "C"
