// sft_batch.cu -- many signals of uneven N, K and kind in one call.
//
// Signals are grouped by shape (everything that fixes the launch sequence:
// N, d, mode, precision, a_max, levels, random shifts, tolerances; K is
// per signal).  Each group owns an internal plan.  The kernels of a group
// read every signal's input pointer, result buffers and K from device
// tables, so any set of buffers can be batched without copies.  The whole
// call -- the group launches back to back -- is captured once into a CUDA
// graph and replayed while the batch composition stays the same; only the
// tables are refreshed per call.  On the first call of a shape an
// autotuner times the queue decoders at 2, 4, 8 and 16 CTAs per SM on that
// call's own data and keeps the fastest.
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
};

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

// Times the group at 2, 4, 8, 16 decode CTAs per SM and keeps the fastest.
cudaError_t tune_group(sft_batch_s* B, Group& g, cudaStream_t s) {
  const int cands[4] = {2, 4, 8, 16};
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 1e30f;
  int pick = 8;
  cudaError_t e = cudaSuccess;
  for (int c : cands) {
    g.plan->dec_ctas_per_sm = c;
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
      pick = c;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  g.plan->dec_ctas_per_sm = pick;
  g.tuned = true;
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

int32_t sft_batch_info(sft_batch_t B, int32_t* n_groups, int64_t* n_graph_nodes, int32_t* n_tuned) {
  if (!B) return -1;
  if (n_groups) *n_groups = B->last_groups;
  if (n_graph_nodes) *n_graph_nodes = (int64_t)B->graph_nodes;
  if (n_tuned) *n_tuned = B->tuned;
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
  // 2. a plan with enough capacity for every group in use
  int32_t ngroups = 0;
  int64_t off = 0;
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
    g.off = off;
    off += size;
  }
  // 3. per-signal tables (pinned staging -> device, ordered before the launches)
  cudaError_t e = grow_tables(B, n);
  if (e == cudaSuccess) e = cudaEventSynchronize(B->staged);  // staging free again
  if (e != cudaSuccess) {
    sft::set_error_detail(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SFT_ENOMEM : SFT_ECUDA;
  }
  for (auto& kv : B->groups) {
    Group& g = kv.second;
    for (size_t j = 0; j < g.members.size(); ++j) {
      const int64_t i = g.members[j];
      B->hx[g.off + (int64_t)j] = const_cast<void*>(x[i]);
      B->hr[g.off + (int64_t)j] = rs[i];
      B->hk[g.off + (int64_t)j] = norm[(size_t)i].K;
    }
  }
  e = cudaMemcpyAsync(B->x_tab, B->hx, n * sizeof(void*), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->r_tab, B->hr, n * sizeof(sft_result), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->k_tab, B->hk, n * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(B->staged, st);
  // 4. autotune shapes seen for the first time
  if (e == cudaSuccess && B->autotune) {
    for (auto& kv : B->groups) {
      Group& g = kv.second;
      if (!g.members.empty() && !g.tuned) {
        drop_graph(B);
        e = tune_group(B, g, st);
        ++B->tuned;
        if (e != cudaSuccess) break;
      }
    }
  }
  // 5. replay the captured graph, or capture one for this composition
  std::vector<int64_t> comp;
  comp.push_back(n);
  for (auto& kv : B->groups) {
    const Group& g = kv.second;
    if (g.members.empty()) continue;
    comp.push_back(reinterpret_cast<int64_t>(g.plan));
    comp.push_back((int64_t)g.members.size());
    comp.push_back(g.off);
    comp.push_back(g.plan->dec_ctas_per_sm);
  }
  if (e == cudaSuccess && B->use_graph) {
    if (!B->exec || comp != B->comp) {
      drop_graph(B);
      // the graph is captured on a private stream and launched on `st`; the
      // groups (independent plans and workspaces) are spread over the lanes,
      // largest first onto the least-loaded lane, so that small groups run
      // side by side
      e = cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) e = cudaEventRecord(B->fork_ev, B->cap_stream);
      for (int i = 0; e == cudaSuccess && i < sft_batch_s::kLanes; ++i)
        e = cudaStreamWaitEvent(B->lane[i], B->fork_ev, 0);
      std::vector<std::pair<double, Group*>> order;
      for (auto& kv : B->groups)
        if (!kv.second.members.empty())
          order.push_back({(double)kv.second.members.size() * (double)kv.second.plan->p.N,
                           &kv.second});
      std::sort(order.begin(), order.end(),
                [](const std::pair<double, Group*>& a, const std::pair<double, Group*>& b) {
                  return a.first > b.first;
                });
      double load[sft_batch_s::kLanes] = {};
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
    for (auto& kv : B->groups)
      if (e == cudaSuccess && !kv.second.members.empty()) e = enqueue_group(B, kv.second, st);
  }
  B->last_groups = ngroups;
  if (e != cudaSuccess) {
    sft::set_error_detail(cudaGetErrorString(e));
    return SFT_ECUDA;
  }
  return SFT_OK;
}

}  // extern "C"
