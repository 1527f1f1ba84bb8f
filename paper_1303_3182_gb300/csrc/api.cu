// C ABI of libtqr (include/tqr.h): argument checks, plan cache, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/tqr.h"
#include "tqr_internal.h"

namespace tqr {

namespace {

std::mutex g_mu;
int64_t g_drop_edge = -1;  // test hook, see tqr_debug_drop_edge
// Claim order of factorization plans (tqr_set_claim_order): mode 0 or 1 as set, or
// the automatic default (mode 2): the bounded-processor CP-method order with built-in
// kernel weights for the tensor-core precisions and FP64, the unbounded-processor order
// for FP32.  The weights are task durations in microseconds measured on GB300:
//   tensor cores (nb 128, split-bf16 x6, the graph with preparation tasks): GEQRT ~236,
//   TTQRT ~239, UNMQR ~25, TTMQR ~28, TSQRT ~267, TSMQR ~28, preparation ~71 (panel
//   weights taken somewhat above their means, as a sweep on the 32768 x 4096 Greedy
//   factorization preferred), split-panel blocks about a quarter of a panel plus the
//   block's own tile loads - panels cost ten updates there, while the thesis's weights
//   give them less than an update;
//   FP64 (nb 256): 5146, 4249, 6394, 6369, TSQRT 6767, TSMQR 9457 - with them FlatTree's
//   32768 x 4096 factorization takes 1488 ms instead of 1635 ms with the unbounded order
//   (its ALAP Derived bound is 1468 ms).
int g_order_mode = 2;
int64_t g_order_w[kNumKinds] = {kWGeqrt, kWTtqrt, kWUnmqr, kWTtmqr, kWUnmqr, kWTtmqr, kWTsqrt, kWTsmqr, kWTsmqr,
                                 1, 1, 1, 2};
int g_order_gen = 0;        // bumped by every tqr_set_claim_order call
// per TaskKind: GEQRT, TTQRT, UNMQR, TTMQR, (apply-Q kinds, unused), TSQRT, TSMQR.  The
// TS kernels' weights are measured task means on GB300 as well: tensor cores 340-375 /
// 29-30 us (TSQRT taken like the tuned panel weights, a little above its mean), FP64
// 6767 / 9457 us (TSMQR 1.37 times faster per flop than UNMQR + TTMQR, as the thesis
// found the TS kernels faster on its CPUs).
constexpr int64_t kTensorOrderWeights[kNumKinds] = {265, 285, 20, 32, 20, 32, 320, 32, 32, 66, 66, 80, 85};
constexpr int64_t kFp64OrderWeights[kNumKinds] = {5146, 4249, 6394, 6369, 6394, 6369, 6767, 9457, 9457, 1, 1, 1, 1};

// Per-kind weights from the four TT-kernel weights of the ABI (GEQRT, TTQRT, UNMQR,
// TTMQR): the TS kernels take the thesis's ratios to their TT counterparts, TSQRT = 3
// TTQRT (6 against 2) and TSMQR = 2 TTMQR (12 against 6).
void expand_weights(const int64_t w4[4], int64_t out[kNumKinds]) {
  out[kGeqrt] = w4[0];
  out[kTtqrt] = w4[1];
  out[kUnmqr] = out[kUnmqrB] = w4[2];
  out[kTtmqr] = out[kTtmqrB] = w4[3];
  out[kTsqrt] = 3 * w4[1];
  out[kTsmqr] = out[kTsmqrB] = 2 * w4[3];
  out[kPrepG] = out[kPrepT] = 1;  // operand images (tensor-core precisions): short
  // a quarter of the TT / TS panel per 32-column block task
  out[kTtqrtS] = std::max<int64_t>(1, out[kTtqrt] / kPanelSplits);
  out[kTsqrtS] = std::max<int64_t>(1, out[kTsqrt] / kPanelSplits);
}

bool valid_tree(int tree) {
  if (tree & ~(kTreeTS | 15)) return false;
  const int b = tree_base(tree);
  return b >= TQR_FLAT && b <= TQR_ASAP;
}

OrderSpec effective_order(int prec) {
  OrderSpec spec;
  const int64_t *w = nullptr;
  if (g_order_mode == 1) {
    w = g_order_w;
    spec.id = 1 + g_order_gen;
  } else if (g_order_mode == 2 && is_tensor_prec(prec)) {
    w = kTensorOrderWeights;
    spec.id = -1;
  } else if (g_order_mode == 2 && prec == TQR_FP64) {
    w = kFp64OrderWeights;
    spec.id = -2;
  }
  if (w) {
    spec.mode = 1;
    for (int c = 0; c < kNumKinds; ++c) spec.w[c] = w[c];
  }
  return spec;
}
int g_debug_plans = 0;
thread_local std::string g_last_error;
int64_t g_wait_limit_ns = 20LL * 1000 * 1000 * 1000;
int g_sync = 1;
int g_timing = 0;
int g_trace = 0;
// device trace of the last traced executor run and the task table it refers to
int64_t *g_trace_buf = nullptr;
size_t g_trace_cap = 0;
std::vector<Task> g_trace_tasks;
// per kernel kind: accumulated device milliseconds and launch count (tqr_kernel_time)
double g_kernel_ms[4] = {0, 0, 0, 0};
int64_t g_kernel_launches[4] = {0, 0, 0, 0};

// Brackets one launch with CUDA events on its stream when timing is enabled; the
// elapsed time is added at the call's synchronization point.
struct LaunchTimer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int kind;
  LaunchTimer(int k, cudaStream_t st) : kind(k) {
    if (!g_timing) return;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
  }
  void stop(cudaStream_t st) {
    if (e1) cudaEventRecord(e1, st);
  }
  // call after the stream was synchronized
  void collect() {
    if (!e0) return;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
      g_kernel_ms[kind] += ms;
      g_kernel_launches[kind] += 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    e0 = e1 = nullptr;
  }
  ~LaunchTimer() { collect(); }
};

// A task graph uploaded to one device, plus its per-run state.
struct Plan {
  Graph g;
  int device = 0;
  int colparts = 1;  // update tasks split into column parts (SIMT factorization plans)
  Task *d_tasks = nullptr;
  int32_t *d_succ_ptr = nullptr, *d_succ_idx = nullptr, *d_indeg = nullptr;
  int32_t *d_counters = nullptr;
  int32_t *d_state = nullptr;  // [0] = ticket, [1] = status
  ~Plan() {
    cudaFree(d_tasks);
    cudaFree(d_succ_ptr);
    cudaFree(d_succ_idx);
    cudaFree(d_indeg);
    cudaFree(d_counters);
    cudaFree(d_state);
  }
};

// kind 0 = factorization, 1 = apply Q^T, 2 = apply Q
// device, kind, P, Q, tree, bs, claim-order identity (0: unbounded order; < 0: a built-in
// weight set; > 0: the generation of a user setting), processors
using PlanKey = std::tuple<int, int, int, int, int, int, int, int>;
std::map<PlanKey, std::unique_ptr<Plan>> g_plans;

struct Scratch {
  int32_t *flags = nullptr;  // trsm ticket + flags, and a status word at [cap]
  int cap = 0;
};
std::map<int, Scratch> g_scratch;

int cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return TQR_ECUDA;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &src) {
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Returns the cached plan for (kind, P, Q, tree, bs) on the current device.
// order: the claim order of a factorization plan (kind 0), with spec.nproc the
// executor's resident CTAs; ignored for the apply-Q plans.
// prep: the tensor-core form of a factorization graph (operand-preparation tasks); split:
// with its TT / TS panels as 32-column block tasks.
int get_plan(int kind, int P, int Q, int tree, int bs, Plan **out, const OrderSpec *order = nullptr,
             bool prep = false, bool split = false, int colparts = 1) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  const int64_t drop = kind == 0 ? g_drop_edge : -1;
  OrderSpec spec;
  if (order) spec = *order;
  spec.nproc = std::max(1, spec.nproc);
  const bool bounded = kind == 0 && spec.mode == 1;
  // the order's identity (spec.id: user weights carry the setting's generation, each
  // built-in weight set a negative key of its own) is part of the key; a plan built with
  // the test hook is never reused: it gets a key of its own
  const int form = kind == 0 && prep ? (split ? 4 : 3) : (kind == 0 && colparts > 1 ? 5 : kind);
  const PlanKey key{dev, drop >= 0 ? 100 + g_debug_plans++ : form, P, Q, tree,
                    tree_base(tree) == TQR_PLASMA ? bs : 0, bounded ? spec.id : 0, bounded ? spec.nproc : 0};
  auto it = g_plans.find(key);
  if (it != g_plans.end()) {
    *out = it->second.get();
    return TQR_OK;
  }
  std::vector<Elim> elims;
  if (!elimination_list(P, Q, tree_base(tree), bs, elims)) return -5;
  auto plan = std::make_unique<Plan>();
  plan->device = dev;
  if (kind == 0)
    build_factor_graph(P, Q, elims, plan->g, drop, bounded ? &spec : nullptr, tree_ts(tree), prep, prep && split,
                       colparts);
  else
    build_applyq_graph(P, Q, elims, kind == 2, plan->g, tree_ts(tree));
  plan->colparts = kind == 0 ? colparts : 1;
  if (drop >= 0) g_drop_edge = -1;  // the test hook applies to one plan only
  const Graph &g = plan->g;
  if ((e = upload(&plan->d_tasks, g.tasks)) != cudaSuccess ||
      (e = upload(&plan->d_succ_ptr, g.succ_ptr)) != cudaSuccess ||
      (e = upload(&plan->d_succ_idx, g.succ_idx)) != cudaSuccess ||
      (e = upload(&plan->d_indeg, g.indeg)) != cudaSuccess ||
      (e = cudaMalloc(&plan->d_counters, std::max<size_t>(1, g.tasks.size()) * sizeof(int32_t))) !=
          cudaSuccess ||
      (e = cudaMalloc(&plan->d_state, 2 * sizeof(int32_t))) != cudaSuccess) {
    g_last_error = std::string("plan upload: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TQR_ENOMEM : TQR_ECUDA;
  }
  *out = plan.get();
  g_plans.emplace(key, std::move(plan));
  return TQR_OK;
}

int get_scratch(int nflags, Scratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lock(g_mu);
  Scratch &s = g_scratch[dev];
  if (s.cap < nflags) {
    cudaFree(s.flags);
    s.flags = nullptr;
    s.cap = 0;
    e = cudaMalloc(&s.flags, (nflags + 1) * sizeof(int32_t));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TQR_ENOMEM : cuda_fail(e, "cudaMalloc");
    s.cap = nflags;
  }
  *out = &s;
  return TQR_OK;
}

// Reads a device status word after synchronizing the stream.
int read_status(int32_t *d_status, cudaStream_t st) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device execution");
  if (h != 0) {
    g_last_error = "device wait exceeded the limit at task " + std::to_string(h >> 8);
    return TQR_ETIMEOUT;
  }
  return TQR_OK;
}

// Runs a plan on the stream: reset counters / ticket / status, launch, check.
int run_plan(Plan *plan, ExecParams prm, bool dbl, cudaStream_t st) {
  const size_t n = plan->g.tasks.size();
  if (n == 0) return TQR_OK;
  cudaError_t e = cudaMemcpyAsync(plan->d_counters, plan->d_indeg, n * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(plan->d_state, 0, 2 * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "plan reset");
  prm.colparts = plan->colparts;
  prm.colw = static_cast<int>(ceil_div(prm.nb, prm.colparts));
  prm.tasks = plan->d_tasks;
  prm.succ_ptr = plan->d_succ_ptr;
  prm.succ_idx = plan->d_succ_idx;
  prm.counters = plan->d_counters;
  prm.next = plan->d_state;
  prm.status = plan->d_state + 1;
  prm.ntask = static_cast<int>(n);
  prm.wait_limit_ns = g_wait_limit_ns;
  prm.trace = nullptr;
  if (g_trace) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_trace_cap < n) {
      cudaFree(g_trace_buf);
      g_trace_buf = nullptr;
      g_trace_cap = 0;
      if (cudaMalloc(&g_trace_buf, n * 8 * sizeof(int64_t)) == cudaSuccess) g_trace_cap = n;
    }
    if (g_trace_buf) {
      prm.trace = g_trace_buf;
      g_trace_tasks = plan->g.tasks;
    }
  }
  LaunchTimer timer(prm.B ? 1 : 0, st);
  const int rc = launch_executor(prm, dbl, st);
  timer.stop(st);
  if (rc != 0) return cuda_fail(static_cast<cudaError_t>(rc), "executor launch");
  if (g_sync) return read_status(plan->d_state + 1, st);
  return TQR_OK;
}

}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

int64_t take_debug_drop_edge() {
  std::lock_guard<std::mutex> lock(g_mu);
  const int64_t e = g_drop_edge;
  g_drop_edge = -1;
  return e;
}

bool is_tensor_prec(int prec) {
  return prec == TQR_BF16 || prec == TQR_FP16 || prec == TQR_BF16X3 || prec == TQR_BF16X6;
}

// 16-bit parts per operand of a tensor-core precision.
int tensor_parts(int prec) { return prec == TQR_BF16X6 ? 3 : (prec == TQR_BF16X3 ? 2 : 1); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int check_tiles(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (nb < 1 || nb > 256) return -3;
  if (is_tensor_prec(prec) && nb != kMixedNB) return -3;
  if (ib < 1 || ib > nb || ib > 32) return -4;
  if (!valid_tree(tree)) return -5;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -6;
  if (prec < TQR_FP64 || prec > TQR_Z64) return -7;
  if (prec == TQR_Z64 && nb > 128) return -3;
  if (ceil_div(m, nb) > 32767 || ceil_div(n, nb) > 32767) return -3;
  return 0;
}

size_t ops_offset(int64_t m, int64_t n, int nb, int ib) {
  const int64_t P = ceil_div(m, nb), Q = ceil_div(n, nb), K = std::min(P, Q);
  return align_up(static_cast<size_t>(2 * P * K) * ib * nb * sizeof(float), 1024);
}

size_t factor_workspace_bytes(int64_t m, int64_t n, int nb, int ib, int prec) {
  const int64_t P = ceil_div(m, nb), Q = ceil_div(n, nb), K = std::min(P, Q);
  const size_t esz = prec == TQR_Z64 ? 2 * sizeof(double) : (prec == TQR_FP64 ? sizeof(double) : sizeof(float));
  if (!is_tensor_prec(prec)) return static_cast<size_t>(2 * P * K) * ib * nb * esz;
  return ops_offset(m, n, nb, ib) + static_cast<size_t>(2 * P * K) * mixed_slot_bytes(tensor_parts(prec));
}


namespace {
std::atomic<int64_t> g_launch_count{0};
}
void count_launch(int64_t k) { g_launch_count.fetch_add(k, std::memory_order_relaxed); }
int64_t wait_limit_ns() { return g_wait_limit_ns; }
bool sync_enabled() { return g_sync != 0; }

}  // namespace tqr

using namespace tqr;

extern "C" {

int tqr_elimlist(int p, int q, int tree, int bs, int32_t *list, int64_t *len, int64_t *cp_units) {
  if (p < 1) return -1;
  if (q < 1) return -2;
  if (!valid_tree(tree)) return -3;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -4;
  if (!len) return -6;
  std::vector<Elim> elims;
  try {
    elimination_list(p, q, tree_base(tree), bs, elims);
    const int64_t E = static_cast<int64_t>(elims.size());
    if (list) {
      if (*len < E) return -6;
      for (int64_t e = 0; e < E; ++e) {
        list[3 * e + 0] = elims[e].k;
        list[3 * e + 1] = elims[e].i;
        list[3 * e + 2] = elims[e].piv;
      }
    }
    *len = E;
    if (cp_units) {
      Graph g;
      build_factor_graph(p, q, elims, g, -1, nullptr, tree_ts(tree));
      *cp_units = g.critical_path;
    }
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  } catch (...) {
    g_last_error = "internal error in tqr_elimlist";
    return TQR_ECUDA;
  }
  return TQR_OK;
}

}  // extern "C"

namespace tqr {
namespace {
// Per-kind weights from 6 weights of the ABI (GEQRT, TTQRT, UNMQR, TTMQR, TSQRT, TSMQR).
void weights6(const int64_t w6[6], int64_t out[kNumKinds]) {
  expand_weights(w6, out);
  out[kTsqrt] = w6[4];
  out[kTsmqr] = out[kTsmqrB] = w6[5];
  out[kTsqrtS] = std::max<int64_t>(1, w6[4] / kPanelSplits);
}

int schedule_impl(int p, int q, int tree, int bs, int nproc, const int64_t w[kNumKinds], int64_t *makespan,
                  int64_t *alap_bound, int64_t *lost_area, bool prep = false, bool split = false) {
  try {
    std::vector<Elim> elims;
    elimination_list(p, q, tree_base(tree), bs, elims);
    GraphBuilder b(p * q * kRegionsPerTile);
    add_factor_program(b, p, q, elims, tree_ts(tree), prep, split);
    const int n = static_cast<int>(b.tasks.size());
    std::vector<std::vector<int32_t>> succ(n);
    std::vector<int32_t> npred(n);
    std::vector<int64_t> wt(n);
    for (int t = 0; t < n; ++t) {
      npred[t] = static_cast<int32_t>(b.preds[t].size());
      for (int32_t x : b.preds[t]) succ[x].push_back(t);
      wt[t] = w[b.tasks[t].kind];
    }
    const std::vector<int64_t> prio = backflow_priorities(succ, wt);
    if (makespan) *makespan = cp_list_schedule(succ, npred, wt, prio, nproc, nullptr);
    int64_t la = 0;
    const int64_t bound = alap_derived_bound(wt, prio, nproc, &la);
    if (alap_bound) *alap_bound = bound;
    if (lost_area) *lost_area = la;
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  } catch (...) {
    g_last_error = "internal error in tqr_schedule";
    return TQR_ECUDA;
  }
  return TQR_OK;
}

int set_claim_order_impl(int mode, const int64_t w[kNumKinds]) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_order_mode = mode;
  for (int c = 0; c < kNumKinds; ++c) g_order_w[c] = w[c];
  ++g_order_gen;
  return TQR_OK;
}
}  // namespace
}  // namespace tqr

extern "C" {

int tqr_schedule(int p, int q, int tree, int bs, int nproc, const int64_t *weights, int64_t *makespan,
                 int64_t *alap_bound, int64_t *lost_area) {
  if (p < 1) return -1;
  if (q < 1) return -2;
  if (!valid_tree(tree)) return -3;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -4;
  if (nproc < 1) return -5;
  int64_t w4[4] = {kWGeqrt, kWTtqrt, kWUnmqr, kWTtmqr}, w[kNumKinds];
  if (weights)
    for (int c = 0; c < 4; ++c) {
      if (weights[c] < 1) return -6;
      w4[c] = weights[c];
    }
  expand_weights(w4, w);
  return schedule_impl(p, q, tree, bs, nproc, w, makespan, alap_bound, lost_area);
}

int tqr_schedule_ts(int p, int q, int tree, int bs, int nproc, const int64_t *weights, int64_t *makespan,
                    int64_t *alap_bound, int64_t *lost_area) {
  if (p < 1) return -1;
  if (q < 1) return -2;
  if (!valid_tree(tree)) return -3;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -4;
  if (nproc < 1) return -5;
  if (!weights) return -6;
  for (int c = 0; c < 6; ++c)
    if (weights[c] < 1) return -6;
  for (int c = 6; c < 9; ++c)
    if (weights[c] < 0) return -6;
  const bool prep = weights[6] > 0, split = prep && weights[7] > 0 && weights[8] > 0;
  int64_t w[kNumKinds];
  weights6(weights, w);
  w[kPrepG] = w[kPrepT] = weights[6];
  if (split) {
    w[kTtqrtS] = weights[7];
    w[kTsqrtS] = weights[8];
  }
  return schedule_impl(p, q, tree, bs, nproc, w, makespan, alap_bound, lost_area, prep, split);
}

int tqr_set_claim_order(int mode, const int64_t *weights) {
  if (mode < 0 || mode > 2) return -1;
  int64_t w4[4] = {kWGeqrt, kWTtqrt, kWUnmqr, kWTtmqr}, w[kNumKinds];
  if (weights && mode == 1)
    for (int c = 0; c < 4; ++c) {
      if (weights[c] < 1) return -2;
      w4[c] = weights[c];
    }
  expand_weights(w4, w);
  return set_claim_order_impl(mode, w);
}

int tqr_set_claim_order_ts(int mode, const int64_t *weights) {
  if (mode < 0 || mode > 2) return -1;
  int64_t w6[6] = {kWGeqrt, kWTtqrt, kWUnmqr, kWTtmqr, kWTsqrt, kWTsmqr}, w[kNumKinds];
  if (weights && mode == 1)
    for (int c = 0; c < 6; ++c) {
      if (weights[c] < 1) return -2;
      w6[c] = weights[c];
    }
  weights6(w6, w);
  return set_claim_order_impl(mode, w);
}

int tqr_debug_split_pairs(int64_t n, const double *x, float *hi, float *lo) {
  if (n < 0) return -1;
  if (n > 0 && (!x || !hi || !lo)) return -2;
  for (int64_t i = 0; i < n; ++i) split_pair(x[i], hi[i], lo[i]);
  return TQR_OK;
}

int tqr_set_claim_order_tc(int mode, const int64_t *weights) {
  if (mode < 0 || mode > 2) return -1;
  int64_t w[kNumKinds];
  for (int c = 0; c < kNumKinds; ++c) w[c] = kTensorOrderWeights[c];
  if (weights && mode == 1) {
    for (int c = 0; c < 9; ++c)
      if (weights[c] < 1) return -2;
    weights6(weights, w);
    w[kPrepG] = w[kPrepT] = weights[6];
    w[kTtqrtS] = weights[7];
    w[kTsqrtS] = weights[8];
  }
  return set_claim_order_impl(mode, w);
}

namespace {
int g_colparts_mode = 1;  // tqr_set_column_parts: 0 never, 1 automatic, 2 always

// Column parts of a SIMT factorization plan: kColParts slices (each at least one 16- or
// 32-column chunk of the update kernels) when the graph's update tasks, split, still fit
// on the GPU's SMs at once - a graph that small is bound by its critical path, on which
// every update then runs on several SMs - or always (mode 2); else 1.
int column_parts(int P, int Q, int nb, bool dbl) {
  int mode;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    mode = g_colparts_mode;
  }
  if (mode == 0 || Q < 2 || Q >= (1 << kColShift)) return 1;
  const int chunk = dbl ? 16 : 32;
  const int parts = std::min<int>(kColParts, static_cast<int>(ceil_div(nb, chunk)));
  if (parts < 2) return 1;
  if (mode == 2) return parts;
  // updates of the TT program: for panel k, (P - k) UNMQR and (P - k - 1) TTMQR per later column
  int64_t nupd = 0;
  for (int k = 0; k < std::min(P, Q); ++k) nupd += static_cast<int64_t>(2 * (P - k) - 1) * (Q - k - 1);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return 1;
  return nupd * parts <= nsm ? parts : 1;
}
}  // namespace

int tqr_set_column_parts(int mode) {
  if (mode < 0 || mode > 2) return -1;
  std::lock_guard<std::mutex> lock(g_mu);
  g_colparts_mode = mode;
  return TQR_OK;
}

int tqr_workspace_size(int64_t m, int64_t n, int nb, int ib, int prec, size_t *T_bytes) {
  const int rc = check_tiles(m, n, nb, ib, TQR_GREEDY, 1, prec);
  if (rc) return rc;
  if (!T_bytes) return -6;
  *T_bytes = factor_workspace_bytes(m, n, nb, ib, prec);
  return TQR_OK;
}

int tqr_factor(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec, void *A, int64_t lda,
               void *T, void *stream) {
  int rc = check_tiles(m, n, nb, ib, tree, bs, prec);
  if (rc) return rc;
  if (!A) return -8;
  if (lda < m) return -9;
  if (!T) return -10;
  const bool dbl = prec == TQR_FP64;
  if (prec == TQR_Z64 ? zexecutor_smem_bytes(nb, ib) == 0
                      : (!is_tensor_prec(prec) && executor_smem_bytes(nb, ib, dbl, false) == 0)) {
    g_last_error = "nb/ib too large for one SM's shared memory";
    return TQR_EUNSUPPORTED;
  }
  try {
    const int P = static_cast<int>(ceil_div(m, nb)), Q = static_cast<int>(ceil_div(n, nb));
    Plan *plan = nullptr;
    OrderSpec order;
    {
      std::lock_guard<std::mutex> lock(g_mu);
      order = effective_order(prec);
    }
    if (order.mode == 1)
      order.nproc = prec == TQR_Z64 ? zexec_slots(nb, ib) : executor_slots(dbl, is_tensor_prec(prec), nb, ib);
    // tensor-core graphs split their TT / TS panels into 32-column block tasks when the
    // inner block divides 32; small SIMT graphs split their updates into column parts
    const bool tensor = is_tensor_prec(prec);
    const int cparts = tensor || prec == TQR_Z64 ? 1 : column_parts(P, Q, nb, dbl);
    if ((rc = get_plan(0, P, Q, tree, bs, &plan, &order, tensor, tensor && kPanelSplitCols % ib == 0, cparts)) != 0)
      return rc;
    ExecParams prm{};
    prm.A = A;
    prm.lda = lda;
    prm.m = m;
    prm.n = n;
    prm.nb = nb;
    prm.ib = ib;
    prm.P = P;
    prm.Q = Q;
    prm.T = T;
    prm.B = nullptr;
    prm.cplx = prec == TQR_Z64 ? 1 : 0;
    if (is_tensor_prec(prec)) {
      prm.mixed = 1;
      prm.ops = static_cast<char *>(T) + ops_offset(m, n, nb, ib);
      prm.nparts = tensor_parts(prec);
      prm.vec4 = (reinterpret_cast<uintptr_t>(A) % 16 == 0 && lda % 4 == 0) ? 1 : 0;
      prm.fmt = prec == TQR_FP16 ? 0 : 1;
    }
    return run_plan(plan, prm, dbl, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  }
}

int tqr_apply_qt(int64_t m, int64_t n, int nb, int ib, int tree, int bs, int prec, int trans,
                 const void *A, int64_t lda, const void *T, double *B, int64_t ldb, int64_t nrhs,
                 void *stream) {
  int rc = check_tiles(m, n, nb, ib, tree, bs, prec);
  if (rc) return rc;
  if (trans != 0 && trans != 1) return -8;
  if (!A) return -9;
  if (lda < m) return -10;
  if (!T) return -11;
  if (!B) return -12;
  if (ldb < m) return -13;
  if (nrhs < 0) return -14;
  if (nrhs == 0) return TQR_OK;
  const bool dbl = prec == TQR_FP64;
  if (prec == TQR_Z64 ? zexecutor_smem_bytes(nb, ib) == 0 : executor_smem_bytes(nb, ib, dbl, true) == 0)
    return TQR_EUNSUPPORTED;
  try {
    const int P = static_cast<int>(ceil_div(m, nb)), Q = static_cast<int>(ceil_div(n, nb));
    Plan *plan = nullptr;
    if ((rc = get_plan(trans ? 2 : 1, P, Q, tree, bs, &plan)) != 0) return rc;
    ExecParams prm{};
    prm.A = const_cast<void *>(A);
    prm.lda = lda;
    prm.m = m;
    prm.n = n;
    prm.nb = nb;
    prm.ib = ib;
    prm.P = P;
    prm.Q = Q;
    prm.T = const_cast<void *>(T);
    prm.B = B;
    prm.ldb = ldb;
    prm.nrhs = nrhs;
    prm.trans = trans;
    prm.cplx = prec == TQR_Z64 ? 1 : 0;
    return run_plan(plan, prm, dbl, static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  }
}

int tqr_trsm(int64_t n, int prec, const void *A, int64_t lda, double *B, int64_t ldb, int64_t nrhs,
             void *stream) {
  if (n < 1) return -1;
  if (prec < TQR_FP64 || prec > TQR_Z64) return -2;
  if (!A) return -3;
  if (lda < n) return -4;
  if (!B) return -5;
  if (ldb < n) return -6;
  if (nrhs < 0) return -7;
  if (nrhs == 0) return TQR_OK;
  if (prec == TQR_Z64) {
    cudaStream_t zst = static_cast<cudaStream_t>(stream);
    LaunchTimer ztimer(2, zst);
    const int zrc = launch_ztrsm(n, A, lda, B, ldb, nrhs, stream);
    ztimer.stop(zst);
    if (zrc) return cuda_fail(static_cast<cudaError_t>(zrc), "complex trsm launch");
    if (g_sync) {
      const cudaError_t e = cudaStreamSynchronize(zst);
      if (e != cudaSuccess) return cuda_fail(e, "complex trsm");
    }
    return TQR_OK;
  }
  Scratch *s = nullptr;
  const int nflags = trsm_flag_count(n);
  int rc = get_scratch(nflags, &s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t *status = s->flags + s->cap;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "trsm reset");
  LaunchTimer timer(2, st);
  rc = launch_trsm(n, A, lda, prec == TQR_FP64, B, ldb, nrhs, s->flags, status, g_wait_limit_ns, st);
  timer.stop(st);
  if (rc) return cuda_fail(static_cast<cudaError_t>(rc), "trsm launch");
  if (g_sync) return read_status(status, st);
  return TQR_OK;
}

int tqr_lstsq_workspace_size(int64_t m, int64_t n, int64_t nrhs, int nb, int ib, int prec, size_t *bytes) {
  int rc = check_tiles(m, n, nb, ib, TQR_GREEDY, 1, prec);
  if (rc) return rc;
  if (nrhs < 0) return -3;
  if (!bytes) return -7;
  size_t tb = 0;
  if ((rc = tqr_workspace_size(m, n, nb, ib, prec, &tb)) != 0) return rc;
  const size_t nr = static_cast<size_t>(std::max<int64_t>(nrhs, 1));
  if (prec == TQR_FP64 || prec == TQR_Z64) {
    const size_t esz = prec == TQR_Z64 ? 2 * sizeof(double) : sizeof(double);
    *bytes = align_up(static_cast<size_t>(m) * n * esz, 256) + align_up(tb, 256) +
             align_up(static_cast<size_t>(m) * nr * esz, 256);
  } else {
    const size_t ldf = align_up(static_cast<size_t>(m), 32);
    const size_t nr64 = std::min<size_t>(nr, 64);
    *bytes = align_up(ldf * n * sizeof(float), 1024) + align_up(tb, 1024) +
             align_up(static_cast<size_t>(m) * nr * sizeof(double), 1024) +
             align_up(lsqr_work_doubles(m, n, static_cast<int>(nr64)) * sizeof(double), 1024);
  }
  return TQR_OK;
}

int tqr_lstsq(int64_t m, int64_t n, int64_t nrhs, int nb, int ib, int tree, int bs, int prec,
              const double *A, int64_t lda, const double *B, int64_t ldb, double *X, int64_t ldx,
              double tol, int max_iter, int *iters, void *workspace, size_t ws_bytes, void *stream) {
  if (m < 1) return -1;
  if (n < 1 || n > m) return -2;
  if (nrhs < 0) return -3;
  int rc = check_tiles(m, n, nb, ib, tree, bs, prec);
  if (rc) return rc == -1 ? -1 : (rc == -2 ? -2 : rc - 1);
  if (!A) return -9;
  if (lda < m) return -10;
  if (!B || ldb < m) return -11;
  if (!X || ldx < n) return -13;
  if (iters) *iters = 0;
  if (nrhs == 0) return TQR_OK;
  size_t need = 0;
  if ((rc = tqr_lstsq_workspace_size(m, n, nrhs, nb, ib, prec, &need)) != 0) return rc;
  if (!workspace || ws_bytes < need) return -18;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *ws = static_cast<char *>(workspace);
  size_t tb = 0;
  tqr_workspace_size(m, n, nb, ib, prec, &tb);
  if (prec == TQR_FP64 || prec == TQR_Z64) {
    // plain QR solve: X = R^{-1} (Q^T B)(0:n) (Q^H for the complex precision); elements of
    // esz bytes (complex: interleaved pairs, leading dimensions in complex elements)
    const size_t esz = prec == TQR_Z64 ? 2 * sizeof(double) : sizeof(double);
    char *Aw = ws;
    void *Tw = ws + align_up(static_cast<size_t>(m) * n * esz, 256);
    double *Bw = reinterpret_cast<double *>(static_cast<char *>(Tw) + align_up(tb, 256));
    cudaError_t e = cudaMemcpy2DAsync(Aw, m * esz, A, lda * esz, m * esz, n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Bw, m * esz, B, ldb * esz, m * esz, nrhs, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "lstsq copy-in");
    if ((rc = tqr_factor(m, n, nb, ib, tree, bs, prec, Aw, m, Tw, stream)) != 0) return rc;
    if ((rc = tqr_apply_qt(m, n, nb, ib, tree, bs, prec, 0, Aw, m, Tw, Bw, m, nrhs, stream)) != 0) return rc;
    if ((rc = tqr_trsm(n, prec, Aw, m, Bw, m, nrhs, stream)) != 0) return rc;
    e = cudaMemcpy2DAsync(X, ldx * esz, Bw, m * esz, n * esz, nrhs, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "lstsq copy-out");
    if (g_sync) {
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "lstsq");
    }
    return TQR_OK;
  }
  // low-precision factorization of an FP32 copy, then FP64 LSQR refinement
  const int64_t ldf = static_cast<int64_t>(align_up(static_cast<size_t>(m), 32));
  float *Af = reinterpret_cast<float *>(ws);
  char *p = ws + align_up(static_cast<size_t>(ldf) * n * sizeof(float), 1024);
  void *Tw = p;
  p += align_up(tb, 1024);
  double *Bw = reinterpret_cast<double *>(p);
  p += align_up(static_cast<size_t>(m) * nrhs * sizeof(double), 1024);
  double *lw = reinterpret_cast<double *>(p);
  int rcv = lsqr_prepare(m, n, A, lda, Af, ldf, lw, stream);
  if (rcv) return cuda_fail(static_cast<cudaError_t>(rcv), "lstsq prepare");
  if ((rc = tqr_factor(m, n, nb, ib, tree, bs, prec, Af, ldf, Tw, stream)) != 0) return rc;
  // LSQR starts from x0 = 0: with R as preconditioner a few extra iterations cost less
  // than forming x0 = R^{-1} (Q^T b)(0:n) by a pass over all reflectors
  (void)Bw;
  cudaError_t e = cudaMemset2DAsync(X, ldx * sizeof(double), 0, n * sizeof(double), nrhs, st);
  if (e != cudaSuccess) return cuda_fail(e, "lstsq init");
  Scratch *s = nullptr;
  if ((rc = get_scratch(trsm_flag_count(n), &s)) != 0) return rc;
  int32_t *status = s->flags + s->cap;
  e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_fail(e, "lstsq reset");
  int worst_iters = 0;
  bool converged = true;
  LaunchTimer timer(3, st);
  for (int64_t r0 = 0; r0 < nrhs; r0 += 64) {
    const int nr = static_cast<int>(std::min<int64_t>(64, nrhs - r0));
    int it = 0;
    const int lrc = lsqr_refine(m, n, nr, A, lda, Af, ldf, B + r0 * ldb, ldb, X + r0 * ldx, ldx,
                                tol > 0 ? tol : 1e-14, max_iter > 0 ? max_iter : 100, &it, r0 == 0, true, lw, s->flags, status,
                                g_wait_limit_ns, stream);
    if (lrc > 0) return cuda_fail(static_cast<cudaError_t>(lrc), "lstsq refinement");
    if (lrc < 0) converged = false;
    worst_iters = std::max(worst_iters, it);
  }
  timer.stop(st);
  if (iters) *iters = worst_iters;
  if ((rc = read_status(status, st)) != 0) return rc;
  if (!converged) g_last_error = "refinement reached max_iter before ||A^T r|| / (||A|| ||r||) <= tol";
  return converged ? TQR_OK : TQR_ENOCONV;
}

double tqr_nominal_flops(int64_t m, int64_t n) {
  const double M = static_cast<double>(m), N = static_cast<double>(n);
  return 2.0 * N * N * (M - N / 3.0);
}

int64_t tqr_set_wait_limit_ns(int64_t ns) {
  const int64_t old = g_wait_limit_ns;
  if (ns > 0) g_wait_limit_ns = ns;
  return old;
}

int tqr_set_sync(int on) {
  const int old = g_sync;
  g_sync = on ? 1 : 0;
  return old;
}

int tqr_sync_status(void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  for (auto &kv : g_plans) {
    if (kv.second->device != dev) continue;
    int32_t h = 0;
    e = cudaMemcpy(&h, kv.second->d_state + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "status read");
    if (h != 0) return TQR_ETIMEOUT;
  }
  return TQR_OK;
}

const char *tqr_strerror(int status) {
  if (status < 0) return "invalid argument";
  switch (status) {
    case TQR_OK: return "success";
    case TQR_ECUDA: return "CUDA error";
    case TQR_ENOMEM: return "out of memory";
    case TQR_ETIMEOUT: return "device dependency wait exceeded the limit";
    case TQR_ENOCONV: return "iterative refinement did not converge";
    case TQR_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char *tqr_last_error(void) { return g_last_error.c_str(); }

void tqr_finalize(void) {
  reset_static_scratch();
  forget_autotune();
  std::lock_guard<std::mutex> lock(g_mu);
  g_plans.clear();
  for (auto &kv : g_scratch) cudaFree(kv.second.flags);
  g_scratch.clear();
  cudaFree(g_trace_buf);
  g_trace_buf = nullptr;
  g_trace_cap = 0;
  g_trace_tasks.clear();
}

int tqr_plan_stats(int64_t m, int64_t n, int nb, int tree, int bs, int64_t out[6]) {
  int64_t all[8];
  const int rc = tqr_plan_counts(m, n, nb, tree, bs, out ? all : nullptr);
  if (rc) return rc;
  for (int c = 0; c < 4; ++c) out[c] = all[c];
  out[4] = all[6];
  out[5] = all[7];
  return TQR_OK;
}

int tqr_plan_counts(int64_t m, int64_t n, int nb, int tree, int bs, int64_t out[8]) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (nb < 1) return -3;
  if (!valid_tree(tree)) return -4;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -5;
  if (!out) return -6;
  const int P = static_cast<int>(ceil_div(m, nb)), Q = static_cast<int>(ceil_div(n, nb));
  std::vector<Elim> elims;
  elimination_list(P, Q, tree_base(tree), bs, elims);
  Graph g;
  build_factor_graph(P, Q, elims, g, -1, nullptr, tree_ts(tree));
  for (int c = 0; c < 4; ++c) out[c] = g.counts[c];
  out[4] = g.counts[kTsqrt];
  out[5] = g.counts[kTsmqr];
  out[6] = static_cast<int64_t>(g.succ_idx.size());
  out[7] = g.critical_path;
  return TQR_OK;
}

int tqr_set_timing(int on) {
  const int old = g_timing;
  g_timing = on ? 1 : 0;
  return old;
}

int tqr_kernel_time(int kind, double *ms_total, int64_t *launches, int reset) {
  if (kind < 0 || kind > 3) return -1;
  if (ms_total) *ms_total = g_kernel_ms[kind];
  if (launches) *launches = g_kernel_launches[kind];
  if (reset) {
    g_kernel_ms[kind] = 0.0;
    g_kernel_launches[kind] = 0;
  }
  return TQR_OK;
}

int tqr_set_trace(int on) {
  const int old = g_trace;
  g_trace = on ? 1 : 0;
  return old;
}

int64_t tqr_trace_fetch(int64_t *out, int64_t cap) {
  std::lock_guard<std::mutex> lock(g_mu);
  const int64_t n = static_cast<int64_t>(g_trace_tasks.size());
  if (!out) return n;
  if (cap < n || !g_trace_buf) return -1;
  std::vector<int64_t> stamps(static_cast<size_t>(n) * 8);
  if (cudaMemcpy(stamps.data(), g_trace_buf, stamps.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return -2;
  for (int64_t t = 0; t < n; ++t) {
    const Task &k = g_trace_tasks[t];
    int64_t *o = out + 12 * t;
    o[0] = k.kind;
    o[1] = k.i;
    o[2] = k.piv;
    o[3] = static_cast<int64_t>(k.k) | (static_cast<int64_t>(k.j) << 16);
    for (int q = 0; q < 8; ++q) o[4 + q] = stamps[8 * t + q];
  }
  return n;
}

int64_t tqr_launch_count(int reset) {
  const int64_t v = reset ? g_launch_count.exchange(0) : g_launch_count.load();
  return v;
}

void tqr_debug_drop_edge(int64_t e) {
  std::lock_guard<std::mutex> lock(g_mu);
  g_drop_edge = e;
}

int tqr_debug_claim_order(int p, int q, int tree, int bs, int mode, int nproc, const int64_t *weights,
                          int32_t *tasks, int64_t *ntask) {
  if (p < 1) return -1;
  if (q < 1) return -2;
  if (!valid_tree(tree)) return -3;
  if (tree_base(tree) == TQR_PLASMA && bs < 1) return -4;
  if (mode != 0 && mode != 1) return -5;
  if (nproc < 1) return -6;
  if (!ntask) return -8;
  OrderSpec spec;
  spec.mode = mode;
  spec.nproc = nproc;
  if (weights) {
    int64_t w4[4];
    for (int c = 0; c < 4; ++c) {
      if (weights[c] < 1) return -7;
      w4[c] = weights[c];
    }
    expand_weights(w4, spec.w);
  }
  try {
    std::vector<Elim> elims;
    elimination_list(p, q, tree_base(tree), bs, elims);
    Graph g;
    build_factor_graph(p, q, elims, g, -1, mode == 1 ? &spec : nullptr, tree_ts(tree));
    const int64_t n = static_cast<int64_t>(g.tasks.size());
    if (tasks) {
      if (*ntask < n) return -8;
      for (int64_t t = 0; t < n; ++t) {
        const Task &x = g.tasks[t];
        tasks[5 * t + 0] = x.kind;
        tasks[5 * t + 1] = x.i;
        tasks[5 * t + 2] = x.piv;
        tasks[5 * t + 3] = x.k;
        tasks[5 * t + 4] = x.j;
      }
    }
    *ntask = n;
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  } catch (...) {
    g_last_error = "internal error in tqr_debug_claim_order";
    return TQR_ECUDA;
  }
  return TQR_OK;
}

}  // extern "C"
