// Batched factorization: the task graphs of many independent matrices merged into one
// task table and run by one persistent executor launch (optionally replayed from a
// CUDA graph).  Each matrix's graph is the graph of Algorithm "elimTR" for its own tile
// size and elimination list (Section 3.1.1, dependencies Eq. ttdeps / ttdeps2); the
// thesis factors one matrix at a time, so the merge order below is this library's own.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tqr.h"
#include "tqr_internal.h"

struct tqr_batch_plan {
  int device = 0;
  int prec = 0;
  int nmat = 0;
  int64_t ntask = 0, nedge = 0;
  int slots = 0;
  int max_nb = 1, max_ib = 1;
  double flops = 0.0;
  tqr::Task *d_tasks = nullptr;
  int32_t *d_mat_of = nullptr, *d_succ_ptr = nullptr, *d_succ_idx = nullptr, *d_indeg = nullptr;
  int32_t *d_counters = nullptr, *d_state = nullptr;  // state: [0] ticket, [1] status
  tqr::BatchMat *d_mats = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~tqr_batch_plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cudaFree(d_tasks);
    cudaFree(d_mat_of);
    cudaFree(d_succ_ptr);
    cudaFree(d_succ_idx);
    cudaFree(d_indeg);
    cudaFree(d_counters);
    cudaFree(d_state);
    cudaFree(d_mats);
  }
};

namespace tqr {
namespace {

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Built-in size classes (used where no tuning table row covers a matrix).  Tensor-core
// precisions have one tile size.  For FP64/FP32 the per-class autotuner (rows 256..8192,
// columns 32..256) chose the largest tile, 256 (fewest tasks: every task's panel work is
// latency-bound), ib 32, and Greedy (BinaryTree within noise) in every class.
void default_params(int64_t m, int64_t n, int prec, int out[4]) {
  (void)n;
  if (is_tensor_prec(prec)) {
    out[0] = kMixedNB;
    out[1] = 32;
  } else {
    const int nb = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(256, m)));
    out[0] = nb;
    out[1] = std::min(nb, 32);
  }
  out[2] = TQR_GREEDY;
  out[3] = 1;
}

int fail(int rc, const std::string &msg) {
  set_error(msg);
  return rc;
}

int cuda_err(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? TQR_ENOMEM : TQR_ECUDA;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), std::max<size_t>(1, count) * sizeof(T));
  if (e == cudaSuccess && count) e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Resets counters / ticket / status and launches the executor on "st" (capturable:
// device-to-device copy, memset and one kernel launch).
int enqueue(tqr_batch_plan *pl, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(pl->d_counters, pl->d_indeg, pl->ntask * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->d_state, 0, 2 * sizeof(int32_t), st);
  if (e != cudaSuccess) return cuda_err(e, "batch reset");
  ExecParams prm{};
  prm.nb = pl->max_nb;
  prm.ib = pl->max_ib;
  prm.mixed = is_tensor_prec(pl->prec) ? 1 : 0;
  prm.nparts = prm.mixed ? tensor_parts(pl->prec) : 0;
  prm.fmt = pl->prec == TQR_FP16 ? 0 : 1;
  prm.tasks = pl->d_tasks;
  prm.succ_ptr = pl->d_succ_ptr;
  prm.succ_idx = pl->d_succ_idx;
  prm.counters = pl->d_counters;
  prm.next = pl->d_state;
  prm.status = pl->d_state + 1;
  prm.ntask = static_cast<int>(pl->ntask);
  prm.wait_limit_ns = wait_limit_ns();
  prm.mat_of = pl->d_mat_of;
  prm.mats = pl->d_mats;
  const int rc = launch_executor(prm, pl->prec == TQR_FP64, st);
  if (rc != 0) return cuda_err(static_cast<cudaError_t>(rc), "batched executor launch");
  return TQR_OK;
}

// The merged task table of a batch (host only).  Matrices start longest critical path
// first, each offset by the work of those before it divided by the resident CTAs; all
// tasks are then merged by offset + earliest start (time in units of nb^3), then the
// longer remaining path, then matrix and own position.
struct Merged {
  std::vector<Task> tasks;
  std::vector<int32_t> mat_of, local, indeg, succ_ptr, succ_idx;
  double flops = 0.0;
};

int merge_batch(int nbatch, const int64_t *m, const int64_t *n, const int *prm, int slots, int prec, Merged &out) {
  if (slots < 1) slots = 1;
  out.flops = 0.0;
  // one graph per distinct (P, Q, tree, bs)
  using Key = std::tuple<int, int, int, int>;
  std::map<Key, std::unique_ptr<Graph>> graphs;
  std::vector<const Graph *> gof(nbatch);
  std::vector<double> unit(nbatch), cp(nbatch), work(nbatch);
  for (int b = 0; b < nbatch; ++b) {
    const int *o = prm + 4 * b;
    const int P = static_cast<int>(cdiv(m[b], o[0])), Q = static_cast<int>(cdiv(n[b], o[0]));
    const bool tensor = is_tensor_prec(prec), split = tensor && kPanelSplitCols % o[1] == 0;
    const Key key{P, Q, o[2] | (split ? 1 << 20 : 0), tree_base(o[2]) == TQR_PLASMA ? o[3] : 0};
    auto it = graphs.find(key);
    if (it == graphs.end()) {
      std::vector<Elim> elims;
      if (!elimination_list(P, Q, tree_base(o[2]), o[3], elims)) return fail(-5, "elimination list");
      auto g = std::make_unique<Graph>();
      build_factor_graph(P, Q, elims, *g, -1, nullptr, tree_ts(o[2]), tensor, split);
      it = graphs.emplace(key, std::move(g)).first;
    }
    gof[b] = it->second.get();
    // a weight unit is nb^3/3 flops
    unit[b] = static_cast<double>(o[0]) * o[0] * o[0];
    cp[b] = static_cast<double>(gof[b]->critical_path) * unit[b];
    int64_t w = 0;
    for (int32_t x : gof[b]->weight) w += x;
    work[b] = static_cast<double>(w) * unit[b];
    out.flops += tqr_nominal_flops(m[b], n[b]);
  }
  // start order: longest critical path first; offset = work before it / resident CTAs
  std::vector<int> order(nbatch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cp[a] > cp[c]; });
  std::vector<double> off(nbatch);
  std::vector<int> rank(nbatch);
  double cum = 0.0;
  for (int r = 0; r < nbatch; ++r) {
    off[order[r]] = cum / slots;
    rank[order[r]] = r;
    cum += work[order[r]];
  }
  std::vector<int64_t> base(nbatch + 1, 0);
  for (int b = 0; b < nbatch; ++b) base[b + 1] = base[b] + static_cast<int64_t>(gof[b]->tasks.size());
  const int64_t N = base[nbatch];
  if (N >= (int64_t{1} << 31) - 1) return fail(TQR_EUNSUPPORTED, "batch has too many tasks");
  struct Ent {
    double key, blev;
    int32_t rank, t;
  };
  std::vector<Ent> ent(static_cast<size_t>(N));
  for (int b = 0; b < nbatch; ++b) {
    const Graph &g = *gof[b];
    for (size_t t = 0; t < g.tasks.size(); ++t)
      ent[base[b] + t] = Ent{off[b] + static_cast<double>(g.start[t]) * unit[b],
                             static_cast<double>(g.bottom[t]) * unit[b], rank[b], static_cast<int32_t>(t)};
  }
  // Within a matrix this is its own order (start, then bottom level, then index), and
  // the start grows along every edge: the merged order stays topological.
  std::sort(ent.begin(), ent.end(), [](const Ent &a, const Ent &c) {
    if (a.key != c.key) return a.key < c.key;
    if (a.blev != c.blev) return a.blev > c.blev;
    if (a.rank != c.rank) return a.rank < c.rank;
    return a.t < c.t;
  });
  std::vector<int32_t> gpos(static_cast<size_t>(N));
  for (int64_t r = 0; r < N; ++r) gpos[base[order[ent[r].rank]] + ent[r].t] = static_cast<int32_t>(r);
  std::vector<Task> &tasks = out.tasks;
  std::vector<int32_t> &mat_of = out.mat_of, &indeg = out.indeg, &succ_ptr = out.succ_ptr;
  std::vector<int32_t> &succ_idx = out.succ_idx;
  tasks.resize(static_cast<size_t>(N));
  mat_of.resize(static_cast<size_t>(N));
  out.local.resize(static_cast<size_t>(N));
  indeg.resize(static_cast<size_t>(N));
  succ_ptr.assign(static_cast<size_t>(N) + 1, 0);
  succ_idx.clear();
  int64_t E = 0;
  for (int b = 0; b < nbatch; ++b) E += static_cast<int64_t>(gof[b]->succ_idx.size());
  if (E >= (int64_t{1} << 31) - 1) return fail(TQR_EUNSUPPORTED, "batch has too many dependencies");
  succ_idx.reserve(static_cast<size_t>(E));
  for (int64_t r = 0; r < N; ++r) {
    const int b = order[ent[r].rank];
    const int t = ent[r].t;
    const Graph &g = *gof[b];
    tasks[r] = g.tasks[t];
    mat_of[r] = b;
    out.local[r] = t;
    indeg[r] = g.indeg[t];
    for (int32_t x = g.succ_ptr[t]; x < g.succ_ptr[t + 1]; ++x) succ_idx.push_back(gpos[base[b] + g.succ_idx[x]]);
    succ_ptr[r + 1] = static_cast<int32_t>(succ_idx.size());
  }
  return TQR_OK;
}

int read_status(tqr_batch_plan *pl, cudaStream_t st) {
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, pl->d_state + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_err(e, "batched execution");
  if (h != 0) return fail(TQR_ETIMEOUT, "device wait exceeded the limit at batched task " + std::to_string(h >> 8));
  return TQR_OK;
}

}  // namespace
}  // namespace tqr

using namespace tqr;

extern "C" {

int tqr_batch_params(int nbatch, const int64_t *m, const int64_t *n, int prec, const int64_t *table, int nrows,
                     int *params) {
  if (nbatch < 1 || !m || !n) return -1;
  if (!params) return -4;
  if (prec < TQR_FP64 || prec >= TQR_Z64) return -7;
  for (int r = 0; table && r < nrows; ++r) {
    const int64_t *row = table + 8 * r;
    const int rc = check_tiles(1, 1, static_cast<int>(row[4]), static_cast<int>(row[5]), static_cast<int>(row[6]),
                               static_cast<int>(row[7]), prec);
    if (rc) return fail(-3, "tuning table row " + std::to_string(r) + " is not a valid tile configuration");
  }
  for (int b = 0; b < nbatch; ++b) {
    if (m[b] < 1 || n[b] < 1) return fail(-2, "matrix " + std::to_string(b) + " has an empty dimension");
    int *o = params + 4 * b;
    default_params(m[b], n[b], prec, o);
    for (int r = 0; table && r < nrows; ++r) {
      const int64_t *row = table + 8 * r;
      if (m[b] >= row[0] && m[b] <= row[1] && n[b] >= row[2] && n[b] <= row[3]) {
        for (int c = 0; c < 4; ++c) o[c] = static_cast<int>(row[4 + c]);
        break;
      }
    }
  }
  return TQR_OK;
}

int tqr_batch_workspace_size(int nbatch, const int64_t *m, const int64_t *n, int prec, const int *params,
                             size_t *offsets) {
  if (nbatch < 1 || !m || !n) return -1;
  if (!offsets) return -4;
  size_t off = 0;
  for (int b = 0; b < nbatch; ++b) {
    int dp[4];
    const int *pp = params ? params + 4 * b : dp;
    if (!params) default_params(m[b], n[b], prec, dp);
    const int rc = check_tiles(m[b], n[b], pp[0], pp[1], pp[2], pp[3], prec);
    if (rc) return fail(rc == -1 || rc == -2 ? -2 : rc, "matrix " + std::to_string(b) + ": invalid size or tuning");
    offsets[b] = off;
    off = align_up(off + factor_workspace_bytes(m[b], n[b], pp[0], pp[1], prec), 256);
  }
  offsets[nbatch] = off;
  return TQR_OK;
}

int tqr_batch_plan_create(int nbatch, const int64_t *m, const int64_t *n, void *const *A, const int64_t *lda,
                          const int *params, int prec, void *const *T, tqr_batch_plan **plan) {
  if (!plan) return -4;
  *plan = nullptr;
  if (nbatch < 1 || !m || !n || !A || !lda || !T) return fail(-1, "empty batch or NULL array");
  if (prec == TQR_Z64) return fail(-7, "the batched factorization has no double-complex form");
  try {
    std::vector<int> prm(4 * static_cast<size_t>(nbatch));
    // no per-matrix tuning given: the autotuned setting of each size class (tuned on the
    // legacy stream on first use, then cached)
    std::vector<std::array<int64_t, 8>> rows;
    if (!params) {
      for (int b = 0; b < nbatch; ++b)
        if (m[b] < 1 || n[b] < 1) return fail(-1, "matrix " + std::to_string(b) + ": size < 1");
      const int rc = autotune_table(nbatch, m, n, prec, nullptr, rows);
      if (rc) return rc;
    }
    for (int b = 0; b < nbatch; ++b) {
      int *o = prm.data() + 4 * b;
      if (params) {
        std::memcpy(o, params + 4 * b, 4 * sizeof(int));
      } else {
        default_params(std::max<int64_t>(m[b], 1), n[b], prec, o);
        for (const auto &r : rows)
          if (m[b] >= r[0] && m[b] <= r[1] && n[b] >= r[2] && n[b] <= r[3]) {
            for (int c = 0; c < 4; ++c) o[c] = static_cast<int>(r[4 + c]);
            break;
          }
      }
      const int rc = check_tiles(m[b], n[b], o[0], o[1], o[2], o[3], prec);
      if (rc) return fail(rc, "matrix " + std::to_string(b) + ": " + tqr_strerror(rc) + " (status " +
                                  std::to_string(rc) + ")");
      if (!A[b] || !T[b] || lda[b] < m[b])
        return fail(-2, "matrix " + std::to_string(b) + ": NULL pointer or lda < m");
      if (!is_tensor_prec(prec) && executor_smem_bytes(o[0], o[1], prec == TQR_FP64, false) == 0)
        return fail(TQR_EUNSUPPORTED, "nb/ib too large for one SM's shared memory");
    }
    auto pl = std::make_unique<tqr_batch_plan>();
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    pl->prec = prec;
    pl->nmat = nbatch;
    for (int b = 0; b < nbatch; ++b) {
      pl->max_nb = std::max(pl->max_nb, prm[4 * b]);
      pl->max_ib = std::max(pl->max_ib, prm[4 * b + 1]);
    }
    pl->slots = executor_slots(prec == TQR_FP64, is_tensor_prec(prec), pl->max_nb, pl->max_ib);
    if (pl->slots < 1) pl->slots = 1;

    Merged mg;
    const int rc = merge_batch(nbatch, m, n, prm.data(), pl->slots, prec, mg);
    if (rc) return rc;
    // test hook (tqr_debug_drop_edge): leave out the release of one merged dependency edge,
    // so that its successor's wait can only end by the wait limit
    const int64_t drop = take_debug_drop_edge();
    if (drop >= 0 && drop < static_cast<int64_t>(mg.succ_idx.size())) {
      const int64_t N0 = static_cast<int64_t>(mg.tasks.size());
      std::vector<int32_t> ptr(N0 + 1, 0), idx;
      idx.reserve(mg.succ_idx.size());
      for (int64_t r = 0; r < N0; ++r) {
        for (int32_t x = mg.succ_ptr[r]; x < mg.succ_ptr[r + 1]; ++x)
          if (x != drop) idx.push_back(mg.succ_idx[x]);
        ptr[r + 1] = static_cast<int32_t>(idx.size());
      }
      mg.succ_ptr.swap(ptr);
      mg.succ_idx.swap(idx);
    }
    pl->flops = mg.flops;
    const int64_t N = static_cast<int64_t>(mg.tasks.size());
    const int64_t E = static_cast<int64_t>(mg.succ_idx.size());
    std::vector<BatchMat> mats(nbatch);
    for (int b = 0; b < nbatch; ++b) {
      const int *o = prm.data() + 4 * b;
      BatchMat &d = mats[b];
      d.A = A[b];
      d.lda = lda[b];
      d.m = m[b];
      d.n = n[b];
      d.nb = o[0];
      d.ib = o[1];
      d.P = static_cast<int>(cdiv(m[b], o[0]));
      d.Q = static_cast<int>(cdiv(n[b], o[0]));
      d.T = T[b];
      d.ops = is_tensor_prec(prec) ? static_cast<char *>(T[b]) + ops_offset(m[b], n[b], o[0], o[1]) : nullptr;
      d.vec4 = (reinterpret_cast<uintptr_t>(A[b]) % 16 == 0 && lda[b] % 4 == 0) ? 1 : 0;
      d.pad = 0;
    }
    pl->ntask = N;
    pl->nedge = E;
    if ((e = upload(&pl->d_tasks, mg.tasks.data(), mg.tasks.size())) != cudaSuccess ||
        (e = upload(&pl->d_mat_of, mg.mat_of.data(), mg.mat_of.size())) != cudaSuccess ||
        (e = upload(&pl->d_succ_ptr, mg.succ_ptr.data(), mg.succ_ptr.size())) != cudaSuccess ||
        (e = upload(&pl->d_succ_idx, mg.succ_idx.data(), mg.succ_idx.size())) != cudaSuccess ||
        (e = upload(&pl->d_indeg, mg.indeg.data(), mg.indeg.size())) != cudaSuccess ||
        (e = upload(&pl->d_mats, mats.data(), mats.size())) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_counters, std::max<size_t>(1, N) * sizeof(int32_t))) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_state, 2 * sizeof(int32_t))) != cudaSuccess)
      return cuda_err(e, "batch plan upload");
    *plan = pl.release();
    return TQR_OK;
  } catch (const std::bad_alloc &) {
    return fail(TQR_ENOMEM, "host memory for the batch plan");
  }
}

int tqr_batch_order(int nbatch, const int64_t *m, const int64_t *n, int prec, const int *params, int slots,
                    int32_t *mat_of, int32_t *local, int64_t *ntask) {
  if (nbatch < 1 || !m || !n) return -1;
  if (!ntask) return -4;
  try {
    std::vector<int> prm(4 * static_cast<size_t>(nbatch));
    for (int b = 0; b < nbatch; ++b) {
      int *o = prm.data() + 4 * b;
      if (params)
        std::memcpy(o, params + 4 * b, 4 * sizeof(int));
      else
        default_params(m[b], n[b], prec, o);
      const int rc = check_tiles(m[b], n[b], o[0], o[1], o[2], o[3], prec);
      if (rc) return fail(rc, "matrix " + std::to_string(b) + ": invalid size or tuning");
    }
    Merged mg;
    const int rc = merge_batch(nbatch, m, n, prm.data(), slots, prec, mg);
    if (rc) return rc;
    const int64_t N = static_cast<int64_t>(mg.tasks.size());
    if (mat_of && local) {
      if (*ntask < N) return -4;
      std::memcpy(mat_of, mg.mat_of.data(), N * sizeof(int32_t));
      std::memcpy(local, mg.local.data(), N * sizeof(int32_t));
    }
    *ntask = N;
    return TQR_OK;
  } catch (const std::bad_alloc &) {
    return fail(TQR_ENOMEM, "host memory for the batch order");
  }
}

int tqr_batch_plan_run(tqr_batch_plan *pl, int use_graph, void *stream) {
  if (!pl) return -1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (pl->ntask == 0) return TQR_OK;
  if (!use_graph) {
    const int rc = enqueue(pl, st);
    if (rc) return rc;
  } else {
    if (!pl->exec) {
      cudaError_t e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_err(e, "capture stream");
      e = cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_err(e, "cudaStreamBeginCapture");
      const int rc = enqueue(pl, pl->cap_stream);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(pl->cap_stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
      pl->graph = g;
      e = cudaGraphInstantiate(&pl->exec, g, 0);
      if (e != cudaSuccess) {
        pl->exec = nullptr;
        return cuda_err(e, "cudaGraphInstantiate");
      }
    }
    cudaError_t e = cudaGraphLaunch(pl->exec, st);
    if (e != cudaSuccess) return cuda_err(e, "cudaGraphLaunch");
    count_launch();
  }
  if (sync_enabled()) return read_status(pl, st);
  return TQR_OK;
}

int tqr_batch_plan_status(tqr_batch_plan *pl, void *stream) {
  if (!pl) return -1;
  return read_status(pl, static_cast<cudaStream_t>(stream));
}

int tqr_batch_plan_info(const tqr_batch_plan *pl, int64_t out[6]) {
  if (!pl || !out) return -1;
  out[0] = pl->ntask;
  out[1] = pl->nedge;
  out[2] = pl->nmat;
  out[3] = pl->slots;
  out[4] = pl->exec ? 1 : 0;
  out[5] = static_cast<int64_t>(pl->flops);
  return TQR_OK;
}

void tqr_batch_plan_destroy(tqr_batch_plan *pl) { delete pl; }

int tqr_factor_batched(int nbatch, const int64_t *m, const int64_t *n, void *const *A, const int64_t *lda,
                       const int *params, int prec, void *const *T, void *stream) {
  tqr_batch_plan *pl = nullptr;
  int rc = tqr_batch_plan_create(nbatch, m, n, A, lda, params, prec, T, &pl);
  if (rc) return rc;
  rc = enqueue(pl, static_cast<cudaStream_t>(stream));
  if (rc == TQR_OK) rc = read_status(pl, static_cast<cudaStream_t>(stream));
  else cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  tqr_batch_plan_destroy(pl);
  return rc;
}

}  // extern "C"
