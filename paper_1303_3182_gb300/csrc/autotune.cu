// Per-size-class autotuner of the batched factorization, inside the library.
//
// The matrices of a batch are grouped into size classes - a row-count bucket times the
// exact column count.  For each class the library factors a sample of that class's own
// shapes (seeded pseudo-random entries in scratch device memory, inputs restored before
// every timed launch) as one batched launch per candidate setting and keeps the fastest:
// first the tile size nb (Greedy, ib = min(nb, 32)), then the inner block ib at that nb,
// then the elimination tree (the thesis's trees and the TS forms of FlatTree and
// PlasmaTree) at that (nb, ib).  Tensor-core precisions have one tile size (128).  Timing
// is device time between CUDA events around the launch.  Results are cached per device,
// precision and class for the life of the process.  The thesis tunes nothing of this
// kind; it picks its trees by critical path (Chapter 3) and measures one matrix at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tqr.h"
#include "tqr_internal.h"

namespace tqr {
namespace {

constexpr int64_t kBuckets[3][2] = {{1, 1024}, {1025, 4096}, {4097, int64_t{1} << 40}};
constexpr int kSample = 32;  // matrices of a class factored per candidate
constexpr int kNbCand[4] = {32, 64, 128, 256};
constexpr int kIbCand[3] = {8, 16, 32};
constexpr int kTreeCand[7][2] = {{TQR_GREEDY, 1}, {TQR_BINARY, 1}, {TQR_FIBONACCI, 1}, {TQR_FLAT, 1},
                                 {TQR_PLASMA, 4}, {TQR_FLAT | TQR_TS, 1}, {TQR_PLASMA | TQR_TS, 4}};

using ClassKey = std::tuple<int, int, int64_t, int64_t, int64_t>;  // device, prec, m_lo, m_hi, n
std::mutex g_tune_mu;
std::map<ClassKey, std::array<int, 4>> g_tune_cache;

// Counter-based fill: entry e of the scratch gets a value uniform in [-1, 1) from the
// splitmix64 finalizer of (seed, e).
template <typename Real>
__global__ void fill_kernel(Real *x, int64_t count, uint64_t seed) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * static_cast<uint64_t>(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[e] = static_cast<Real>(static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

int bucket_of(int64_t m) {
  for (int b = 0; b < 3; ++b)
    if (m >= kBuckets[b][0] && m <= kBuckets[b][1]) return b;
  return 2;
}

struct Scratch2 {
  void *A = nullptr, *A0 = nullptr, *T = nullptr;
  size_t a_bytes = 0, t_bytes = 0;
  ~Scratch2() {
    cudaFree(A);
    cudaFree(A0);
    cudaFree(T);
  }
};

// Device ms of one batched launch of the sample with the given setting (or < 0 when the
// setting does not run: too large for shared memory, or a launch error).
double time_setting(const std::vector<int64_t> &ms, int64_t n, int prec, const int cand[4], Scratch2 &sc,
                    cudaStream_t st) {
  const int nmat = static_cast<int>(ms.size());
  std::vector<int> params(4 * static_cast<size_t>(nmat));
  for (int b = 0; b < nmat; ++b)
    for (int c = 0; c < 4; ++c) params[4 * b + c] = cand[c];
  std::vector<int64_t> nn(nmat, n), lda(ms);
  for (int b = 0; b < nmat; ++b)
    if (check_tiles(ms[b], n, cand[0], cand[1], cand[2], cand[3], prec)) return -1.0;
  if (!is_tensor_prec(prec) && executor_smem_bytes(cand[0], cand[1], prec == TQR_FP64, false) == 0) return -1.0;
  std::vector<size_t> off(nmat + 1);
  if (tqr_batch_workspace_size(nmat, ms.data(), nn.data(), prec, params.data(), off.data()) != TQR_OK) return -1.0;
  if (off[nmat] > sc.t_bytes) {
    cudaFree(sc.T);
    sc.T = nullptr;
    sc.t_bytes = 0;
    if (cudaMalloc(&sc.T, off[nmat]) != cudaSuccess) return -1.0;
    sc.t_bytes = off[nmat];
  }
  const size_t esz = prec == TQR_FP64 ? sizeof(double) : sizeof(float);
  std::vector<void *> A(nmat), T(nmat);
  size_t aoff = 0;
  for (int b = 0; b < nmat; ++b) {
    A[b] = static_cast<char *>(sc.A) + aoff;
    aoff += align_up(static_cast<size_t>(ms[b]) * n * esz, 256);
    T[b] = static_cast<char *>(sc.T) + off[b];
  }
  tqr_batch_plan *pl = nullptr;
  if (tqr_batch_plan_create(nmat, ms.data(), nn.data(), A.data(), lda.data(), params.data(), prec, T.data(), &pl) !=
      TQR_OK)
    return -1.0;
  const int old_sync = tqr_set_sync(0);
  double best = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up; the second is timed
      if (cudaMemcpyAsync(sc.A, sc.A0, sc.a_bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess) break;
      cudaEventRecord(e0, st);
      if (tqr_batch_plan_run(pl, 0, st) != TQR_OK) break;
      cudaEventRecord(e1, st);
      if (tqr_batch_plan_status(pl, st) != TQR_OK) break;
      float ms_ = 0.f;
      if (cudaEventElapsedTime(&ms_, e0, e1) != cudaSuccess) break;
      if (rep == 1) best = ms_;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  tqr_set_sync(old_sync);
  tqr_batch_plan_destroy(pl);
  return best;
}

// Tunes one class from the row counts of its sample; returns 0 or a status.
int tune_class(int prec, const std::vector<int64_t> &ms, int64_t n, cudaStream_t st, std::array<int, 4> &out) {
  const size_t esz = prec == TQR_FP64 ? sizeof(double) : sizeof(float);
  Scratch2 sc;
  for (int64_t m : ms) sc.a_bytes += align_up(static_cast<size_t>(m) * n * esz, 256);
  if (cudaMalloc(&sc.A, sc.a_bytes) != cudaSuccess || cudaMalloc(&sc.A0, sc.a_bytes) != cudaSuccess) {
    set_error("tqr_batch_autotune: scratch allocation");
    return TQR_ENOMEM;
  }
  const int64_t count = static_cast<int64_t>(sc.a_bytes / esz);
  if (prec == TQR_FP64)
    fill_kernel<double><<<1024, 256, 0, st>>>(static_cast<double *>(sc.A0), count, 1303318204ull + n);
  else
    fill_kernel<float><<<1024, 256, 0, st>>>(static_cast<float *>(sc.A0), count, 1303318204ull + n);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return TQR_ECUDA;
  const int64_t m_max = *std::max_element(ms.begin(), ms.end());
  double best_t = -1.0;
  std::array<int, 4> best{kMixedNB, 32, TQR_GREEDY, 1};
  auto consider = [&](const int cand[4]) {
    const double t = time_setting(ms, n, prec, cand, sc, st);
    if (t > 0 && (best_t < 0 || t < best_t)) {
      best_t = t;
      best = {cand[0], cand[1], cand[2], cand[3]};
    }
    return t;
  };
  if (!is_tensor_prec(prec)) {
    // tile size with Greedy and ib = min(nb, 32)
    for (int nb : kNbCand) {
      if (nb > std::max<int64_t>(32, m_max)) continue;
      const int cand[4] = {nb, std::min(nb, 32), TQR_GREEDY, 1};
      consider(cand);
    }
    // inner block at the best tile size
    const int nb = best[0];
    for (int ib : kIbCand) {
      if (ib > nb) continue;
      const int cand[4] = {nb, ib, TQR_GREEDY, 1};
      consider(cand);
    }
  } else {
    for (int ib : {16, 32}) {
      const int cand[4] = {kMixedNB, ib, TQR_GREEDY, 1};
      consider(cand);
    }
  }
  // elimination tree at the best (nb, ib)
  const int nb = best[0], ib = best[1];
  for (const auto &tr : kTreeCand) {
    const int cand[4] = {nb, ib, tr[0], tr[1]};
    consider(cand);
  }
  if (best_t < 0) {
    set_error("tqr_batch_autotune: no candidate setting ran");
    return TQR_ECUDA;
  }
  out = best;
  return TQR_OK;
}

}  // namespace

int autotune_table(int nbatch, const int64_t *m, const int64_t *n, int prec, void *stream,
                   std::vector<std::array<int64_t, 8>> &rows) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TQR_ECUDA;
  // classes in first-appearance order, with the row counts of their first kSample members
  std::map<std::tuple<int, int64_t>, std::vector<int64_t>> members;
  std::vector<std::tuple<int, int64_t>> order;
  for (int b = 0; b < nbatch; ++b) {
    const auto key = std::make_tuple(bucket_of(m[b]), n[b]);
    auto it = members.find(key);
    if (it == members.end()) {
      order.push_back(key);
      it = members.emplace(key, std::vector<int64_t>()).first;
    }
    if (static_cast<int>(it->second.size()) < kSample) it->second.push_back(m[b]);
  }
  std::sort(order.begin(), order.end());
  rows.clear();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (const auto &key : order) {
    const int bk = std::get<0>(key);
    const int64_t nn = std::get<1>(key), lo = kBuckets[bk][0], hi = kBuckets[bk][1];
    const ClassKey ck{dev, prec, lo, hi, nn};
    std::array<int, 4> setting{};
    bool cached = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tune_cache.find(ck);
      if (it != g_tune_cache.end()) {
        setting = it->second;
        cached = true;
      }
    }
    if (!cached) {
      const int rc = tune_class(prec, members[key], nn, st, setting);
      if (rc) return rc;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tune_cache[ck] = setting;
    }
    rows.push_back({lo, hi, nn, nn, setting[0], setting[1], setting[2], setting[3]});
  }
  return TQR_OK;
}

void forget_autotune() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
}

}  // namespace tqr

extern "C" int tqr_batch_autotune(int nbatch, const int64_t *m, const int64_t *n, int prec, int64_t *table,
                                  int capacity, int *nrows, void *stream) {
  using namespace tqr;
  if (nbatch < 1) return -1;
  if (!m || !n) return -2;
  for (int b = 0; b < nbatch; ++b)
    if (m[b] < 1 || n[b] < 1) return -2;
  if (prec < TQR_FP64 || prec >= TQR_Z64) return -4;
  if (!nrows) return -7;
  try {
    std::vector<std::array<int64_t, 8>> rows;
    const int rc = autotune_table(nbatch, m, n, prec, stream, rows);
    if (rc) return rc;
    *nrows = static_cast<int>(rows.size());
    if (table) {
      if (capacity < static_cast<int>(rows.size())) return -6;
      for (size_t r = 0; r < rows.size(); ++r)
        for (int c = 0; c < 8; ++c) table[8 * r + c] = rows[r][c];
    }
  } catch (const std::bad_alloc &) {
    return TQR_ENOMEM;
  }
  return TQR_OK;
}
