// Triangular solve R X = B for the upper-triangular R of a tiled QR (the last step of
// the least-squares solve x = R^{-1} (Q^T b)(0:n)).
//
// Wavefront over row blocks of TB rows: CTAs take tickets in launch order and handle
// the row blocks bottom-up; block kb waits for every block below it (published through
// a per-block flag with release/acquire), subtracts R(kb, kk) X(kk), then solves its
// diagonal block by back substitution (one warp per right-hand side).  A block only
// waits for blocks whose tickets were taken earlier, so the wavefront cannot deadlock.
// Waits are bounded like the executor's and report kStatusTimeout.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/tqr.h"
#include "tqr_internal.h"

namespace tqr {
namespace {

__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr int kTB = 64;        // rows per block
constexpr int kRHS = 32;       // right-hand sides per pass
constexpr int kThreads = 256;

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acq(const int32_t *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_rel(int32_t *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ double ld_cg(const float *p) { return static_cast<double>(__ldcg(p)); }

// kLowerT = false: solve R X = B (backward, blocks bottom-up);
// kLowerT = true : solve R^T X = B (forward, blocks top-down).
template <typename Real, bool kLowerT>
__global__ void __launch_bounds__(kThreads) trsm_kernel(int64_t n, const Real *A, int64_t lda, double *B,
                                                        int64_t ldb, int nrhs, int32_t *flags,
                                                        int32_t *status, int64_t wait_limit_ns) {
  extern __shared__ double trsm_smem[];
  double(*Cs)[kRHS + 1] = reinterpret_cast<double(*)[kRHS + 1]>(trsm_smem);
  double(*Xs)[kRHS + 1] = reinterpret_cast<double(*)[kRHS + 1]>(trsm_smem + kTB * (kRHS + 1));
  double(*Rs)[kTB + 1] = reinterpret_cast<double(*)[kTB + 1]>(trsm_smem + 2 * kTB * (kRHS + 1));
  __shared__ int s_kb, s_stop;
  const int nblk = static_cast<int>((n + kTB - 1) / kTB);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    const int ticket = atomicAdd(flags, 1);
    s_kb = kLowerT ? (ticket < nblk ? ticket : -1) : nblk - 1 - ticket;
    s_stop = 0;
  }
  __syncthreads();
  const int kb = s_kb;
  if (kb < 0) return;
  const int64_t r0 = static_cast<int64_t>(kb) * kTB;
  const int rb = static_cast<int>(lmin(kTB, n - r0));
  for (int idx = tid; idx < rb * nrhs; idx += kThreads) {
    const int j = idx / rb, r = idx - j * rb;
    Cs[r][j] = ld_cg(B + r0 + r + j * ldb);
  }
  for (int step = 0; step < (kLowerT ? kb : nblk - 1 - kb); ++step) {
    const int kk = kLowerT ? step : nblk - 1 - step;
    if (tid == 0) {
      const uint64_t t0 = gtimer();
      for (uint64_t it = 0; ld_acq(flags + 1 + kk) == 0; ++it) {
        if (*(volatile int32_t *)status != 0) { s_stop = 1; break; }
        if (gtimer() - t0 > static_cast<uint64_t>(wait_limit_ns) ||
            it > (static_cast<uint64_t>(wait_limit_ns) >> 4) + 1000000ull) {
          atomicCAS(status, 0, kStatusTimeout | (kk << 8));
          s_stop = 1;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    __syncthreads();
    if (s_stop) return;
    const int64_t c0 = static_cast<int64_t>(kk) * kTB;
    const int cb = static_cast<int>(lmin(kTB, n - c0));
    for (int idx = tid; idx < rb * cb; idx += kThreads) {
      const int c = idx / rb, r = idx - c * rb;
      // block (kb, kk) of R, or of R^T = block (kk, kb) of R transposed
      Rs[r][c] = kLowerT ? ld_cg(A + (c0 + c) + (r0 + r) * lda) : ld_cg(A + (r0 + r) + (c0 + c) * lda);
    }
    for (int idx = tid; idx < cb * nrhs; idx += kThreads) {
      const int j = idx / cb, r = idx - j * cb;
      Xs[r][j] = ld_cg(B + c0 + r + j * ldb);
    }
    __syncthreads();
    for (int idx = tid; idx < rb * nrhs; idx += kThreads) {
      const int j = idx / rb, r = idx - j * rb;
      double acc = 0.0;
      for (int c = 0; c < cb; ++c) acc += Rs[r][c] * Xs[c][j];
      Cs[r][j] -= acc;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < rb * rb; idx += kThreads) {
    const int c = idx / rb, r = idx - c * rb;
    if (kLowerT)
      Rs[r][c] = (c <= r) ? ld_cg(A + (r0 + c) + (r0 + r) * lda) : 0.0;
    else
      Rs[r][c] = (r <= c) ? ld_cg(A + (r0 + r) + (r0 + c) * lda) : 0.0;
  }
  __syncthreads();
  // reciprocals of the diagonal, formed in parallel once (an FP64 division is slow)
  __shared__ double s_rinv[kTB];
  if (tid < rb) s_rinv[tid] = 1.0 / Rs[tid][tid];
  __syncthreads();
  // substitution, one warp per right-hand side; lane owns rows lane and lane+32
  for (int j = warp; j < nrhs; j += kThreads / 32) {
    double c_lo = lane < rb ? Cs[lane][j] : 0.0;
    double c_hi = lane + 32 < rb ? Cs[lane + 32][j] : 0.0;
    for (int step = 0; step < rb; ++step) {
      const int i = kLowerT ? step : rb - 1 - step;
      const double ci = __shfl_sync(0xffffffffu, i < 32 ? c_lo : c_hi, i & 31);
      const double xi = ci * s_rinv[i];
      if (lane == (i & 31)) {
        if (i < 32) c_lo = xi; else c_hi = xi;
      }
      if (kLowerT) {
        if (lane > i && lane < rb) c_lo -= Rs[lane][i] * xi;
        if (lane + 32 > i && lane + 32 < rb) c_hi -= Rs[lane + 32][i] * xi;
      } else {
        if (lane < i) c_lo -= Rs[lane][i] * xi;
        if (lane + 32 < i) c_hi -= Rs[lane + 32][i] * xi;
      }
    }
    if (lane < rb) Cs[lane][j] = c_lo;
    if (lane + 32 < rb) Cs[lane + 32][j] = c_hi;
  }
  __syncthreads();
  for (int idx = tid; idx < rb * nrhs; idx += kThreads) {
    const int j = idx / rb, r = idx - j * rb;
    B[r0 + r + j * ldb] = Cs[r][j];
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_rel(flags + 1 + kb, 1);
  }
}

int trsm_flag_count_impl(int64_t n) { return static_cast<int>((n + kTB - 1) / kTB) + 1; }

template <typename Real, bool kLowerT>
cudaError_t launch_one(int nblk, size_t smem, cudaStream_t st, int64_t n, const void *A, int64_t lda, double *B,
                       int64_t ldb, int nr, int32_t *flags, int32_t *status, int64_t wait_limit_ns) {
  auto kern = trsm_kernel<Real, kLowerT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<nblk, kThreads, smem, st>>>(n, static_cast<const Real *>(A), lda, B, ldb, nr, flags, status, wait_limit_ns);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int launch_trsm(int64_t n, const void *A, int64_t lda, bool real_is_double, double *B, int64_t ldb,
                int64_t nrhs, int32_t *flags, int32_t *status, int64_t wait_limit_ns, void *stream,
                bool lower_transposed) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = sizeof(double) * (2 * kTB * (kRHS + 1) + kTB * (kTB + 1));
  const int nblk = static_cast<int>((n + kTB - 1) / kTB);
  for (int64_t j0 = 0; j0 < nrhs; j0 += kRHS) {
    const int nr = static_cast<int>(nrhs - j0 < kRHS ? nrhs - j0 : kRHS);
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int32_t) * (nblk + 1), st);
    if (e != cudaSuccess) return static_cast<int>(e);
    if (real_is_double)
      e = lower_transposed ? launch_one<double, true>(nblk, smem, st, n, A, lda, B + j0 * ldb, ldb, nr, flags, status, wait_limit_ns)
                           : launch_one<double, false>(nblk, smem, st, n, A, lda, B + j0 * ldb, ldb, nr, flags, status, wait_limit_ns);
    else
      e = lower_transposed ? launch_one<float, true>(nblk, smem, st, n, A, lda, B + j0 * ldb, ldb, nr, flags, status, wait_limit_ns)
                           : launch_one<float, false>(nblk, smem, st, n, A, lda, B + j0 * ldb, ldb, nr, flags, status, wait_limit_ns);
    if (e != cudaSuccess) return static_cast<int>(e);
  }
  return 0;
}

int trsm_flag_count(int64_t n) { return trsm_flag_count_impl(n); }

// ---------------------------------------------------------------------------------
// Inverses of the 64 x 64 diagonal blocks of R (FP64), the starting point of the
// refinement's preconditioner set-up (precond.cu).
namespace {

// Dinv[k] = inverse of the k-th 64 x 64 diagonal block of the upper-triangular R.
template <typename Real>
__global__ void __launch_bounds__(kThreads) diag_inverse_kernel(int64_t n, const Real *A, int64_t lda,
                                                                double *Dinv) {
  extern __shared__ double dinv_smem[];
  double(*Rs)[kTB + 1] = reinterpret_cast<double(*)[kTB + 1]>(dinv_smem);
  double(*Xs)[kTB + 1] = reinterpret_cast<double(*)[kTB + 1]>(dinv_smem + kTB * (kTB + 1));  // inverse
  __shared__ double rinv[kTB];
  const int kb = blockIdx.x;
  const int64_t r0 = static_cast<int64_t>(kb) * kTB;
  const int rb = static_cast<int>(lmin(kTB, n - r0));
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
    const int c = idx / kTB, r = idx - c * kTB;
    double v = 0.0;
    if (r < rb && c < rb && r <= c) v = ld_cg(A + (r0 + r) + (r0 + c) * lda);
    if (r == c && r >= rb) v = 1.0;  // identity on the padding of a partial last block
    Rs[r][c] = v;
    Xs[r][c] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid < kTB) rinv[tid] = 1.0 / Rs[tid][tid];
  __syncthreads();
  // back substitution on all 64 columns of the identity at once
  for (int i = kTB - 1; i >= 0; --i) {
    for (int j = tid; j < kTB; j += kThreads) Xs[i][j] *= rinv[i];
    __syncthreads();
    for (int idx = tid; idx < i * kTB; idx += kThreads) {
      const int j = idx / i, l = idx - j * i;
      Xs[l][j] -= Rs[l][i] * Xs[i][j];
    }
    __syncthreads();
  }
  double *out = Dinv + static_cast<int64_t>(kb) * kTB * kTB;
  for (int idx = tid; idx < kTB * kTB; idx += kThreads) {
    const int c = idx / kTB, r = idx - c * kTB;
    out[r + c * kTB] = Xs[r][c];
  }
}

}  // namespace

int launch_diag_inverse(int64_t n, const void *A, int64_t lda, bool real_is_double, double *Dinv, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nblk = static_cast<int>((n + kTB - 1) / kTB);
  const size_t smem = sizeof(double) * 2 * kTB * (kTB + 1);
  cudaError_t e = real_is_double
      ? cudaFuncSetAttribute(diag_inverse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
      : cudaFuncSetAttribute(diag_inverse_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  if (real_is_double)
    diag_inverse_kernel<double><<<nblk, kThreads, smem, st>>>(n, static_cast<const double *>(A), lda, Dinv);
  else
    diag_inverse_kernel<float><<<nblk, kThreads, smem, st>>>(n, static_cast<const float *>(A), lda, Dinv);
  count_launch();
  return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------------
// Scratch for tqr_trsm_static: a ticket, one flag per 64-row block and a status word,
// in a fixed array that exists on every GPU that loads this library (until the process
// exits).  Its size caps n at kStaticMaxBlocks * 64 rows.
constexpr int kStaticMaxBlocks = 4096;
static __device__ __align__(256) int32_t g_trsm_static_scratch[kStaticMaxBlocks + 2];

namespace {
std::mutex g_static_mu;
constexpr int kMaxDevices = 64;
int32_t *g_static_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  The host-side symbol is
// only a stand-in, so the address is looked up once per device (with that device
// current) and cached; this lookup is the only set-up the entry point needs.  The cached
// address belongs to the device's primary context: after a cudaDeviceReset the module is
// loaded again and the array may move, so tqr_finalize() forgets the cached addresses
// (reset_static_scratch) and the next call looks them up again.
int static_scratch(int32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return TQR_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return TQR_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    int32_t *p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_trsm_static_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return TQR_ECUDA;
    }
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return TQR_OK;
}
}  // namespace

void reset_static_scratch() {
  std::lock_guard<std::mutex> lock(g_static_mu);
  for (int d = 0; d < kMaxDevices; ++d) g_static_ptr[d] = nullptr;
}

}  // namespace tqr

extern "C" int tqr_trsm_static(int64_t n, int prec, const void *A, int64_t lda, double *B, int64_t ldb,
                               int64_t nrhs, void *stream) {
  using namespace tqr;
  if (n < 1) return -1;
  if (prec < TQR_FP64 || prec >= TQR_Z64) return -2;
  if (!A) return -3;
  if (lda < n) return -4;
  if (!B) return -5;
  if (ldb < n) return -6;
  if (nrhs < 0) return -7;
  const int64_t nblk = (n + 63) / 64;
  if (nblk > kStaticMaxBlocks) {
    set_error("tqr_trsm_static: n exceeds the static scratch limit of " +
              std::to_string(static_cast<long long>(kStaticMaxBlocks) * 64) + " rows");
    return -1;
  }
  if (nrhs == 0) return TQR_OK;
  int32_t *scratch = nullptr;
  int rc = static_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t *status = scratch + kStaticMaxBlocks + 1;
  // the array keeps the previous call's contents: the status word starts at zero, and
  // launch_trsm zeroes the ticket and flags before every pass
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) {
    set_error(std::string("tqr_trsm_static: ") + cudaGetErrorString(e));
    return TQR_ECUDA;
  }
  rc = launch_trsm(n, A, lda, prec == TQR_FP64, B, ldb, nrhs, scratch, status, wait_limit_ns(), stream);
  if (rc) {
    set_error(std::string("tqr_trsm_static: ") + cudaGetErrorString(static_cast<cudaError_t>(rc)));
    return TQR_ECUDA;
  }
  if (!sync_enabled()) return TQR_OK;
  int32_t h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error(std::string("tqr_trsm_static: ") + cudaGetErrorString(e));
    return TQR_ECUDA;
  }
  if (h != 0) {
    set_error("tqr_trsm_static: device wait exceeded the limit at block " + std::to_string(h >> 8));
    return TQR_ETIMEOUT;
  }
  return TQR_OK;
}
