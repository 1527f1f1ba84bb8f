// Preconditioner solves of the refinement: y = R^{-1} v and y = R^{-T} v with the same
// upper-triangular R (the low-precision factor, float or double) for every LSQR step.
//
// Set-up (once per refinement): a transposed copy of R's upper triangle (so that both
// solves read R along contiguous columns) and the inverses of R's 1024 x 1024 diagonal
// blocks, formed in FP64 from the 64 x 64 block inverses by four doubling steps
//   inv([R11 R12; 0 R22]) = [R11^{-1}, -R11^{-1} R12 R22^{-1}; 0, R22^{-1}]
// and kept as FP32 pairs (hi, lo) for the solves.
// Solve: one cooperative launch walks the big blocks (4 for n = 4096); each step is two
// grid-wide phases separated by a grid barrier - x_s = Y_s b_s over all SMs, then the
// update of the remaining right-hand-side rows with R's off-diagonal column block - so
// the sequential depth is ceil(n / 1024) steps instead of ceil(n / 64).  The products
// run in double-float arithmetic (about 2^-44 relative: a preconditioner applied to the
// same accuracy as the refinement's pair products with A); partial sums meet in FP64
// atomics (results reproducible to rounding, not bit for bit).  Every grid barrier wait
// is bounded and reports kStatusTimeout like the executor's waits.
#include <cuda_runtime.h>

#include <cstdint>

#include "tqr_internal.h"

namespace tqr {
namespace {

constexpr int kBig = 1024;     // rows of a big diagonal block
constexpr int kCT = kBig / 64; // 64-column tiles across a big block
constexpr int kP1 = (kBig / 32) * kCT;  // 32 x 64 tiles of a big block (phase-1 items)
constexpr int kSmall = 64;     // rows of the blocks whose inverses the set-up starts from
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRhsMax = 4;     // right-hand sides per solve launch

__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

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

// ---- set-up ---------------------------------------------------------------------------

// Y[s] (kBig x kBig, column-major, FP32 pairs): the 64 x 64 inverses on the diagonal
// (identity for 64-blocks beyond n), zeros elsewhere.
__global__ void big_init_kernel(int64_t n, const double *Dinv64, float2 *Y, int nbig) {
  const int nblk64 = static_cast<int>((n + kSmall - 1) / kSmall);
  const int64_t total = static_cast<int64_t>(nbig) * kBig * kBig;
  for (int64_t idx = blockIdx.x * static_cast<int64_t>(kThreads) + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * kThreads) {
    const int s = static_cast<int>(idx / (kBig * kBig));
    const int rem = static_cast<int>(idx - static_cast<int64_t>(s) * kBig * kBig);
    const int c = rem / kBig, r = rem - c * kBig;
    double v = 0.0;
    if (r / kSmall == c / kSmall) {
      const int b64 = s * (kBig / kSmall) + c / kSmall;
      if (b64 < nblk64)
        v = Dinv64[static_cast<int64_t>(b64) * kSmall * kSmall + (r % kSmall) + (c % kSmall) * kSmall];
      else
        v = r == c ? 1.0 : 0.0;
    }
    float2 pv;
    split_pair(v, pv.x, pv.y);
    Y[idx] = pv;
  }
}

// Operator entries as FP32 pairs (hi, lo): an FP32 entry of R is (x, 0); an FP64 entry
// is split (split_pair); a pair of the block inverses (stored as pairs) is itself.
__device__ __forceinline__ float2 as_pair(float x) { return make_float2(x, 0.f); }
__device__ __forceinline__ float2 as_pair(double x) {
  float2 r;
  split_pair(x, r.x, r.y);
  return r;
}
__device__ __forceinline__ float2 as_pair(float2 x) { return x; }
template <typename Mt> __device__ __forceinline__ Mt zero_of() { return Mt(0); }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.f, 0.f); }

// acc (an unevaluated FP32 pair) += a * b for FP32 pairs a, b: the leading product exact
// as p + e by an FMA, the cross terms added to the error, Knuth's TwoSum for the sum.
__device__ __forceinline__ void df_mac(float2 &acc, float2 a, float2 b) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p) + fmaf(a.x, b.y, a.y * b.x);
  const float t = acc.x + p;
  const float bb = t - acc.x;
  acc.y += ((acc.x - (t - bb)) + (p - bb)) + e;
  acc.x = t;
}

// One doubling step at half-width h for every pair of every big block, in two products:
//   stage 0: Tmp = Y11 R12        stage 1: Y12 = -Tmp Y22
// Y11 = Y[s](p, p), Y22 = Y[s](p+h, p+h) (h x h, already inverses), R12 = R(p, p+h) of
// big block s (zero beyond n), p = 2 h q; Y and Tmp hold FP32 pairs and the products run
// in double-float arithmetic on the FP32 units (about 2^-44 relative per sum).  32 x 32
// output tile per CTA, 2 x 2 per thread: both factors with an inverse are upper triangular
// (Y11(row, k) = 0 for k < row in stage 0, Y22(k, col) = 0 for k > col in stage 1), so
// each tile's k range stops at the triangle, and the small tiles spread the uneven ranges
// over all SMs.
template <typename Real>
__global__ void __launch_bounds__(kThreads) merge_kernel(int64_t n, const Real *R, int64_t ldr, float2 *Y,
                                                         float2 *Tmp, int h, int stage) {
  constexpr int kM = 32;
  __shared__ float2 As[kM][kM + 1];
  __shared__ float2 Bs[kM][kM + 1];
  const int tiles = h / kM;
  const int tr = blockIdx.x % tiles, tc = blockIdx.x / tiles;  // output tile
  const int q = blockIdx.y, s = blockIdx.z;
  const int p = 2 * h * q;
  float2 *Ys = Y + static_cast<int64_t>(s) * kBig * kBig;
  float2 *Tq = Tmp + (static_cast<int64_t>(s) * (kBig / (2 * h)) + q) * h * h;
  const int64_t g0 = static_cast<int64_t>(s) * kBig;  // first row of the big block in R
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  float2 acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = make_float2(0.f, 0.f);
  const int k_lo = stage == 0 ? tr * kM : 0;
  const int k_hi = stage == 0 ? h : (tc * kM + kM < h ? tc * kM + kM : h);
  for (int k0 = k_lo; k0 < k_hi; k0 += kM) {
    // A tile: kM rows x kM k;  B tile: kM k x kM cols
    for (int idx = tid; idx < kM * kM; idx += kThreads) {
      const int kk = idx / kM, r = idx % kM;
      const int row = tr * kM + r, k = k0 + kk;
      As[r][kk] = stage == 0 ? Ys[(p + row) + static_cast<int64_t>(p + k) * kBig] : Tq[row + static_cast<int64_t>(k) * h];
    }
    for (int idx = tid; idx < kM * kM; idx += kThreads) {
      const int c = idx / kM, kk = idx % kM;
      const int col = tc * kM + c, k = k0 + kk;
      float2 v;
      if (stage == 0) {
        const int64_t gr = g0 + p + k, gc = g0 + p + h + col;
        v = (gr < n && gc < n) ? as_pair(__ldcg(R + gr + gc * ldr)) : make_float2(0.f, 0.f);
      } else {
        v = Ys[(p + h + k) + static_cast<int64_t>(p + h + col) * kBig];
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kM; ++kk) {
      const float2 a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
      const float2 b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      df_mac(acc[0][0], a0, b0);
      df_mac(acc[0][1], a0, b1);
      df_mac(acc[1][0], a1, b0);
      df_mac(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int row = tr * kM + ty * 2 + u, col = tc * kM + tx * 2 + v;
      // renormalised pair (|lo| <= half an ulp of hi)
      const float hi = acc[u][v].x + acc[u][v].y;
      const float lo = acc[u][v].y - (hi - acc[u][v].x);
      if (stage == 0)
        Tq[row + static_cast<int64_t>(col) * h] = make_float2(hi, lo);
      else
        Ys[(p + row) + static_cast<int64_t>(p + h + col) * kBig] = make_float2(-hi, -lo);
    }
}

// Rt = R^T of the upper triangle (column-major n x n, ld n; zero below its diagonal), so
// that the update of the upper solve reads contiguous columns like the lower one.
template <typename Real>
__global__ void transpose_upper_kernel(int64_t n, const Real *R, int64_t ldr, Real *Rt) {
  __shared__ Real t[32][33];
  const int64_t bi = static_cast<int64_t>(blockIdx.y) * 32, bj = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  if (bi > bj + 31) {  // R's tile is below its diagonal: the Rt tile (rows bj.., columns bi..) is zero
    for (int y = ty; y < 32; y += 8)
      if (bj + tx < n && bi + y < n) Rt[(bj + tx) + (bi + y) * n] = Real(0);
    return;
  }
  for (int y = ty; y < 32; y += 8) {
    const int64_t r = bi + tx, c = bj + y;  // R(r, c)
    t[y][tx] = (r < n && c < n && r <= c) ? R[r + c * ldr] : Real(0);
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int64_t rr = bj + tx, cc = bi + y;  // Rt(rr, cc) = R(cc, rr)
    if (rr < n && cc < n) Rt[rr + cc * n] = t[tx][y];
  }
}

// ---- solve ----------------------------------------------------------------------------

// Grid barrier of a cooperative launch: every CTA arrives once per phase; the counter
// only grows, so barrier g waits for g * gridDim.x arrivals.  Bounded like every wait.
__device__ bool grid_barrier(int32_t *bar, int &gen, int32_t *status, int64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++gen;
    __threadfence();
    atomicAdd(bar, 1);
    const int target = gen * static_cast<int>(gridDim.x);
    int ok = 1;
    const uint64_t t0 = gtimer();
    for (uint64_t it = 0; ld_acq(bar) < target; ++it) {
      if (*(volatile int32_t *)status != 0) {
        ok = 0;
        break;
      }
      if (gtimer() - t0 > static_cast<uint64_t>(limit_ns) || it > (static_cast<uint64_t>(limit_ns) >> 4) + 1000000ull) {
        atomicCAS(status, 0, kStatusTimeout | (0x7ffff0 << 8));
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One warp's 32 x 64 tile of an operator, Op(i, c) for rows i0.. (i < ilim) and columns
// c0.. (c < clim), staged in the warp's shared-memory slice as FP32 pairs st[c][i - i0]:
// Op(i, c) = M[i + c*ldm] (kTrans = false: lanes read consecutive rows) or M[c + i*ldm]
// (kTrans = true: lanes read consecutive columns).  The loads are unrolled so that many
// are in flight; the tile does not depend on the solution, so it is fetched before the
// grid barrier that precedes its use.
template <typename Mt, bool kTrans>
__device__ void tile_load(float2 (*st)[33], const Mt *M, int64_t ldm, int64_t i0, int64_t ilim, int64_t c0,
                          int64_t clim) {
  const int lane = threadIdx.x & 31;
  // groups of 32 loads into registers, then the shared-memory stores: every load of a
  // group is in flight before the first store needs its value
  constexpr int kGroup = 32;
  if (!kTrans) {
    const int64_t i = i0 + lane;
    const bool ok = i < ilim;
    for (int cb = 0; cb < 64; cb += kGroup) {
      Mt v[kGroup];
#pragma unroll
      for (int u = 0; u < kGroup; ++u)
        v[u] = (ok && c0 + cb + u < clim) ? __ldcg(M + i + (c0 + cb + u) * ldm) : zero_of<Mt>();
#pragma unroll
      for (int u = 0; u < kGroup; ++u) st[cb + u][lane] = as_pair(v[u]);
    }
  } else {
    constexpr int kRows = kGroup / 2;
    for (int ib = 0; ib < 32; ib += kRows) {
      Mt v[kGroup];
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int64_t row = i0 + ib + u;
        const bool ok = row < ilim;
        v[2 * u] = (ok && c0 + lane < clim) ? __ldcg(M + (c0 + lane) + row * ldm) : zero_of<Mt>();
        v[2 * u + 1] = (ok && c0 + 32 + lane < clim) ? __ldcg(M + (c0 + 32 + lane) + row * ldm) : zero_of<Mt>();
      }
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        st[lane][ib + u] = as_pair(v[2 * u]);
        st[lane + 32][ib + u] = as_pair(v[2 * u + 1]);
      }
    }
  }
  __syncwarp();
}

// out(i, j) += sign * sum_c st[c][i - i0] v(c0 + c, j) for the staged tile; kR right-hand
// sides.  The products run in double-float arithmetic on the FP32 units (operator entry
// and vector entry as FP32 pairs: the leading product exact as p + e by an FMA, the cross
// terms added to the error; Knuth's TwoSum keeps the running sum as an unevaluated pair) -
// about 2^-44 relative, with FP32 instructions instead of FP64 ones, which on this GPU
// bound a phase at one FP64 instruction per element; partial sums meet in FP64 atomics.
template <int kR>
__device__ void tile_apply_r(float2 (*st)[33], int64_t i0, int64_t ilim, int64_t c0, int64_t clim, const double *v,
                             int64_t ldv, double *out, int64_t ldo, double sign) {
  const int lane = threadIdx.x & 31;
  float2 va[kR], vb[kR];
#pragma unroll
  for (int j = 0; j < kR; ++j) {
    va[j] = as_pair(c0 + lane < clim ? __ldcg(v + (c0 + lane) + j * ldv) : 0.0);
    vb[j] = as_pair(c0 + 32 + lane < clim ? __ldcg(v + (c0 + 32 + lane) + j * ldv) : 0.0);
  }
  float hi[kR], lo[kR];
#pragma unroll
  for (int j = 0; j < kR; ++j) hi[j] = lo[j] = 0.f;
#pragma unroll 8
  for (int c = 0; c < 64; ++c) {
    const float2 m = st[c][lane];
#pragma unroll
    for (int j = 0; j < kR; ++j) {
      const float xh = __shfl_sync(0xffffffffu, c < 32 ? va[j].x : vb[j].x, c & 31);
      const float xl = __shfl_sync(0xffffffffu, c < 32 ? va[j].y : vb[j].y, c & 31);
      const float p = m.x * xh;
      const float e = fmaf(m.x, xh, -p) + fmaf(m.x, xl, m.y * xh);
      const float t = hi[j] + p;
      const float bb = t - hi[j];
      lo[j] += ((hi[j] - (t - bb)) + (p - bb)) + e;
      hi[j] = t;
    }
  }
  const int64_t i = i0 + lane;
  if (i < ilim) {
#pragma unroll
    for (int j = 0; j < kR; ++j)
      atomicAdd(out + i + j * ldo, sign * (static_cast<double>(hi[j]) + static_cast<double>(lo[j])));
  }
  __syncwarp();  // the slice may be refilled next
}

__device__ void tile_apply(float2 (*st)[33], int64_t i0, int64_t ilim, int64_t c0, int64_t clim, const double *v,
                           int64_t ldv, double *out, int64_t ldo, int nrhs, double sign) {
  switch (nrhs) {
    case 1: tile_apply_r<1>(st, i0, ilim, c0, clim, v, ldv, out, ldo, sign); break;
    case 2: tile_apply_r<2>(st, i0, ilim, c0, clim, v, ldv, out, ldo, sign); break;
    case 3: tile_apply_r<3>(st, i0, ilim, c0, clim, v, ldv, out, ldo, sign); break;
    default: tile_apply_r<4>(st, i0, ilim, c0, clim, v, ldv, out, ldo, sign); break;
  }
}

// Solves R X = B (kLowerT = false) or R^T X = B (true) in place, nrhs <= kRhsMax.
// Y: the big-block inverses; xs: 2 x kBig x kRhsMax doubles (zeroed by the launcher);
// bar: the grid barrier counter (zeroed by the launcher).  Work items are 32 x 64 tiles,
// one per warp while there are enough warps; a warp's first tile of each phase is staged
// before the barrier that precedes the phase.
template <typename Real, bool kLowerT>
__global__ void __launch_bounds__(kThreads) big_trsv_kernel(int64_t n, const Real *R, int64_t ldr, const Real *Rt,
                                                            const float2 *Y, double *B, int64_t ldb, int nrhs,
                                                            double *xs, int32_t *bar, int32_t *status,
                                                            int64_t limit_ns) {
  extern __shared__ float2 pc_smem[];
  float2(*st)[33] = reinterpret_cast<float2(*)[33]>(pc_smem + (threadIdx.x >> 5) * 64 * 33);
  const int nbig = static_cast<int>((n + kBig - 1) / kBig);
  const int warp = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * kWarps + warp, nwarps = gridDim.x * kWarps;
  int gen = 0;
  // phase-1 tiles: the triangle of Y_s (or Y_s^T) in (kBig / 32) x kCT tiles of 32 x 64
  auto p1_skip = [&](int item) {
    const int r0 = (item / kCT) * 32, c0 = (item % kCT) * 64;
    return kLowerT ? (c0 > r0 + 31) : (c0 + 63 < r0);
  };
  auto p1_first = [&]() {
    for (int item = gwarp; item < kP1; item += nwarps)
      if (!p1_skip(item)) return item;
    return -1;
  };
  auto block_of = [&](int step) { return kLowerT ? step : nbig - 1 - step; };
  auto load_p1 = [&](int step, int item) {
    const int s = block_of(step);
    const int64_t g0 = static_cast<int64_t>(s) * kBig;
    const int rb = static_cast<int>(lmin(kBig, n - g0));
    tile_load<float2, kLowerT>(st, Y + static_cast<int64_t>(s) * kBig * kBig, kBig, (item / kCT) * 32, rb,
                               (item % kCT) * 64, rb);
  };
  // phase-2 rows of step: [lo, hi)
  auto p2_range = [&](int step, int64_t &lo, int64_t &hi, int64_t &g0, int &rb) {
    const int s = block_of(step);
    g0 = static_cast<int64_t>(s) * kBig;
    rb = static_cast<int>(lmin(kBig, n - g0));
    lo = kLowerT ? g0 + rb : 0;
    hi = kLowerT ? n : g0;
  };
  auto load_p2 = [&](int step, int64_t item) {
    int64_t lo, hi, g0;
    int rb;
    p2_range(step, lo, hi, g0, rb);
    const int64_t i0 = lo + (item / kCT) * 32;
    const int c0 = static_cast<int>(item % kCT) * 64;
    if (!kLowerT)  // R(i, g0 + c) = Rt(g0 + c, i)
      tile_load<Real, true>(st, Rt + g0, n, i0, hi, c0, rb);
    else           // R^T(i, g0 + c) = R(g0 + c, i)
      tile_load<Real, true>(st, R + g0, ldr, i0, hi, c0, rb);
  };
  const int first1 = p1_first();
  if (first1 >= 0) load_p1(0, first1);
  for (int step = 0; step < nbig; ++step) {
    const int s = block_of(step);
    const int64_t g0 = static_cast<int64_t>(s) * kBig;
    const int rb = static_cast<int>(lmin(kBig, n - g0));
    double *x = xs + (step & 1) * kBig * kRhsMax;
    double *xo = xs + ((step + 1) & 1) * kBig * kRhsMax;
    // phase 1: x = Y_s b_s (or Y_s^T b_s)
    for (int item = gwarp; item < kP1; item += nwarps) {
      if (p1_skip(item)) continue;
      if (item != first1) load_p1(step, item);
      tile_apply(st, (item / kCT) * 32, rb, (item % kCT) * 64, rb, B + g0, ldb, x, kBig, nrhs, 1.0);
    }
    int64_t lo, hi, g0b;
    int rbb;
    p2_range(step, lo, hi, g0b, rbb);
    const int64_t nitem2 = ((hi - lo + 31) / 32) * kCT;
    if (gwarp < nitem2) load_p2(step, gwarp);
    if (!grid_barrier(bar, gen, status, limit_ns)) return;
    // phase 2: the remaining rows lose R's coupling to block s; block s's rows take x
    if (blockIdx.x == 0) {
      for (int idx = threadIdx.x; idx < kBig * nrhs; idx += kThreads) {
        const int j = idx / kBig, r = idx - j * kBig;
        if (r < rb) B[g0 + r + j * ldb] = __ldcg(x + r + j * kBig);
        xo[r + j * kBig] = 0.0;  // the other buffer, read by no one in this phase
      }
    }
    for (int64_t item = gwarp; item < nitem2; item += nwarps) {
      if (item != gwarp) load_p2(step, item);
      const int64_t i0 = lo + (item / kCT) * 32;
      const int c0 = static_cast<int>(item % kCT) * 64;
      tile_apply(st, i0, hi, c0, rb, x, kBig, B, ldb, nrhs, -1.0);
    }
    if (step + 1 < nbig && first1 >= 0) load_p1(step + 1, first1);
    if (!grid_barrier(bar, gen, status, limit_ns)) return;
  }
}

template <typename Real>
int setup_typed(int64_t n, const Real *R, int64_t ldr, const double *Dinv64, float2 *Y, float2 *Tmp, Real *Rt,
                cudaStream_t st) {
  const int nbig = static_cast<int>((n + kBig - 1) / kBig);
  {
    const dim3 tg(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((n + 31) / 32));
    transpose_upper_kernel<Real><<<tg, kThreads, 0, st>>>(n, R, ldr, Rt);
    count_launch();
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return static_cast<int>(e0);
  }
  big_init_kernel<<<1216, kThreads, 0, st>>>(n, Dinv64, Y, nbig);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_cast<int>(e);
  for (int h = kSmall; h < kBig; h *= 2) {
    const int tiles = (h / 32) * (h / 32);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(kBig / (2 * h)), static_cast<unsigned>(nbig));
    for (int stage = 0; stage < 2; ++stage) {
      merge_kernel<Real><<<grid, kThreads, 0, st>>>(n, R, ldr, Y, Tmp, h, stage);
      count_launch();
      if ((e = cudaGetLastError()) != cudaSuccess) return static_cast<int>(e);
    }
  }
  return 0;
}

template <typename Real, bool kLowerT>
int solve_typed(int64_t n, const Real *R, int64_t ldr, const Real *Rt, const float2 *Y, double *B, int64_t ldb,
                int64_t nrhs, double *xs, int32_t *bar, int32_t *status, int64_t limit_ns, cudaStream_t st) {
  auto kern = big_trsv_kernel<Real, kLowerT>;
  const size_t smem = sizeof(float2) * kWarps * 64 * 33;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  if (per_sm < 1) return static_cast<int>(cudaErrorCooperativeLaunchTooLarge);
  const int grid = nsm;  // one CTA per SM: all co-resident, as the grid barrier needs
  for (int64_t j0 = 0; j0 < nrhs; j0 += kRhsMax) {
    int nr = static_cast<int>(nrhs - j0 < kRhsMax ? nrhs - j0 : kRhsMax);
    if ((e = cudaMemsetAsync(xs, 0, sizeof(double) * 2 * kBig * kRhsMax, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(bar, 0, sizeof(int32_t), st)) != cudaSuccess)
      return static_cast<int>(e);
    double *Bj = B + j0 * ldb;
    void *args[] = {&n, &R, &ldr, &Rt, &Y, &Bj, &ldb, &nr, &xs, &bar, &status, &limit_ns};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<void *>(kern), dim3(grid), dim3(kThreads), args, smem, st);
    count_launch();
    if (e != cudaSuccess) return static_cast<int>(e);
  }
  return 0;
}

}  // namespace

size_t precond_work_doubles(int64_t n, bool real_is_double) {
  const size_t nbig = static_cast<size_t>((n + kBig - 1) / kBig);
  const size_t nn = static_cast<size_t>(n) * static_cast<size_t>(n);
  // Y, the doubling products (at most kBig/2 squared per big block), two x buffers, and
  // R^T (n x n in R's element type)
  return nbig * kBig * kBig + nbig * (kBig / 2) * (kBig / 2) + 2 * kBig * kRhsMax +
         (real_is_double ? nn : (nn + 1) / 2);
}

namespace {
struct Layout {
  float2 *Y, *Tmp;  // FP32 pairs (one double's storage each)
  double *xs;
  void *Rt;
};
Layout layout(int64_t n, const double *work) {
  const size_t nbig = static_cast<size_t>((n + kBig - 1) / kBig);
  Layout l;
  double *w = const_cast<double *>(work);
  l.Y = reinterpret_cast<float2 *>(w);
  l.Tmp = reinterpret_cast<float2 *>(w + nbig * kBig * kBig);
  l.xs = w + nbig * kBig * kBig + nbig * (kBig / 2) * (kBig / 2);
  l.Rt = l.xs + 2 * kBig * kRhsMax;
  return l;
}
}  // namespace

int precond_setup(int64_t n, const void *R, int64_t ldr, bool real_is_double, const double *Dinv64, double *work,
                  void *stream) {
  const Layout l = layout(n, work);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return real_is_double
             ? setup_typed(n, static_cast<const double *>(R), ldr, Dinv64, l.Y, l.Tmp, static_cast<double *>(l.Rt), st)
             : setup_typed(n, static_cast<const float *>(R), ldr, Dinv64, l.Y, l.Tmp, static_cast<float *>(l.Rt), st);
}

int precond_solve(int64_t n, const void *R, int64_t ldr, bool real_is_double, const double *work, double *B,
                  int64_t ldb, int64_t nrhs, int32_t *bar, int32_t *status, int64_t wait_limit_ns, void *stream,
                  bool lower_transposed) {
  const Layout l = layout(n, work);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (real_is_double) {
    const double *Rd = static_cast<const double *>(R), *Rt = static_cast<const double *>(l.Rt);
    return lower_transposed ? solve_typed<double, true>(n, Rd, ldr, Rt, l.Y, B, ldb, nrhs, l.xs, bar, status,
                                                        wait_limit_ns, st)
                            : solve_typed<double, false>(n, Rd, ldr, Rt, l.Y, B, ldb, nrhs, l.xs, bar, status,
                                                         wait_limit_ns, st);
  }
  const float *Rf = static_cast<const float *>(R), *Rt = static_cast<const float *>(l.Rt);
  return lower_transposed
             ? solve_typed<float, true>(n, Rf, ldr, Rt, l.Y, B, ldb, nrhs, l.xs, bar, status, wait_limit_ns, st)
             : solve_typed<float, false>(n, Rf, ldr, Rt, l.Y, B, ldb, nrhs, l.xs, bar, status, wait_limit_ns, st);
}

}  // namespace tqr
