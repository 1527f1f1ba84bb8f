// Persistent tile-task executor and the SIMT tile kernels GEQRT, TTQRT, UNMQR, TTMQR
// (Table "Kernels for tiled QR"; TT elimination of Algorithm "elimTR", Section 3.1.1).
//
// One launch runs a whole task graph.  Each CTA repeatedly claims the next task index
// (executor order is topological), waits until the task's predecessor counter reaches
// zero, runs the kernel with all 256 threads, and releases its successors.  Because a
// task only ever waits for tasks with a smaller index, which were claimed earlier by
// running CTAs, the executor cannot deadlock whatever the number of resident CTAs.
// Every wait is bounded (globaltimer deadline + iteration cap): on expiry the CTA
// records kStatusTimeout and the failing task in the status word and every CTA returns.
//
// Tiles are nb x nb blocks of the column-major matrix; a tile that sticks out of the
// m x n matrix is processed as if zero-padded: padded rows and columns are never read
// or written, and reflectors that would act only on padding have tau = 0.
//
// Reflector conventions (LAPACK): H = I - tau v v^T, v(0) = 1, beta = -sign(alpha) *
// ||[alpha; x]||, tau = (beta - alpha) / beta, v = x / (alpha - beta), tau = 0 when
// x = 0.  T factors: compact-WY (Schreiber & Van Loan, 1989), blocks of ib reflectors,
// stored ib x nb per factored tile (block b in columns b*ib..).  Householder sums of
// squares are FP64-accurate for every storage precision (FP32 storage accumulates them
// with error-free FP32 transformations); beta, tau and the scaling of v are formed in
// FP64 for FP64 storage and, from that sum, in FP32 for FP32 storage (FP64 outside the
// range where FP32 keeps full precision).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "tqr_internal.h"

namespace tqr {
namespace {

__host__ __device__ __forceinline__ int64_t lmin(int64_t a, int64_t b) { return a < b ? a : b; }

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Columns of an update chunk held in shared memory: 32 for FP32 storage, 16 for FP64
// (whose 256-row chunks would not fit twice in one SM's shared memory at 32).
__host__ __device__ constexpr int chunk_cols(size_t s_size) { return s_size == sizeof(float) ? 32 : 16; }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire_gpu(const int32_t *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int32_t *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Loads through L2 only: tiles written by other SMs must never be served from a stale
// L1 line of this SM.
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ double ldcg(const float *p) { return static_cast<double>(__ldcg(p)); }

// Optional phase accounting of one task for the execution trace: ph[0] holds the last
// timestamp, ph[1..4] accumulate the time spent in up to four phases (thread 0 only).
__device__ __forceinline__ void phase_mark(uint64_t *ph, int slot) {
  if (ph && threadIdx.x == 0) {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    ph[1 + slot] += t - ph[0];
    ph[0] = t;
  }
}

template <typename S>
__device__ __forceinline__ S warp_sum(S v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout of one CTA (element type S = compute type).
template <typename S>
struct Smem {
  S *tau_s;      // [ib] tau of each reflector of the current block
  S *scal_s;     // [ib] 1 / (alpha - beta) of each reflector of the block
  S *V;          // [ldv * ib]  panel / reflector block
  S *C;          // [ldv * chunk] update chunk (C, or C2 of a TT pair)
  S *C1;         // [ldv * chunk] C1 chunk of a TT pair
  S *W;          // [ldw * chunk]
  S *T;          // [ldt * ib]
  S *G;          // [ldt * ib]  Gram matrix of the reflectors of a block
  S *P1;         // [ldt * ib]  diagonal block of R(piv) during TTQRT
  float *Wv;     // FP32 storage: [32 * kWvLd] W by rows (16-byte aligned), else null
  float *red;    // FP32 storage: [3 * 32 * 33] partial sums of V^T C, else null
  int ldv, ldw, ldt;
  int ldp;       // leading dimension of P1 (ldt, or that of a resident pivot tile)
  uint64_t *ph;  // phase clock of the execution trace, or null
};

__host__ __device__ inline int odd_ld(int x) { return x | 1; }

// Row stride of the FP32 row-major copy of W (a multiple of 4 floats: 16-byte rows).
constexpr int kWvLd = 36;
constexpr size_t kF32Extra = 16 + (32 * kWvLd + 3 * 32 * 33) * sizeof(float);

__host__ __device__ inline size_t smem_elems(int nb, int ib, size_t s_size) {
  const size_t ldv = odd_ld(nb), ldw = ib + 1, ldt = ib + 1;
  const size_t cw = chunk_cols(s_size);
  const size_t s_elems = ldv * ib + 2 * ldv * cw + ldw * cw + 3 * ldt * ib + 2 * ib;
  return s_elems * s_size + (s_size == sizeof(float) ? kF32Extra : 0);
}

template <typename S>
__device__ Smem<S> carve(unsigned char *raw, int nb, int ib) {
  Smem<S> s;
  s.ldv = odd_ld(nb);
  s.ldw = ib + 1;
  s.ldt = ib + 1;
  s.ldp = s.ldt;
  S *p = reinterpret_cast<S *>(raw);
  s.V = p;
  p += s.ldv * ib;
  s.C = p;
  p += s.ldv * chunk_cols(sizeof(S));
  s.C1 = p;
  p += s.ldv * chunk_cols(sizeof(S));
  s.W = p;
  p += s.ldw * chunk_cols(sizeof(S));
  s.T = p;
  p += s.ldt * ib;
  s.G = p;
  p += s.ldt * ib;
  s.P1 = p;
  p += s.ldt * ib;
  s.tau_s = p;
  p += ib;
  s.scal_s = p;
  p += ib;
  s.Wv = nullptr;
  s.red = nullptr;
  if (sizeof(S) == sizeof(float)) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~static_cast<uintptr_t>(15);
    s.Wv = reinterpret_cast<float *>(a);
    s.red = s.Wv + 32 * kWvLd;
  }
  return s;
}

// Tile loads keep many loads in flight per thread: every load of a pass is issued before
// the first shared-memory store, so their latencies (hundreds of cycles from L2 or HBM)
// overlap instead of adding up element by element.
//
// dst[r + c*ldd] = value(r, c) for r < nrows, c < ncols, where mode(r, c) selects the
// value: kLoad -> src[r + c*lds] (through L2), kOne -> 1, kZero -> 0.  Warps take columns,
// lanes rows; a pass covers kCU columns per warp and kRG groups of 32 rows.
enum : int { kZero = 0, kOne = 1, kLoad = 2 };

template <int kRG, int kCU, typename S, typename G, typename Mode>
__device__ __forceinline__ void load_block_pass(S *dst, int ldd, const G *src, int64_t lds, int nrows,
                                                int ncols, Mode mode) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r0 = 0; r0 < nrows; r0 += 32 * kRG)
    for (int c0 = warp; c0 < ncols; c0 += kWarps * kCU) {
      S v[kCU][kRG];
#pragma unroll
      for (int u = 0; u < kCU; ++u)
#pragma unroll
        for (int g = 0; g < kRG; ++g) {
          const int c = c0 + kWarps * u, r = r0 + lane + 32 * g;
          const int md = (c < ncols && r < nrows) ? mode(r, c) : kZero;
          v[u][g] = md == kLoad ? static_cast<S>(ldcg(src + r + static_cast<int64_t>(c) * lds))
                                : (md == kOne ? S(1) : S(0));
        }
#pragma unroll
      for (int u = 0; u < kCU; ++u)
#pragma unroll
        for (int g = 0; g < kRG; ++g) {
          const int c = c0 + kWarps * u, r = r0 + lane + 32 * g;
          if (c < ncols && r < nrows) dst[r + c * ldd] = v[u][g];
        }
    }
}

template <typename S, typename G, typename Mode>
__device__ void load_block_mode(S *dst, int ldd, const G *src, int64_t lds, int nrows, int ncols, Mode mode) {
  if (nrows <= 128)
    load_block_pass<4, 4>(dst, ldd, src, lds, nrows, ncols, mode);
  else
    load_block_pass<8, 2>(dst, ldd, src, lds, nrows, ncols, mode);
}

// dst[r + c*ldd] = src[r + c*lds], r < nrows, c < ncols.
template <typename S, typename G>
__device__ void load_block(S *dst, int ldd, const G *src, int64_t lds, int nrows, int ncols) {
  load_block_mode(dst, ldd, src, lds, nrows, ncols, [](int, int) { return static_cast<int>(kLoad); });
}

template <typename S, typename G>
__device__ void store_block(G *dst, int64_t ldd, const S *src, int lds, int nrows, int ncols) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < ncols; c += kWarps)
    for (int r = lane; r < nrows; r += 32)
      dst[r + static_cast<int64_t>(c) * ldd] = static_cast<G>(src[r + c * lds]);
}

// Applies the block reflector of kb reflectors to a chunk of ncols columns:
//   W = [C1(0:kb, :)] + V^T C          (C1 present for TT pairs: identity part)
//   W = T^T W  (Q^T, transpose_q = false)   or   W = T W  (Q, transpose_q = true)
//   C1(0:kb, :) -= W,   C -= V W
// V is nrows x kb (explicit zeros / unit entries), T upper triangular kb x kb.
//
// FP32 storage (s.Wv, s.red present) takes a register-blocked form: V^T C as 4 x 4 blocks
// of W per thread over a quarter of the rows (four row groups, partial sums added in
// shared memory), and C -= V W with 8 columns of a W row per 16-byte load.  Each thread
// keeps the summation order of its own partial sums, so results are deterministic.
__device__ void apply_block_f32(float *C, int ldc, int nrows, float *C1, int ldc1, int ncols, const float *V,
                                int ldv, const float *T, int ldt, int kb, float *Wv, float *red, bool transpose_q) {
  const int tid = threadIdx.x;
  {
    // W = C1 + V^T C: thread -> 4 x 4 block (a = 4 ab + x, c = 4 cb + y), row group rg
    const int blk = tid & 63, rg = tid >> 6;
    const int ab = blk & 7, cb = blk >> 3;
    const float *va[4], *cc[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) va[x] = V + min(4 * ab + x, kb - 1) * ldv;
#pragma unroll
    for (int y = 0; y < 4; ++y) cc[y] = C + min(4 * cb + y, ncols - 1) * ldc;
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int r = rg; r < nrows; r += 4) {
      float v[4], c[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) v[x] = va[x][r];
#pragma unroll
      for (int y = 0; y < 4; ++y) c[y] = cc[y][r];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += v[x] * c[y];
    }
    if (rg > 0) {
      float *part = red + (rg - 1) * 32 * 33;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) part[(4 * ab + x) + (4 * cb + y) * 33] = acc[x][y];
    }
    __syncthreads();
    if (rg == 0) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int a = 4 * ab + x, c = 4 * cb + y, o = a + c * 33;
          float w = acc[x][y] + red[o] + red[32 * 33 + o] + red[2 * 32 * 33 + o];
          if (a < kb && c < ncols) {
            if (C1) w += C1[a + c * ldc1];
            red[o] = w;  // the full sum replaces this slot of the first partial buffer
          }
        }
    }
    __syncthreads();
  }
  {
    // W = op(T) W (W read from red's first buffer, ld 33); C1 -= W; W kept by rows in Wv
    const int a = tid & 31, g = tid >> 5;
    float nw[4] = {0.f, 0.f, 0.f, 0.f};
    if (a < kb) {
      // the four columns' sums advance together (one T load, four independent FMA chains
      // per step); each sum still runs over b in order.  Columns beyond ncols read
      // unused slots of red and are not stored.
      const float *r0 = red + g * 33;
      if (!transpose_q) {
        for (int b = 0; b <= a; ++b) {
          const float t = T[b + a * ldt];
#pragma unroll
          for (int u = 0; u < 4; ++u) nw[u] += t * r0[b + kWarps * 33 * u];
        }
      } else {
        for (int b = a; b < kb; ++b) {
          const float t = T[a + b * ldt];
#pragma unroll
          for (int u = 0; u < 4; ++u) nw[u] += t * r0[b + kWarps * 33 * u];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = g + kWarps * u;
        if (c < ncols) {
          Wv[a * kWvLd + c] = nw[u];
          if (C1) C1[a + c * ldc1] -= nw[u];
        }
      }
    }
    __syncthreads();
  }
  {
    // C -= V W: thread -> rows rt + 64 x (x < NX, the row groups the block has),
    // columns 8 cg .. 8 cg + 7
    const int rt = tid & 63, cg = tid >> 6;
    auto rows_times_w = [&](auto nx) {
      constexpr int NX = decltype(nx)::value;
      float acc[NX][8];
#pragma unroll
      for (int x = 0; x < NX; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
      int rr[NX];
#pragma unroll
      for (int x = 0; x < NX; ++x) rr[x] = min(rt + 64 * x, nrows - 1);
#pragma unroll 4
      for (int b = 0; b < kb; ++b) {
        const float4 w0 = *reinterpret_cast<const float4 *>(Wv + b * kWvLd + 8 * cg);
        const float4 w1 = *reinterpret_cast<const float4 *>(Wv + b * kWvLd + 8 * cg + 4);
        const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int x = 0; x < NX; ++x) {
          const float v = V[rr[x] + b * ldv];
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] += v * w[y];
        }
      }
#pragma unroll
      for (int x = 0; x < NX; ++x) {
        const int r = rt + 64 * x;
        if (r < nrows) {
#pragma unroll
          for (int y = 0; y < 8; ++y) {
            const int c = 8 * cg + y;
            if (c < ncols) C[r + c * ldc] -= acc[x][y];
          }
        }
      }
    };
    if (8 * cg < ncols) {
      switch ((nrows + 63) / 64) {
        case 1: rows_times_w(std::integral_constant<int, 1>{}); break;
        case 2: rows_times_w(std::integral_constant<int, 2>{}); break;
        case 3: rows_times_w(std::integral_constant<int, 3>{}); break;
        default: rows_times_w(std::integral_constant<int, 4>{}); break;
      }
    }
    __syncthreads();
  }
}

template <typename S>
__device__ void apply_block(S *C, int ldc, int nrows, S *C1, int ldc1, int ncols, const S *V,
                            int ldv, const S *T, int ldt, int kb, S *W, int ldw, bool transpose_q,
                            float *Wv = nullptr, float *red = nullptr) {
  if constexpr (sizeof(S) == sizeof(float)) {
    if (Wv) {
      apply_block_f32(C, ldc, nrows, C1, ldc1, ncols, V, ldv, T, ldt, kb, Wv, red, transpose_q);
      return;
    }
  }
  // Each phase spreads its outputs over all threads (a small kb or a short tile leaves no
  // thread idle; FP64 instructions are the cost on this GPU), and each output's sum runs
  // in a fixed order, so results are deterministic.
  const int tid = threadIdx.x;
  constexpr int kMaxOut = 4;  // outputs of W per thread: kb * ncols <= 32 * 32
  static_assert(kMaxOut * kThreads >= 32 * 32, "W outputs per thread");
  // W = C1 + V^T C: output (a, c) per thread step, a fastest (V loads hit distinct banks,
  // C loads broadcast); two partial sums over even and odd rows
  for (int idx = tid; idx < kb * ncols; idx += kThreads) {
    const int c = idx / kb, a = idx - c * kb;
    const S *va = V + a * ldv, *cc = C + c * ldc;
    S acc0 = 0, acc1 = 0;
    int r = 0;
    for (; r + 1 < nrows; r += 2) {
      acc0 += va[r] * cc[r];
      acc1 += va[r + 1] * cc[r + 1];
    }
    if (r < nrows) acc0 += va[r] * cc[r];
    W[a + c * ldw] = (acc0 + acc1) + (C1 ? C1[a + c * ldc1] : S(0));
  }
  __syncthreads();
  // W = op(T) W, every output formed before any is stored
  S nw[kMaxOut];
#pragma unroll
  for (int u = 0; u < kMaxOut; ++u) {
    const int idx = tid + u * kThreads;
    nw[u] = 0;
    if (idx < kb * ncols) {
      const int c = idx / kb, a = idx - c * kb;
      S s = 0;
      if (!transpose_q) {
        for (int b = 0; b <= a; ++b) s += T[b + a * ldt] * W[b + c * ldw];
      } else {
        for (int b = a; b < kb; ++b) s += T[a + b * ldt] * W[b + c * ldw];
      }
      nw[u] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kMaxOut; ++u) {
    const int idx = tid + u * kThreads;
    if (idx < kb * ncols) {
      const int c = idx / kb, a = idx - c * kb;
      W[a + c * ldw] = nw[u];
      if (C1) C1[a + c * ldc1] -= nw[u];
    }
  }
  __syncthreads();
  // C -= V W: row r and four consecutive columns per thread step, r fastest
  const int ngrp = (ncols + 3) / 4;
  for (int idx = tid; idx < nrows * ngrp; idx += kThreads) {
    const int g = idx / nrows, r = idx - g * nrows;
    const int c0 = 4 * g;
    const S *w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) w[u] = W + min(c0 + u, ncols - 1) * ldw;
    S acc[4] = {0, 0, 0, 0};
    for (int b = 0; b < kb; ++b) {
      const S v = V[r + b * ldv];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += v * w[u][b];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (c0 + u < ncols) C[r + (c0 + u) * ldc] -= acc[u];
  }
  __syncthreads();
}

// FP64 reflector parameters from alpha and ||x||^2 (LAPACK convention):
// beta = -sign(alpha) sqrt(alpha^2 + ||x||^2), tau = (beta - alpha) / beta,
// scal = 1 / (alpha - beta).  With p = beta (alpha - beta), one reciprocal d = 1/p gives
// both 1/beta = (alpha - beta) d and scal = beta d.  1/sqrt and 1/p start from FP32 seeds
// and take two Newton steps in FP64 (quadratic convergence: 2^-23 -> 2^-46 -> FP64
// rounding), which is shorter on this GPU's FP64 pipe than sqrt and two divisions.
template <int kNewton>
__device__ __forceinline__ void reflector(double alpha, double xx, double *beta, double *tau,
                                          double *scal) {
  if (xx == 0.0) {
    *beta = alpha;
    *tau = 0.0;
    *scal = 0.0;
    return;
  }
  const double s = fma(alpha, alpha, xx);
  if (!(s > 1e-30 && s < 1e30)) {  // outside the FP32 seed range: plain FP64 operations
    const double nrm = sqrt(s);
    const double b = alpha >= 0.0 ? -nrm : nrm;
    *beta = b;
    *tau = (b - alpha) / b;
    *scal = 1.0 / (alpha - b);
    return;
  }
  double r = static_cast<double>(rsqrtf(static_cast<float>(s)));
#pragma unroll
  for (int it = 0; it < kNewton; ++it) {
    const double h = fma(-s * r, r, 1.0);  // 1 - s r^2
    r = fma(0.5 * r, h, r);
  }
  const double nrm = s * r;
  const double b = alpha >= 0.0 ? -nrm : nrm;
  const double amb = alpha - b;
  const double pp = b * amb;
  double d = static_cast<double>(1.0f / static_cast<float>(pp));
#pragma unroll
  for (int it = 0; it < kNewton; ++it) d = fma(d, fma(-pp, d, 1.0), d);
  *beta = b;
  *scal = b * d;
  *tau = fma(-alpha, amb * d, 1.0);
}

// Sum of squares of FP32 values to FP64 accuracy with FP32 instructions: each square
// is split exactly (x*x = p + e, e = fma(x, x, -p)) and the parts are accumulated with
// error-free TwoSum (Knuth) into a (hi, lo) pair; the pair is converted to FP64 once.
struct DFloat {
  float hi, lo;
};

__device__ __forceinline__ DFloat df_add(DFloat a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b - bb);
  return DFloat{s, a.lo + err};
}

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
  DFloat r = df_add(a, b.hi);
  r.lo += b.lo;
  return r;
}

__device__ __forceinline__ DFloat df_sq_acc(DFloat acc, float x) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  DFloat r = df_add(acc, p);
  r.lo += e;
  return r;
}

__device__ __forceinline__ DFloat df_warp_reduce(DFloat v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DFloat w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

// FP32 reflector parameters (LAPACK convention, as reflector() above) from alpha and a
// double-float ||x||^2: alpha^2 is split exactly and added in double-float, so that
// s = alpha^2 + ||x||^2 carries one FP32 rounding; beta = -sign(alpha) sqrt(s),
// alpha - beta has no cancellation, tau = (beta - alpha) / beta, scal = 1 / (alpha - beta).
// Each scalar is within a few FP32 ulps, the precision they are stored in.  Returns false
// (nothing written) when s is outside the range where FP32 keeps full precision.
__device__ __forceinline__ bool reflector_f32(float alpha, DFloat xx, float *beta, float *tau, float *scal) {
  if (xx.hi == 0.f && xx.lo == 0.f) {
    *beta = alpha;
    *tau = 0.f;
    *scal = 0.f;
    return true;
  }
  const float a2 = alpha * alpha;
  DFloat sd = df_add(xx, a2);
  sd.lo += fmaf(alpha, alpha, -a2);
  const float sv = sd.hi + sd.lo;
  if (!(sv > 1e-30f && sv < 1e30f)) return false;
  const float nrm = sqrtf(sv);
  const float b = alpha >= 0.f ? -nrm : nrm;
  const float amb = alpha - b;
  *beta = b;
  *scal = 1.0f / amb;
  *tau = -amb / b;
  return true;
}

// Householder factorization of one panel block (kb columns) held in shared memory.
// kPanel selects the kernel: 0 GEQRT, 1 TTQRT, 2 TSQRT.
//   GEQRT: column c of s.V; head = V(c, c), tail = V(c+1 .. rows-1, c)
//   TT:    head = P1(c, c) (row c of R(piv)), tail = V(0 .. min(c0+c+1, mb)-1, c)
//   TS:    head = P1(c, c), tail = V(0 .. rows-1, c) (the whole square tile's column)
// Reflector c updates every later column cc of the block:
//   w = head(c, cc) + v . tail(cc);  head(c, cc) -= tau w;  tail(cc) -= tau v w,
// with v = tail(c) * scal.  Warp 0 updates column c+1 first and, in the same pass over
// its rows, accumulates the sum of squares of the next reflector's tail (FP64-accurate),
// then forms that reflector; warps 1.. update the remaining columns, four at a time;
// column c's tail is scaled in place one step later, when no warp reads it any more.
// One block-wide barrier per reflector.  On return the tails hold v, the heads beta,
// and s.tau_s / s.scal_s the taus and 1 / (alpha - beta).  FP32 storage takes its
// scalars in FP32 from the FP64-accurate sum of squares (reflector_f32).
// kR bounds the rows per lane (rows of the block <= 32 kR): the row loops are unrolled
// and each lane issues all its shared-memory loads of a pass at once.
template <typename S, int kPanel, int kR>
__device__ void panel_factor(Smem<S> &s, int kb, int rows, int c0, int mb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr bool kTT = kPanel != 0;  // TT and TS: the head is a row of R(piv)
  auto head = [&](int c, int cc) -> S & { return kTT ? s.P1[c + cc * s.ldp] : s.V[c + cc * s.ldv]; };
  auto tlo = [&](int c) { return kTT ? 0 : c + 1; };
  auto thi = [&](int c) { return kPanel == 1 ? min(c0 + c + 1, mb) : rows; };
  auto col = [&](int c) -> S * { return s.V + c * s.ldv; };
  constexpr bool kF32 = sizeof(S) == sizeof(float);
  // Sum of squares accumulated per lane: double-float for FP32 storage (FP64-accurate
  // with FP32 instructions), plain FP64 otherwise.
  struct Acc {
    DFloat d;
    double x;
  };
  auto acc_add = [&](Acc &a, S v) {
    if (kF32)
      a.d = df_sq_acc(a.d, static_cast<float>(v));
    else
      a.x = fma(static_cast<double>(v), static_cast<double>(v), a.x);
  };
  // Lane 0 turns column c's reduced sum of squares into its reflector: beta over the
  // head, tau and 1 / (alpha - beta) into shared memory.
  auto set_reflector = [&](int c, Acc a) {
    if (kF32) {
      a.d = df_warp_reduce(a.d);
    } else {
      a.x = warp_sum(a.x);
    }
    if (lane == 0) {
      if (kF32) {
        float beta, tau, scal;
        if (!reflector_f32(static_cast<float>(head(c, c)), a.d, &beta, &tau, &scal)) {
          double bd, td, sd;  // outside FP32's comfortable range: FP64 scalars
          reflector<1>(static_cast<double>(head(c, c)), static_cast<double>(a.d.hi) + a.d.lo, &bd, &td, &sd);
          beta = static_cast<float>(bd);
          tau = static_cast<float>(td);
          scal = static_cast<float>(sd);
        }
        head(c, c) = static_cast<S>(beta);
        s.tau_s[c] = static_cast<S>(tau);
        s.scal_s[c] = static_cast<S>(scal);
      } else {
        double beta, tau, scal;
        reflector<2>(static_cast<double>(head(c, c)), a.x, &beta, &tau, &scal);
        head(c, c) = static_cast<S>(beta);
        s.tau_s[c] = static_cast<S>(tau);
        s.scal_s[c] = static_cast<S>(scal);
      }
    }
  };
  auto fresh_reflector = [&](int c) {
    Acc a{{0.f, 0.f}, 0.0};
    const S *x = col(c);
    for (int r = tlo(c) + lane; r < thi(c); r += 32) acc_add(a, x[r]);
    set_reflector(c, a);
  };
  // Warp 0, look-ahead: reflector c applied to column c+1, whose updated values feed
  // the sum of squares of reflector c+1 in the same pass.
  auto update_and_reflect = [&](int c, S t, S sc) {
    const int cn = c + 1;
    const S *x = col(c);
    S *y = col(cn);
    const int lo = tlo(c), hi = thi(c), nlo = tlo(cn), nhi = thi(cn);
    const int rlo = min(lo, nlo), rhi = max(hi, nhi);
    // the lane's rows rlo + lane + 32u: v = x * scal (zero outside reflector c's tail)
    // and the column c+1 entries, loaded once for both passes
    S xv[kR], yv[kR];
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      const int r = rlo + lane + 32 * u;
      xv[u] = (r >= lo && r < hi) ? x[r] * sc : S(0);
      yv[u] = r < rhi ? y[r] : S(0);
    }
    const S hd = head(c, cn);
    S tw = 0;
    if (t != S(0)) {
      S part = 0;
#pragma unroll
      for (int u = 0; u < kR; ++u) part += xv[u] * yv[u];
      const S w = hd + warp_sum(part);
      tw = t * w;
      if (lane == 0) head(c, cn) = hd - tw;
    }
    Acc a{{0.f, 0.f}, 0.0};
#pragma unroll
    for (int u = 0; u < kR; ++u) {
      const int r = rlo + lane + 32 * u;
      S v = yv[u];
      if (r >= lo && r < hi && t != S(0)) {
        v -= xv[u] * tw;
        y[r] = v;
      }
      if (r >= nlo && r < nhi) acc_add(a, v);
    }
    __syncwarp();  // alpha of column c+1 (GEQRT: row c+1, updated above) for lane 0
    set_reflector(cn, a);
  };
  // Warps 1..: reflector c applied to up to kG columns cc0, cc0 + step, ... at once, so
  // that their dot products and butterfly reductions overlap.
  constexpr int kG = 4;
  auto update_group = [&](int c, int cc0, int step, int count, S t, S sc) {
    const S *x = col(c);
    const int lo = tlo(c), hi = thi(c);
    S part[kG];
#pragma unroll
    for (int u = 0; u < kG; ++u) part[u] = 0;
    S xv[kR];
#pragma unroll
    for (int w = 0; w < kR; ++w) {
      const int r = lo + lane + 32 * w;
      xv[w] = r < hi ? x[r] * sc : S(0);
    }
#pragma unroll
    for (int w = 0; w < kR; ++w) {
      const int r = lo + lane + 32 * w;
      if (r < hi) {
#pragma unroll
        for (int u = 0; u < kG; ++u)
          if (u < count) part[u] += xv[w] * col(cc0 + u * step)[r];
      }
    }
    S tw[kG];
    if constexpr (kF32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int u = 0; u < kG; ++u) part[u] += __shfl_xor_sync(0xffffffffu, part[u], o);
#pragma unroll
      for (int u = 0; u < kG; ++u) tw[u] = u < count ? t * (head(c, cc0 + u * step) + part[u]) : S(0);
      __syncwarp();
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < kG; ++u)
          if (u < count) head(c, cc0 + u * step) -= tw[u];
      }
    } else {
      // FP64: a reduce-scatter butterfly (six additions on the narrow FP64 pipe instead
      // of twenty) leaves lane l with the whole sum of slot (l >> 3) & 3; the lanes of a
      // slot form its t * w and lane 8u hands it to the warp.
      const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
      S k0 = up16 ? part[2] : part[0], k1 = up16 ? part[3] : part[1];
      const S o0 = up16 ? part[0] : part[2], o1 = up16 ? part[1] : part[3];
      k0 += __shfl_xor_sync(0xffffffffu, o0, 16);
      k1 += __shfl_xor_sync(0xffffffffu, o1, 16);
      S k = up8 ? k1 : k0;
      const S o2 = up8 ? k0 : k1;
      k += __shfl_xor_sync(0xffffffffu, o2, 8);
      k += __shfl_xor_sync(0xffffffffu, k, 4);
      k += __shfl_xor_sync(0xffffffffu, k, 2);
      k += __shfl_xor_sync(0xffffffffu, k, 1);
      const int slot = (lane >> 3) & 3;
      S mine = 0;
      if (slot < count) mine = t * (head(c, cc0 + slot * step) + k);
#pragma unroll
      for (int u = 0; u < kG; ++u) tw[u] = __shfl_sync(0xffffffffu, mine, 8 * u);
      __syncwarp();
      if ((lane & 7) == 0 && slot < count) head(c, cc0 + slot * step) -= mine;
    }
#pragma unroll
    for (int w = 0; w < kR; ++w) {
      const int r = lo + lane + 32 * w;
      if (r < hi) {
#pragma unroll
        for (int u = 0; u < kG; ++u)
          if (u < count) col(cc0 + u * step)[r] -= xv[w] * tw[u];
      }
    }
  };
  auto scale_tail = [&](int c) {
    const S sc = s.scal_s[c];
    S *x = col(c);
    for (int r = tlo(c) + lane; r < thi(c); r += 32) x[r] = x[r] * sc;
  };
  if (warp == 0) fresh_reflector(0);
  __syncthreads();
  for (int c = 0; c < kb; ++c) {
    const S t = s.tau_s[c];
    const S sc = s.scal_s[c];
    if (warp == 0) {
      if (c + 1 < kb) update_and_reflect(c, t, sc);
    } else if (t != S(0) && (kF32 || warp != kWarps / 2)) {
      // FP64: warp kWarps/2 shares warp 0's scheduler (and its FP64 unit), so it stays
      // out of the updates and the reflector chain runs alone there
      constexpr int kStep = kF32 ? kWarps - 1 : kWarps - 2;
      const int widx = (!kF32 && warp > kWarps / 2) ? warp - 1 : warp;
      for (int cc0 = c + 1 + widx; cc0 < kb; cc0 += kG * kStep) {
        const int count = min(kG, (kb - 1 - cc0) / kStep + 1);
        update_group(c, cc0, kStep, count, t, sc);
      }
    }
    if (warp == kWarps - 1 && c >= 1) scale_tail(c - 1);
    __syncthreads();
  }
  if (warp == kWarps - 1) scale_tail(kb - 1);
  __syncthreads();
}

// panel_factor with the tight rows-per-lane bound ceil(rows / 32) (rows <= 256).
template <typename S, int kPanel>
__device__ void panel_factor_dispatch(Smem<S> &s, int kb, int rows, int c0, int mb) {
  switch ((rows + 31) / 32) {
    case 1: panel_factor<S, kPanel, 1>(s, kb, rows, c0, mb); break;
    case 2: panel_factor<S, kPanel, 2>(s, kb, rows, c0, mb); break;
    case 3: panel_factor<S, kPanel, 3>(s, kb, rows, c0, mb); break;
    case 4: panel_factor<S, kPanel, 4>(s, kb, rows, c0, mb); break;
    case 5: panel_factor<S, kPanel, 5>(s, kb, rows, c0, mb); break;
    case 6: panel_factor<S, kPanel, 6>(s, kb, rows, c0, mb); break;
    case 7: panel_factor<S, kPanel, 7>(s, kb, rows, c0, mb); break;
    default: panel_factor<S, kPanel, 8>(s, kb, rows, c0, mb); break;
  }
}

// Gram matrix G(a, c) = v_a . v_c (a < c < kb) of a panel block's reflectors, held
// explicitly in s.V (GEQRT: unit diagonal and zeros above written in; TT: zeros below
// the triangle from the load).  Only the strict upper triangle is formed - the T
// recurrence reads nothing else - pair idx by thread idx mod kThreads, a fastest within a
// column c (a warp's V(r, a) loads hit distinct banks, its V(r, c) loads broadcast); each
// sum runs over the rows in order.
template <typename S>
__device__ void panel_gram(Smem<S> &s, int kb, int nrows) {
  const int npairs = kb * (kb - 1) / 2;
  // column c holds the pairs c (c - 1) / 2 .. c (c + 1) / 2 - 1
  auto pair_of = [](int idx, int &a, int &c) {
    c = static_cast<int>((1.0f + sqrtf(1.0f + 8.0f * static_cast<float>(idx))) * 0.5f);
    while (c * (c - 1) / 2 > idx) --c;
    while (c * (c + 1) / 2 <= idx) ++c;
    a = idx - c * (c - 1) / 2;
  };
  // a thread's two pairs (idx and idx + kThreads) advance together: two independent sums
  for (int idx = threadIdx.x; idx < npairs; idx += 2 * kThreads) {
    const bool two = idx + kThreads < npairs;
    int a0, c0, a1, c1;
    pair_of(idx, a0, c0);
    pair_of(two ? idx + kThreads : idx, a1, c1);
    const S *va0 = s.V + a0 * s.ldv, *vc0 = s.V + c0 * s.ldv;
    const S *va1 = s.V + a1 * s.ldv, *vc1 = s.V + c1 * s.ldv;
    S acc0 = 0, acc1 = 0;
#pragma unroll 4
    for (int r = 0; r < nrows; ++r) {
      acc0 += va0[r] * vc0[r];
      acc1 += va1[r] * vc1[r];
    }
    s.G[a0 + c0 * s.ldt] = acc0;
    if (two) s.G[a1 + c1 * s.ldt] = acc1;
  }
  __syncthreads();
}

// Builds T (kb x kb, upper) from the Gram matrix G and tau.  The compact-WY recurrence
// (Schreiber-Van Loan) T(c,c) = tau_c, T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c) makes
// T the inverse of the upper-triangular S with S(c,c) = 1/tau_c and S(a,c) = G(a,c)
// above the diagonal (the inverse of [S1 g; 0 1/tau] has last column
// [-tau S1^{-1} g; tau]).  Column j of T by back substitution without a division:
// x_j = tau_j, x_a = -tau_a sum_{a<k<=j} G(a,k) x_k, the sums accumulated right to left
// (k from j down), so that each step is one FMA per row.  Warp w forms columns j = w,
// w + kWarps, ...: lane a holds row a's running sum, lane k hands x_k to the warp at step
// k.  The longest chain is the last column's j steps, shared out by column over the warps
// (one warp doing all columns would issue kb^2 / 2 dependent steps).  tau_c = 0 (an
// identity reflector) gives a zero row and column, as the recurrence does.
template <typename S>
__device__ void build_t(Smem<S> &s, int kb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < kb; j += kWarps) {
    S acc = 0;
    for (int k = j; k >= 0; --k) {
      const S mine = k == j ? s.tau_s[j] : -s.tau_s[k] * acc;  // meaningful in lane k
      const S xk = __shfl_sync(0xffffffffu, mine, k);
      if (lane == k) s.T[k + j * s.ldt] = xk;
      if (lane < k) acc += s.G[lane + k * s.ldt] * xk;
    }
    if (lane > j && lane < kb) s.T[lane + j * s.ldt] = S(0);  // zero below the diagonal
  }
  __syncthreads();
}

// Writes the ib x width slice of a T factor for reflectors c0 .. c0+width-1: the kb x kb
// block from shared memory and zeros elsewhere.
template <typename S, typename Real>
__device__ void store_t(Real *Tg, int ib, int c0, int width, const Smem<S> &s, int kb) {
  for (int idx = threadIdx.x; idx < ib * width; idx += kThreads) {
    const int c = idx / ib, a = idx - c * ib;
    S v = 0;
    if (a < kb && c < kb) v = s.T[a + c * s.ldt];
    Tg[a + static_cast<int64_t>(c0 + c) * ib] = static_cast<Real>(v);
  }
}

template <typename S, typename Real>
__device__ void load_t(S *dst, int ldt, const Real *Tg, int ib, int c0, int kb) {
  load_block(dst, ldt, Tg + static_cast<int64_t>(c0) * ib, ib, kb, kb);
}

struct TileGeom {
  int64_t m, n;
  int nb;
  __device__ int rows(int i) const { return static_cast<int>(lmin(nb, m - int64_t(i) * nb)); }
  __device__ int cols(int j) const { return static_cast<int>(lmin(nb, n - int64_t(j) * nb)); }
};

template <typename Real>
__device__ __forceinline__ Real *tile_ptr(Real *A, int64_t lda, int nb, int i, int j) {
  return A + static_cast<int64_t>(j) * nb * lda + static_cast<int64_t>(i) * nb;
}

template <typename Real>
__device__ __forceinline__ Real *t_ptr(Real *T, int P, int ib, int nb, int i, int k, int which) {
  return T + (static_cast<int64_t>(k) * P + i) * 2 * ib * nb + static_cast<int64_t>(which) * ib * nb;
}

// ---------------------------------------------------------------------------------
// GEQRT(i,k): Householder QR of one tile, blocked by ib (R above, V below the diagonal).
template <typename Real, typename S>
__device__ void task_geqrt(const ExecParams &p, Smem<S> &s, int i, int k) {
  const TileGeom geo{p.m, p.n, p.nb};
  const int nb = p.nb, ib = p.ib;
  Real *A = static_cast<Real *>(p.A);
  Real *tile = tile_ptr(A, p.lda, nb, i, k);
  Real *Tg = t_ptr(static_cast<Real *>(p.T), p.P, ib, nb, i, k, 0);
  const int mb = geo.rows(i), ncol = geo.cols(k), K = min(mb, ncol);
  for (int c0 = 0; c0 < nb; c0 += ib) {
    const int width = min(ib, nb - c0);
    const int kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      store_t(Tg, ib, c0, width, s, 0);
      continue;
    }
    const int rows = mb - c0;
    Real *blk = tile + c0 + static_cast<int64_t>(c0) * p.lda;
    load_block(s.V, s.ldv, blk, p.lda, rows, kb);
    __syncthreads();
    panel_factor_dispatch<S, 0>(s, kb, rows, c0, mb);
    phase_mark(s.ph, 0);
    store_block(blk, p.lda, s.V, s.ldv, rows, kb);
    __syncthreads();
    // explicit reflector block: unit diagonal, zeros above
    for (int idx = threadIdx.x; idx < kb * kb; idx += kThreads) {
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) s.V[r + c * s.ldv] = (r == c) ? S(1) : S(0);
    }
    __syncthreads();
    panel_gram(s, kb, rows);
    build_t(s, kb);
    store_t(Tg, ib, c0, width, s, kb);
    __syncthreads();
    phase_mark(s.ph, 1);
    constexpr int kCW = chunk_cols(sizeof(S));
    for (int cs = c0 + kb; cs < ncol; cs += kCW) {
      const int w = min(kCW, ncol - cs);
      Real *cblk = tile + c0 + static_cast<int64_t>(cs) * p.lda;
      load_block(s.C, s.ldv, cblk, p.lda, rows, w);
      __syncthreads();
      apply_block(s.C, s.ldv, rows, static_cast<S *>(nullptr), 0, w, s.V, s.ldv, s.T, s.ldt, kb,
                  s.W, s.ldw, false, s.Wv, s.red);
      store_block(cblk, p.lda, s.C, s.ldv, rows, w);
      __syncthreads();
    }
    phase_mark(s.ph, 2);
  }
}

// ---------------------------------------------------------------------------------
// TTQRT(i,piv,k): QR of the upper triangle of tile (piv,k) stacked on the upper
// triangle of tile (i,k); reflector c acts on row c of (piv,k) and rows 0..c of (i,k),
// its tail is stored in column c of (i,k)'s upper triangle.
// TSQRT(i,piv,k) (kTS): the same with the whole square tile (i,k) below the triangle
// (Algorithm "elimSQ"): reflector c acts on row c of (piv,k) and every row of (i,k), its
// tail overwrites column c of (i,k).
template <typename Real, typename S, bool kTS>
__device__ void task_ttqrt(const ExecParams &p, Smem<S> &s, int i, int piv, int k) {
  const TileGeom geo{p.m, p.n, p.nb};
  const int nb = p.nb, ib = p.ib;
  Real *A = static_cast<Real *>(p.A);
  Real *t1 = tile_ptr(A, p.lda, nb, piv, k);
  Real *t2 = tile_ptr(A, p.lda, nb, i, k);
  Real *Tt = t_ptr(static_cast<Real *>(p.T), p.P, ib, nb, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = 0; c0 < nb; c0 += ib) {
    const int width = min(ib, nb - c0);
    const int kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      store_t(Tt, ib, c0, width, s, 0);
      continue;
    }
    const int rb = kTS ? mb : min(c0 + kb, mb);  // rows of tile i touched by this block
    // P2 = tile i, rows 0..rb-1 (TT: its upper part only), columns c0..c0+kb-1
    load_block_mode(s.V, s.ldv, t2 + static_cast<int64_t>(c0) * p.lda, p.lda, rb, kb,
                    [c0](int r, int c) { return (kTS || r <= c0 + c) ? static_cast<int>(kLoad) : static_cast<int>(kZero); });
    // P1 = upper part of the diagonal block of R(piv)
    load_block_mode(s.P1, s.ldp, t1 + c0 + static_cast<int64_t>(c0) * p.lda, p.lda, kb, kb,
                    [](int r, int c) { return r <= c ? static_cast<int>(kLoad) : static_cast<int>(kZero); });
    __syncthreads();
    panel_factor_dispatch<S, kTS ? 2 : 1>(s, kb, rb, c0, mb);
    phase_mark(s.ph, 0);
    panel_gram(s, kb, rb);
    build_t(s, kb);
    // write back (TT: the upper parts only, the lower parts hold GEQRT reflectors)
    for (int c = warp; c < kb; c += kWarps)
      for (int r = lane; r < rb; r += 32)
        if (kTS || r <= c0 + c) t2[r + static_cast<int64_t>(c0 + c) * p.lda] = static_cast<Real>(s.V[r + c * s.ldv]);
    for (int idx = threadIdx.x; idx < kb * kb; idx += kThreads) {
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) t1[(c0 + r) + static_cast<int64_t>(c0 + c) * p.lda] = static_cast<Real>(s.P1[r + c * s.ldp]);
    }
    store_t(Tt, ib, c0, width, s, kb);
    __syncthreads();
    phase_mark(s.ph, 1);
    // trailing columns of the same tile column: [R(piv) rows c0..c0+kb-1 ; tile i rows 0..rb-1]
    constexpr int kCW = chunk_cols(sizeof(S));
    for (int cs = c0 + kb; cs < K; cs += kCW) {
      const int w = min(kCW, K - cs);
      Real *c1 = t1 + c0 + static_cast<int64_t>(cs) * p.lda;
      Real *c2 = t2 + static_cast<int64_t>(cs) * p.lda;
      load_block(s.C1, s.ldv, c1, p.lda, kb, w);
      load_block(s.C, s.ldv, c2, p.lda, rb, w);
      __syncthreads();
      apply_block(s.C, s.ldv, rb, s.C1, s.ldv, w, s.V, s.ldv, s.T, s.ldt, kb, s.W, s.ldw, false, s.Wv, s.red);
      store_block(c1, p.lda, s.C1, s.ldv, kb, w);
      store_block(c2, p.lda, s.C, s.ldv, rb, w);
      __syncthreads();
    }
    phase_mark(s.ph, 2);
  }
}

// ---------------------------------------------------------------------------------
// UNMQR: C <- Q^T C (or Q C) with the reflectors of GEQRT(i,k).  C is mb x ncols at
// cptr (leading dimension ldc); it is tile (i,j) of A or tile row i of B.
template <typename Real, typename S, typename CT>
__device__ void task_unmqr(const ExecParams &p, Smem<S> &s, int i, int k, CT *cptr, int64_t ldc,
                           int ncols, bool transpose_q) {
  const TileGeom geo{p.m, p.n, p.nb};
  const int nb = p.nb, ib = p.ib;
  const Real *vt = tile_ptr(static_cast<Real *>(p.A), p.lda, nb, i, k);
  const Real *Tg = t_ptr(static_cast<Real *>(p.T), p.P, ib, nb, i, k, 0);
  const int mb = geo.rows(i), K = min(mb, geo.cols(k));
  const int nblk = (K + ib - 1) / ib;
  constexpr int kCW = chunk_cols(sizeof(S));
  for (int cs = 0; cs < ncols; cs += kCW) {
    const int w = min(kCW, ncols - cs);
    CT *cblk = cptr + static_cast<int64_t>(cs) * ldc;
    load_block(s.C, s.ldv, cblk, ldc, mb, w);
    for (int bb = 0; bb < nblk; ++bb) {
      const int b = transpose_q ? nblk - 1 - bb : bb;
      const int c0 = b * ib, kb = min(ib, K - c0), rows = mb - c0;
      const Real *vb = vt + c0 + static_cast<int64_t>(c0) * p.lda;
      load_block_mode(s.V, s.ldv, vb, p.lda, rows, kb, [](int r, int c) {
        return r > c ? static_cast<int>(kLoad) : (r == c ? static_cast<int>(kOne) : static_cast<int>(kZero));
      });
      load_t(s.T, s.ldt, Tg, ib, c0, kb);
      __syncthreads();
      apply_block(s.C + c0, s.ldv, rows, static_cast<S *>(nullptr), 0, w, s.V, s.ldv, s.T, s.ldt, kb,
                  s.W, s.ldw, transpose_q, s.Wv, s.red);
    }
    store_block(cblk, ldc, s.C, s.ldv, mb, w);
    __syncthreads();
  }
}

// TTMQR: [C1; C2] <- Q^T [C1; C2] (or Q [C1; C2]) with the reflectors of the TTQRT that
// zeroed tile (i,k) (ts: of the TSQRT, whose reflectors fill the whole tile).  C1 is the
// pivot row's tile (nb rows), C2 row i's tile (mb rows).
template <typename Real, typename S, typename CT>
__device__ void task_ttmqr(const ExecParams &p, Smem<S> &s, int i, int k, CT *c1ptr, CT *c2ptr,
                           int64_t ldc, int ncols, bool transpose_q, bool ts = false) {
  const TileGeom geo{p.m, p.n, p.nb};
  const int nb = p.nb, ib = p.ib;
  const Real *vt = tile_ptr(static_cast<Real *>(p.A), p.lda, nb, i, k);
  const Real *Tt = t_ptr(static_cast<Real *>(p.T), p.P, ib, nb, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  const int nblk = (K + ib - 1) / ib;
  constexpr int kCW = chunk_cols(sizeof(S));
  for (int cs = 0; cs < ncols; cs += kCW) {
    const int w = min(kCW, ncols - cs);
    CT *b1 = c1ptr + static_cast<int64_t>(cs) * ldc;
    CT *b2 = c2ptr + static_cast<int64_t>(cs) * ldc;
    load_block(s.C1, s.ldv, b1, ldc, K, w);
    load_block(s.C, s.ldv, b2, ldc, mb, w);
    for (int bb = 0; bb < nblk; ++bb) {
      const int b = transpose_q ? nblk - 1 - bb : bb;
      const int c0 = b * ib, kb = min(ib, K - c0), rb = ts ? mb : min(c0 + kb, mb);
      load_block_mode(s.V, s.ldv, vt + static_cast<int64_t>(c0) * p.lda, p.lda, rb, kb, [c0, ts](int r, int c) {
        return (ts || r <= c0 + c) ? static_cast<int>(kLoad) : static_cast<int>(kZero);
      });
      load_t(s.T, s.ldt, Tt, ib, c0, kb);
      __syncthreads();
      apply_block(s.C, s.ldv, rb, s.C1 + c0, s.ldv, w, s.V, s.ldv, s.T, s.ldt, kb, s.W, s.ldw,
                  transpose_q, s.Wv, s.red);
    }
    store_block(b1, ldc, s.C1, s.ldv, K, w);
    store_block(b2, ldc, s.C, s.ldv, mb, w);
    __syncthreads();
  }
}

}  // namespace
}  // namespace tqr

#include "mixed_tasks.cuh"

namespace tqr {
namespace {

// Bounded wait until *counter == 0.  Returns false if this CTA must stop.
__device__ bool wait_ready(const ExecParams &p, int t) {
  const int32_t *cnt = p.counters + t;
  if (ld_acquire_gpu(cnt) <= 0) return true;
  const uint64_t t0 = globaltimer_ns();
  const uint64_t limit = static_cast<uint64_t>(p.wait_limit_ns);
  for (uint64_t it = 0;; ++it) {
    if (ld_acquire_gpu(cnt) <= 0) return true;
    if (ld_relaxed_gpu(p.status) != 0) return false;
    if (globaltimer_ns() - t0 > limit || it > (limit >> 4) + 1000000ull) {
      atomicCAS(p.status, 0, kStatusTimeout | (min(t, (1 << 23) - 1) << 8));
      return false;
    }
    __nanosleep(64);
  }
}

// Target tile column of an update task, and the columns c0 .. c0+ncols-1 of that tile it
// updates: the whole tile, or column part task_part(j) of colw columns (ncols may be 0 at
// the ragged edge of the matrix).
__device__ __forceinline__ int update_columns(const ExecParams &q, int j, int &ncols, int &c0) {
  const int jc = task_col(j, q.colparts);
  const int tcols = static_cast<int>(lmin(q.nb, q.n - int64_t(jc) * q.nb));
  if (q.colparts > 1) {
    c0 = task_part(j, q.colparts) * q.colw;
    ncols = max(0, min(q.colw, tcols - c0));
  } else {
    c0 = 0;
    ncols = tcols;
  }
  return jc;
}

// L2 prefetch hints for the tiles task ta reads and writes (GEQRT: its tile; TTQRT: the
// two triangles' tiles; UNMQR / TTMQR: the target tile(s)), one tile column per thread in
// 128-byte lines.  Every hinted address is an element of the matrix.  A hint only moves
// data towards L2 (the point of coherence), so it may be issued before the task's
// predecessors have finished, with no effect on results.
template <typename Real>
__device__ void prefetch_task_tiles(const ExecParams &p, int ta) {
  const Task task = p.tasks[ta];
  const Real *A = static_cast<const Real *>(p.A);
  int64_t lda = p.lda, m = p.m, n = p.n;
  int nb = p.nb;
  if (p.mats) {
    const BatchMat *d = p.mats + p.mat_of[ta];
    A = static_cast<const Real *>(d->A);
    lda = d->lda;
    m = d->m;
    n = d->n;
    nb = d->nb;
  }
  int tcol = task.k, nt = 0;  // tile column; tile rows task.i and (second tile) task.piv
  switch (task.kind) {
    case kGeqrt: nt = 1; break;
    case kTtqrt: case kTsqrt: nt = 2; break;
    case kUnmqr: tcol = task_col(task.j, p.colparts); nt = 1; break;
    case kTtmqr: case kTsmqr: tcol = task_col(task.j, p.colparts); nt = 2; break;
    default: return;
  }
  for (int w = threadIdx.x; w < nt * nb; w += kThreads) {
    const bool second = w >= nb;
    const int c = second ? w - nb : w;
    const int64_t row0 = static_cast<int64_t>(second ? task.piv : task.i) * nb;
    const int64_t col = static_cast<int64_t>(tcol) * nb + c;
    if (col >= n || row0 >= m) continue;
    const int64_t bytes = lmin(nb, m - row0) * static_cast<int64_t>(sizeof(Real));
    const char *base = reinterpret_cast<const char *>(A + row0 + col * lda);
    for (int64_t off = 0; off < bytes; off += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + bytes - 1));
  }
}

template <typename Real, typename S, bool kMixed>
__global__ void __launch_bounds__(kThreads, 1) executor_kernel(ExecParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task, s_stop, s_ahead;
  __shared__ int s_fail;  // a bounded tensor-core wait of this block gave up
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ uint32_t s_tmem;
  __shared__ uint64_t s_ph[5];
  __shared__ ExecParams s_q;  // the current task's parameters in a batched launch
  Smem<S> s0 = carve<S>(smem_raw, p.nb, p.ib);
  s0.ph = p.trace ? s_ph : nullptr;
  MixedState ms{};
  ms.ph = s0.ph;
  ms.fail = &s_fail;
  ms.ld_pending = false;
  if (threadIdx.x == 0) s_fail = 0;
  if (kMixed) {
    if (threadIdx.x == 0) {
      umma::mbar_init(&s_bar[0], 1);
      umma::mbar_init(&s_bar[1], 1);
      umma::mbar_init_fence();
    }
    if (threadIdx.x < 32) umma::tmem_alloc(&s_tmem, 512);
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    ms.bar_ld = &s_bar[0];
    ms.bar_mma = &s_bar[1];
    ms.tmem = s_tmem;
    ms.ld_phase = 0;
    ms.mma_phase = 0;
  }
  // task functions read the parameters from shared memory; the claim barrier below
  // publishes this copy (and each batched task's geometry) to the block
  if (threadIdx.x == 0) s_q = p;
  // While task t runs, a SIMT executor's CTA pulls the tiles of task t + gridDim.x into
  // L2: with every CTA claiming one task per task duration, that task is claimed about one
  // round later.
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(p.next, 1);
      // a wait that gave up anywhere stops every CTA at its next claim
      int stop = t >= p.ntask || ld_relaxed_gpu(p.status) != 0;
      s_ahead = t + static_cast<int>(gridDim.x) < p.ntask ? t + static_cast<int>(gridDim.x) : -1;
      const uint64_t t_claim = p.trace ? globaltimer_ns() : 0;
      if (!stop && !wait_ready(p, t)) stop = 1;
      if (p.trace && !stop) {
        uint32_t sm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        const uint64_t now = globaltimer_ns();
        p.trace[8 * static_cast<int64_t>(t) + 0] = static_cast<int64_t>(t_claim);
        p.trace[8 * static_cast<int64_t>(t) + 1] = static_cast<int64_t>(now);
        p.trace[8 * static_cast<int64_t>(t) + 3] = sm;
        s_ph[0] = now;
        s_ph[1] = s_ph[2] = s_ph[3] = s_ph[4] = 0;
      }
      // a batched launch carries each task's matrix in a descriptor
      if (!stop && p.mats) {
        const BatchMat *d = p.mats + p.mat_of[t];
        s_q.A = d->A;
        s_q.lda = d->lda;
        s_q.m = d->m;
        s_q.n = d->n;
        s_q.nb = d->nb;
        s_q.ib = d->ib;
        s_q.P = d->P;
        s_q.Q = d->Q;
        s_q.T = d->T;
        s_q.ops = d->ops;
        s_q.vec4 = d->vec4;
      }
      s_task = t;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    const int t = s_task;
    // (the tensor-core executor runs faster without it: its tasks are short and the
    // prefetched tiles add DRAM traffic)
    if (!kMixed && s_ahead >= 0) prefetch_task_tiles<Real>(p, s_ahead);
    const Task task = p.tasks[t];
    const ExecParams &q = s_q;
    const int nb = q.nb;
    Smem<S> s = s0;
    if (p.mats) {
      s = carve<S>(smem_raw, nb, q.ib);
      s.ph = s0.ph;
    }
    switch (task.kind) {
      case kGeqrt:
        if (kMixed)  // tensor-core path (FP32, nb 128): the tile stays in shared memory
          task_geqrt_resident(q, smem_raw, s.ph, task.i, task.k);
        else
          task_geqrt<Real, S>(q, s, task.i, task.k);
        break;
      case kTtqrt:
        if (kMixed)
          task_pairqrt_resident<false>(q, smem_raw, s.ph, task.i, task.piv, task.k);
        else
          task_ttqrt<Real, S, false>(q, s, task.i, task.piv, task.k);
        break;
      case kTsqrt:
        if (kMixed)
          task_pairqrt_resident<true>(q, smem_raw, s.ph, task.i, task.piv, task.k);
        else
          task_ttqrt<Real, S, true>(q, s, task.i, task.piv, task.k);
        break;
      case kTtqrtS:  // tensor-core graphs only: block j of a split TTQRT / TSQRT
        if (kMixed) task_pairqrt_split<false>(q, smem_raw, s.ph, task.i, task.piv, task.k, task.j);
        break;
      case kTsqrtS:
        if (kMixed) task_pairqrt_split<true>(q, smem_raw, s.ph, task.i, task.piv, task.k, task.j);
        break;
      case kPrepG:  // tensor-core graphs only: the operand images of GEQRT(i,k)
        if (kMixed) prep_geqrt_ops(q, smem_raw, s.ph, task.i, task.k);
        phase_mark(s.ph, 3);
        break;
      case kPrepT:  // ... of the TTQRT (piv >= 0 and tile upper part) or TSQRT that zeroed (i,k)
        if (kMixed) prep_ttqrt_ops(q, smem_raw, s.ph, task.i, task.k, task.j != 0);
        phase_mark(s.ph, 3);
        break;
      case kUnmqr: {
        if (kMixed) {
          task_unmqr_umma(q, smem_raw, ms, task.i, task.k, task.j);
          break;
        }
        Real *A = static_cast<Real *>(q.A);
        int ncols, c0;
        const int jc = update_columns(q, task.j, ncols, c0);
        if (ncols > 0)
          task_unmqr<Real, S, Real>(q, s, task.i, task.k, tile_ptr(A, q.lda, nb, task.i, jc) + int64_t(c0) * q.lda,
                                    q.lda, ncols, false);
        break;
      }
      case kTtmqr:
      case kTsmqr: {
        if (kMixed) {
          // the TSQRT operand images are dense, the TTQRT ones upper triangular: one kernel
          task_ttmqr_umma(q, smem_raw, ms, task.i, task.piv, task.k, task.j);
          break;
        }
        Real *A = static_cast<Real *>(q.A);
        int ncols, c0;
        const int jc = update_columns(q, task.j, ncols, c0);
        if (ncols > 0)
          task_ttmqr<Real, S, Real>(q, s, task.i, task.k, tile_ptr(A, q.lda, nb, task.piv, jc) + int64_t(c0) * q.lda,
                                    tile_ptr(A, q.lda, nb, task.i, jc) + int64_t(c0) * q.lda, q.lda, ncols, false,
                                    task.kind == kTsmqr);
        break;
      }
      case kUnmqrB:
        task_unmqr<Real, S, double>(q, s, task.i, task.k, q.B + static_cast<int64_t>(task.i) * nb, q.ldb,
                                    static_cast<int>(q.nrhs), q.trans != 0);
        break;
      case kTtmqrB:
      case kTsmqrB:
        task_ttmqr<Real, S, double>(q, s, task.i, task.k, q.B + static_cast<int64_t>(task.piv) * nb,
                                    q.B + static_cast<int64_t>(task.i) * nb, q.ldb,
                                    static_cast<int>(q.nrhs), q.trans != 0, task.kind == kTsmqrB);
        break;
      default:
        break;
    }
    __threadfence();
    __syncthreads();
    // an abandoned task (a tensor-core wait gave up) releases no successor: stop here
    if (kMixed && s_fail) break;
    if (threadIdx.x == 0) {
      if (p.trace) {
        p.trace[8 * static_cast<int64_t>(t) + 2] = static_cast<int64_t>(globaltimer_ns());
        for (int q = 0; q < 4; ++q) p.trace[8 * static_cast<int64_t>(t) + 4 + q] = static_cast<int64_t>(s_ph[1 + q]);
      }
      __threadfence();
      for (int e = p.succ_ptr[t]; e < p.succ_ptr[t + 1]; ++e) atomicSub(p.counters + p.succ_idx[e], 1);
    }
  }
  if (kMixed) {
    if (s_fail && threadIdx.x == 0) {
      // drain the tensor-core work this thread issued (bounded) before tensor memory is
      // freed: one more commit tracks every MMA issued so far, and a pending operand copy
      // completes its own load phase
      constexpr uint64_t kDrainNs = 10ull * 1000 * 1000;
      umma::commit(ms.bar_mma);
      umma::mbar_wait(ms.bar_mma, ms.mma_phase, kDrainNs);
      if (ms.ld_pending) umma::mbar_wait(ms.bar_ld, ms.ld_phase, kDrainNs);
    }
    umma::fence_before();
    __syncthreads();
    if (threadIdx.x < 32) umma::tmem_dealloc(s_tmem, 512);
  }
}

template <typename Real, typename S, bool kMixed>
int launch_typed(const ExecParams &p, void *stream, size_t smem) {
  auto kern = executor_kernel<Real, S, kMixed>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  if (per_sm < 1) per_sm = 1;
  int grid = nsm * per_sm;
  if (grid > p.ntask) grid = p.ntask;
  if (grid < 1) grid = 1;
  kern<<<grid, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  count_launch();
  return static_cast<int>(cudaGetLastError());
}

template <typename Real, typename S, bool kMixed>
int slots_typed(size_t smem) {
  auto kern = executor_kernel<Real, S, kMixed>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return 0;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess) return 0;
  return nsm * (per_sm < 1 ? 1 : per_sm);
}

}  // namespace
}  // namespace tqr
