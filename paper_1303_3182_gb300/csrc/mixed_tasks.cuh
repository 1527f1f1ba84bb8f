// Mixed-precision tile tasks (included by executor.cuh; uses its SIMT helpers).
//
// The matrix is FP32.  GEQRT and TTQRT run the SIMT kernels with FP64 Householder norms
// and tau, then turn the tile's reflectors into tensor-core operand images:
//   T_full : the nb x nb compact-WY factor of all nb reflectors of the tile, assembled
//            from the stored ib-blocks by T(0:c0, blk) = -T(0:c0,0:c0) (V(:,0:c0)^T
//            V(:,blk)) T(blk,blk)  (Schreiber & Van Loan, 1989)
//   GEQRT  : V (B operand of W^T = C^T V) and Z = V T_full^T (A operand of C -= Z W)
//   TTQRT  : V2, Z2 = V2 T_full^T and T_full^T (A operand of C1 -= T^T W)
// each written as split bf16 (x = hi + lo) or fp16 images in the swizzled K-major layout
// the tensor cores read, so that an update task fetches them with bulk copies.
//
// UNMQR(i,k,j) on C (nb x nb):   W^T = C^T V  (tcgen05, TMEM)  ->  C -= Z W
// TTMQR(i,piv,k,j) on [C1; C2]:  W^T = C1^T + C2^T V2,  C2 -= Z2 W,  C1 -= T^T W
// (TSMQR: the same with a dense V2)
// Operands are split into 1, 2 or 3 16-bit parts (x = p0 + p1 + p2, each the rounding of
// what the previous parts leave) and multiplied as the sum of the part products whose
// orders add up to less than the part count: one bf16/fp16 product, split-bf16 x3
// (hi*hi + hi*lo + lo*hi, ~2^-16 relative) or split-bf16 x6 (three parts, ~2^-24),
// accumulated in FP32 in tensor memory into fresh accumulators, small part products first
// (issue_levels); the old tile values are added to the update in FP32 by the epilogue.
// The tensor-core tile is nb = 128.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "umma.cuh"

namespace tqr {
namespace {

constexpr int kMNB = 128;                       // tile size of the tensor-core path
constexpr int kMLD = kMNB + 1;                  // padded leading dimension of FP32 smem matrices
constexpr uint32_t kImg = kMNB * kMNB * 2;      // one 16-bit operand image, bytes
constexpr size_t kMixedSmem = 6 * kImg + 1024;  // operand buffers (<= 192 KB) + alignment

__host__ __device__ inline size_t mixed_smem_bytes() {
  const size_t prep = 3 * static_cast<size_t>(kMNB) * kMLD * sizeof(float) + 1024;
  return prep > kMixedSmem ? prep : kMixedSmem;
}

// Operand images of one factored tile: up to three operands (V, Z, T^T) x nparts parts.
__host__ __device__ inline size_t slot_bytes(int nparts) { return 3 * static_cast<size_t>(nparts) * kImg; }

struct MixedState {
  uint64_t *bar_ld, *bar_mma;
  uint32_t tmem;
  uint32_t ld_phase, mma_phase;
  uint64_t *ph;      // phase clock of the execution trace, or null
  volatile int *fail;  // shared: a bounded wait of this block gave up (the task is abandoned)
  bool ld_pending;   // thread 0: a bulk copy was issued whose completion was not yet seen
};

__device__ __forceinline__ unsigned char *ops_slot(const ExecParams &p, int i, int k, int which) {
  return static_cast<unsigned char *>(p.ops) +
         ((static_cast<size_t>(k) * p.P + i) * 2 + which) * slot_bytes(p.nparts);
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *raw) {
  const uint32_t a = umma::smem_u32(raw);
  return raw + ((1024u - (a & 1023u)) & 1023u);
}

// Splits 8 floats into NP 16-bit parts x = p0 + p1 + p2 (each the rounding to nearest of
// what the previous parts leave), packed 8 to a uint4.  Two values are converted per
// instruction (packed bf16x2 / f16x2 conversions; the rounding of each value is the same
// as a single conversion's).
template <int NP>
__device__ __forceinline__ void split8(const float *x, uint4 *parts, int fmt) {
  float rem[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) rem[j] = x[j];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (fmt == 1) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(rem[2 * j], rem[2 * j + 1]);
        if (q + 1 < NP) {
          const float2 back = __bfloat1622float2(h);
          rem[2 * j] -= back.x;
          rem[2 * j + 1] -= back.y;
        }
        w[j] = *reinterpret_cast<const uint32_t *>(&h);
      } else {
        const __half2 h = __floats2half2_rn(rem[2 * j], rem[2 * j + 1]);
        if (q + 1 < NP) {
          const float2 back = __half22float2(h);
          rem[2 * j] -= back.x;
          rem[2 * j + 1] -= back.y;
        }
        w[j] = *reinterpret_cast<const uint32_t *>(&h);
      }
    }
    parts[q] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Calls f(std::integral_constant<int, NP>) with the compile-time part count NP = nparts.
template <typename F>
__device__ __forceinline__ void with_parts(int nparts, F f) {
  if (nparts == 3)
    f(std::integral_constant<int, 3>{});
  else if (nparts == 2)
    f(std::integral_constant<int, 2>{});
  else
    f(std::integral_constant<int, 1>{});
}

// Writes the nparts images (consecutive, kImg apart) of an operand whose element
// (row, kk) is get(row, kk).
template <typename F>
__device__ void write_image(unsigned char *img, F get, int fmt, int nparts) {
  with_parts(nparts, [&](auto np) {
    constexpr int NP = decltype(np)::value;
    for (int ch = threadIdx.x; ch < kMNB * kMNB / 8; ch += kThreads) {
      const int kb = ch >> 10, rem = ch & 1023, row = rem >> 3, sub = rem & 7;
      const int k0 = kb * 64 + ((sub ^ (row & 7)) << 3);
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = get(row, k0 + j);
      uint4 parts[NP];
      split8<NP>(x, parts, fmt);
#pragma unroll
      for (int q = 0; q < NP; ++q) reinterpret_cast<uint4 *>(img + q * kImg)[ch] = parts[q];
    }
  });
}

// The column group of warp w in V T^T: groups g and 7 - g (long and short ranges of the
// triangular T) go to warps g and g + 4, which share a scheduler, so every scheduler gets
// the same work.
__device__ __forceinline__ int prep_group(int warp) {
  static_assert(kWarps == 8, "eight warps, eight 16-column groups");
  return warp < 4 ? warp : 11 - warp;
}

// G(a, c) = sum_r V(r, a) V(r, c) for a < c.  Thread (warp w, lane l) forms rows
// a = l + 32x (x < 4) of columns c = 16w .. 16w+15: the V(r, a) loads of a warp hit
// consecutive words, the V(r, c) loads are broadcasts.  range(c_lo, r0, r1) bounds r.
template <typename RowRange>
__device__ void gram_upper(float *G, const float *V, RowRange range) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cb = warp * 16;
  int r0, r1;
  range(cb, r0, r1);
  float acc[4][16];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 16; ++y) acc[x][y] = 0.f;
#pragma unroll 2
  for (int r = r0; r < r1; ++r) {
    float va[4], vc[16];
#pragma unroll
    for (int x = 0; x < 4; ++x) va[x] = V[r + (lane + 32 * x) * kMLD];
#pragma unroll
    for (int y = 0; y < 16; ++y) vc[y] = V[r + (cb + y) * kMLD];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 16; ++y) acc[x][y] += va[x] * vc[y];
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 16; ++y)
      if (lane + 32 * x < cb + y) G[(lane + 32 * x) + (cb + y) * kMLD] = acc[x][y];
}

// T_full from its ib x ib diagonal blocks (already in Ts) and the Gram matrix (Gs).
// Block column j: X = G(0:c0, blk) T(blk, blk);  T(0:c0, blk) = -T(0:c0, 0:c0) X.
// Thread (warp w, lane l) forms rows a = l + 32x of the block column's w-th group of
// columns (w < w_blk / 4 ... one column per warp when w_blk = 32), so loads of a warp are
// consecutive words or broadcasts.
__device__ void assemble_t(float *Ts, float *Gs, int ib) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c0 = ib; c0 < kMNB; c0 += ib) {
    const int w = min(ib, kMNB - c0);
    const int nx = (c0 + 31) / 32;  // row groups of 32 above the block
    // columns of the block column handled by this warp: cc = warp, warp + 8, ...
    float acc[4][4];
    // X = G(0:c0, blk) T(blk, blk): X(a, cc) = sum_{b <= cc} G(a, c0+b) T(c0+b, c0+cc)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int b = 0; b < w; ++b) {
      float g[4], t[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) g[x] = (x < nx) ? Gs[(lane + 32 * x) + (c0 + b) * kMLD] : 0.f;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int cc = warp + 8 * y;
        t[y] = (cc < w) ? Ts[(c0 + b) + (c0 + cc) * kMLD] : 0.f;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += g[x] * t[y];
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int a = lane + 32 * x, cc = warp + 8 * y;
        if (a < c0 && cc < w) Gs[a + (c0 + cc) * kMLD] = acc[x][y];
      }
    __syncthreads();
    // T(0:c0, blk) = -T(0:c0, 0:c0) X: T(a, c0+cc) = -sum_{a <= b < c0} T(a, b) X(b, cc)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int b = 0; b < c0; ++b) {
      float t[4], xv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) t[x] = (x < nx) ? Ts[(lane + 32 * x) + b * kMLD] : 0.f;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int cc = warp + 8 * y;
        xv[y] = (cc < w) ? Gs[b + (c0 + cc) * kMLD] : 0.f;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += t[x] * xv[y];
    }
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int a = lane + 32 * x, cc = warp + 8 * y;
        if (a < c0 && cc < w) Ts[a + (c0 + cc) * kMLD] = -acc[x][y];
      }
    __syncthreads();
  }
}

// Z(r, a) = sum_b V(r, b) T(a, b) (= V T^T).  Thread (warp w, lane l) forms rows
// r = l + 32x of the columns a of its warp's 16-column group; bounds(a_lo, b0, b1)
// limits b.
template <typename Bounds>
__device__ void v_times_tt(float *Z, const float *V, const float *Ts, Bounds bounds) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ab = prep_group(warp) * 16;
  int b0, b1;
  bounds(ab, b0, b1);
  float acc[4][16];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 16; ++y) acc[x][y] = 0.f;
#pragma unroll 2
  for (int b = b0; b < b1; ++b) {
    float vr[4], tt[16];
#pragma unroll
    for (int x = 0; x < 4; ++x) vr[x] = V[(lane + 32 * x) + b * kMLD];
#pragma unroll
    for (int y = 0; y < 16; ++y) tt[y] = Ts[(ab + y) + b * kMLD];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 16; ++y) acc[x][y] += vr[x] * tt[y];
  }
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 16; ++y) Z[(lane + 32 * x) + (ab + y) * kMLD] = acc[x][y];
}

// Fills the 128 x 128 shared-memory matrix dst[r + c * kMLD] with *src(r, c) (a global
// address, loaded through L2) or zero where src(r, c) is null.  Each thread issues 16
// loads before its first store, so that their latencies overlap.
template <typename Src>
__device__ void gather_tile(float *dst, Src src) {
  constexpr int kB = 16;
  static_assert(kMNB * kMNB % (kThreads * kB) == 0, "whole passes");
  for (int e0 = threadIdx.x; e0 < kMNB * kMNB; e0 += kThreads * kB) {
    float v[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * kThreads, r = e % kMNB, c = e / kMNB;
      const float *ptr = src(r, c);
      v[u] = ptr ? __ldcg(ptr) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = e0 + u * kThreads, r = e % kMNB, c = e / kMNB;
      dst[r + c * kMLD] = v[u];
    }
  }
}

// Loads the ib-blocked T of a factored tile into the block diagonal of Ts (zeros elsewhere).
__device__ void load_t_blocks(float *Ts, const float *Tg, int ib) {
  gather_tile(Ts, [&](int a, int c) -> const float * {
    const int cb = (c / ib) * ib;
    return (a >= cb && a <= c) ? Tg + (a - cb) + static_cast<int64_t>(c) * ib : nullptr;
  });
}

// Operand images of GEQRT(i,k): V and Z = V T_full^T.
__device__ void prep_geqrt_ops(const ExecParams &p, unsigned char *raw, uint64_t *ph, int i, int k) {
  const TileGeom geo{p.m, p.n, kMNB};
  float *Vs = reinterpret_cast<float *>(raw);
  float *Ts = Vs + kMNB * kMLD;
  float *Gs = Ts + kMNB * kMLD;
  const float *tile = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, k);
  const float *Tg = t_ptr(static_cast<float *>(p.T), p.P, p.ib, kMNB, i, k, 0);
  const int mb = geo.rows(i), K = min(mb, geo.cols(k));
  load_block_mode(Vs, kMLD, tile, p.lda, kMNB, kMNB, [K, mb](int r, int c) {
    if (c >= K || r >= mb) return static_cast<int>(kZero);
    return r > c ? static_cast<int>(kLoad) : (r == c ? static_cast<int>(kOne) : static_cast<int>(kZero));
  });
  load_t_blocks(Ts, Tg, p.ib);
  __syncthreads();
  phase_mark(ph, 0);  // trace phases: 0 loads, 1 Gram and T_full, 2 Z, 3 the images
  // G(a, c) = v_a . v_c over rows r >= c (v_c is zero above its diagonal)
  gram_upper(Gs, Vs, [](int c_lo, int &r0, int &r1) { r0 = c_lo; r1 = kMNB; });
  __syncthreads();
  assemble_t(Ts, Gs, p.ib);
  phase_mark(ph, 1);
  // Z = V T^T: Z(r, a) = sum_{a <= b <= r} V(r, b) T(a, b)
  v_times_tt(Gs, Vs, Ts, [](int a_lo, int &b0, int &b1) { b0 = a_lo; b1 = kMNB; });
  __syncthreads();
  phase_mark(ph, 2);
  unsigned char *slot = ops_slot(p, i, k, 0);
  const int np = p.nparts;
  write_image(slot, [&](int row, int kk) { return Vs[kk + row * kMLD]; }, p.fmt, np);
  write_image(slot + np * kImg, [&](int row, int kk) { return Gs[row + kk * kMLD]; }, p.fmt, np);
  __syncthreads();
}

// Operand images of TTQRT(i,piv,k): V2 (upper part of tile i), Z2 = V2 T_full^T, T_full^T.
// ts: of TSQRT(i,piv,k), whose V2 is the whole tile i (Algorithm "elimSQ").
__device__ void prep_ttqrt_ops(const ExecParams &p, unsigned char *raw, uint64_t *ph, int i, int k, bool ts) {
  const TileGeom geo{p.m, p.n, kMNB};
  float *Vs = reinterpret_cast<float *>(raw);
  float *Ts = Vs + kMNB * kMLD;
  float *Gs = Ts + kMNB * kMLD;
  const float *tile = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, k);
  const float *Tt = t_ptr(static_cast<float *>(p.T), p.P, p.ib, kMNB, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  load_block_mode(Vs, kMLD, tile, p.lda, kMNB, kMNB, [K, mb, ts](int r, int c) {
    return (c < K && r < mb && (ts || r <= c)) ? static_cast<int>(kLoad) : static_cast<int>(kZero);
  });
  load_t_blocks(Ts, Tt, p.ib);
  __syncthreads();
  phase_mark(ph, 0);
  // G(a, c) = v_a . v_c over the rows the tails occupy (TT: r <= a, within the upper
  // triangle; TS: every row)
  if (ts)
    gram_upper(Gs, Vs, [](int, int &r0, int &r1) { r0 = 0; r1 = kMNB; });
  else
    gram_upper(Gs, Vs, [](int c_lo, int &r0, int &r1) { r0 = 0; r1 = min(c_lo + 16, kMNB); });
  __syncthreads();
  assemble_t(Ts, Gs, p.ib);
  phase_mark(ph, 1);
  // Z2(r, a) = sum_{b >= a} V2(r, b) T(a, b)
  v_times_tt(Gs, Vs, Ts, [](int a_lo, int &b0, int &b1) { b0 = a_lo; b1 = kMNB; });
  __syncthreads();
  phase_mark(ph, 2);
  unsigned char *slot = ops_slot(p, i, k, 1);
  const int np = p.nparts;
  write_image(slot, [&](int row, int kk) { return Vs[kk + row * kMLD]; }, p.fmt, np);
  write_image(slot + np * kImg, [&](int row, int kk) { return Gs[row + kk * kMLD]; }, p.fmt, np);
  write_image(slot + 2 * np * kImg, [&](int row, int kk) { return Ts[kk + row * kMLD]; }, p.fmt, np);
  __syncthreads();
}

// ---------------------------------------------------------------------------------
// Panel tasks of the tensor-core path with the tile resident in shared memory: the tile
// (and, for TTQRT / TSQRT, the pivot tile's upper triangle) is read once, every ib-block
// is factored and applied to the later columns in shared memory, and the result is
// written back once - the in-tile trailing updates make no round trips to global memory.
// The arithmetic is that of task_geqrt / task_ttqrt (the same SIMT panel, Gram, T and
// block-reflector code), so the results are bit for bit those of the chunked tasks.
struct ResBufs {
  float *Ct, *Rp, *save;  // resident tile, resident pivot triangle, R block of a GEQRT
  Smem<float> s;
};

constexpr size_t kResidentFloats = 2 * static_cast<size_t>(kMLD) * kMNB + 4 * 33 * 32 + 2 * 32 + 4 + 32 * kWvLd +
                                   3 * 32 * 33;
static_assert(kResidentFloats * sizeof(float) <= 3 * static_cast<size_t>(kMNB) * kMLD * sizeof(float) + 1024,
              "the resident panel fits the tensor-core executor's shared memory");

__device__ ResBufs res_carve(unsigned char *raw, int ib, uint64_t *ph) {
  ResBufs r;
  float *p = reinterpret_cast<float *>(raw);
  r.Ct = p;
  p += kMLD * kMNB;
  r.Rp = p;
  p += kMLD * kMNB;
  Smem<float> &s = r.s;
  s.ldv = kMLD;
  s.ldw = ib + 1;
  s.ldt = ib + 1;
  s.ldp = kMLD;
  s.W = p;
  p += 33 * 32;
  s.T = p;
  p += 33 * 32;
  s.G = p;
  p += 33 * 32;
  s.tau_s = p;
  p += 32;
  s.scal_s = p;
  p += 32;
  r.save = p;
  p += 33 * 32;
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~static_cast<uintptr_t>(15);
  s.Wv = reinterpret_cast<float *>(a);
  s.red = s.Wv + 32 * kWvLd;
  s.V = r.Ct;
  s.C = s.C1 = nullptr;
  s.P1 = r.Rp;
  s.ph = ph;
  return r;
}

// GEQRT(i,k) with the tile resident.
__device__ void task_geqrt_resident(const ExecParams &p, unsigned char *raw, uint64_t *ph, int i, int k) {
  const TileGeom geo{p.m, p.n, kMNB};
  const int ib = p.ib;
  ResBufs rb = res_carve(raw, ib, ph);
  Smem<float> &s = rb.s;
  float *tile = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, k);
  float *Tg = t_ptr(static_cast<float *>(p.T), p.P, ib, kMNB, i, k, 0);
  const int mb = geo.rows(i), ncol = geo.cols(k), K = min(mb, ncol);
  load_block(rb.Ct, kMLD, tile, p.lda, mb, ncol);
  __syncthreads();
  phase_mark(s.ph, 3);  // trace phases: 3 the loads, then per ib-block 0 panel, 1 T, 2 trailing update
  for (int c0 = 0; c0 < kMNB; c0 += ib) {
    const int width = min(ib, kMNB - c0), kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      store_t(Tg, ib, c0, width, s, 0);
      continue;
    }
    const int rows = mb - c0;
    s.V = rb.Ct + c0 + c0 * kMLD;
    panel_factor_dispatch<float, 0>(s, kb, rows, c0, mb);
    phase_mark(s.ph, 0);
    // the explicit reflector block (unit diagonal, zeros above) for the Gram matrix and the
    // block reflector; the R block it covers is kept aside and put back afterwards
    for (int idx = threadIdx.x; idx < kb * kb; idx += kThreads) {
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) {
        rb.save[r + c * 33] = s.V[r + c * kMLD];
        s.V[r + c * kMLD] = r == c ? 1.f : 0.f;
      }
    }
    __syncthreads();
    panel_gram(s, kb, rows);
    build_t(s, kb);
    store_t(Tg, ib, c0, width, s, kb);
    __syncthreads();
    phase_mark(s.ph, 1);
    for (int cs = c0 + kb; cs < ncol; cs += 32) {
      const int w = min(32, ncol - cs);
      apply_block(rb.Ct + c0 + cs * kMLD, kMLD, rows, static_cast<float *>(nullptr), 0, w, s.V, kMLD, s.T, s.ldt, kb,
                  s.W, s.ldw, false, s.Wv, s.red);
    }
    for (int idx = threadIdx.x; idx < kb * kb; idx += kThreads) {
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) s.V[r + c * kMLD] = rb.save[r + c * 33];
    }
    __syncthreads();
    phase_mark(s.ph, 2);
  }
  store_block(tile, p.lda, rb.Ct, kMLD, mb, ncol);
  __syncthreads();
}

// TTQRT(i,piv,k) (ts false) / TSQRT(i,piv,k) (ts true) with both tiles resident: the
// upper triangle of (piv,k) and the upper triangle (TT) or the whole (TS) of (i,k).
template <bool kTS>
__device__ void task_pairqrt_resident(const ExecParams &p, unsigned char *raw, uint64_t *ph, int i, int piv, int k) {
  const TileGeom geo{p.m, p.n, kMNB};
  const int ib = p.ib;
  ResBufs rb = res_carve(raw, ib, ph);
  Smem<float> &s = rb.s;
  float *A = static_cast<float *>(p.A);
  float *t1 = tile_ptr(A, p.lda, kMNB, piv, k), *t2 = tile_ptr(A, p.lda, kMNB, i, k);
  float *Tt = t_ptr(static_cast<float *>(p.T), p.P, ib, kMNB, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  auto upper = [](int r, int c) { return r <= c ? static_cast<int>(kLoad) : static_cast<int>(kZero); };
  load_block_mode(rb.Rp, kMLD, t1, p.lda, K, K, upper);
  load_block_mode(rb.Ct, kMLD, t2, p.lda, mb, K,
                  [](int r, int c) { return (kTS || r <= c) ? static_cast<int>(kLoad) : static_cast<int>(kZero); });
  __syncthreads();
  phase_mark(s.ph, 3);
  for (int c0 = 0; c0 < kMNB; c0 += ib) {
    const int width = min(ib, kMNB - c0), kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      store_t(Tt, ib, c0, width, s, 0);
      continue;
    }
    const int rbk = kTS ? mb : min(c0 + kb, mb);
    s.V = rb.Ct + c0 * kMLD;
    s.P1 = rb.Rp + c0 + c0 * kMLD;
    panel_factor_dispatch<float, kTS ? 2 : 1>(s, kb, rbk, c0, mb);
    phase_mark(s.ph, 0);
    panel_gram(s, kb, rbk);
    build_t(s, kb);
    store_t(Tt, ib, c0, width, s, kb);
    __syncthreads();
    phase_mark(s.ph, 1);
    for (int cs = c0 + kb; cs < K; cs += 32) {
      const int w = min(32, K - cs);
      apply_block(rb.Ct + cs * kMLD, kMLD, rbk, rb.Rp + c0 + cs * kMLD, kMLD, w, s.V, kMLD, s.T, s.ldt, kb, s.W,
                  s.ldw, false, s.Wv, s.red);
    }
    phase_mark(s.ph, 2);
  }
  // write back what the kernel owns: the triangles (TT) or the triangle and the whole tile (TS)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < K; c += kWarps) {
    for (int r = lane; r < mb; r += 32)
      if (kTS || r <= c) t2[r + static_cast<int64_t>(c) * p.lda] = rb.Ct[r + c * kMLD];
    for (int r = lane; r <= c; r += 32) t1[r + static_cast<int64_t>(c) * p.lda] = rb.Rp[r + c * kMLD];
  }
  __syncthreads();
}

// Block b of a split TTQRT (ts false) / TSQRT (ts true): the ib-blocks of columns
// 32b .. 32b+31 of the elimination, with rows 32b .. 32b+31 of the pivot's R and the zeroed
// tile's columns 32b .. K-1 resident (TT: its upper part, rows < 32b + 32; TS: all rows).
// Blocks run in order for one elimination (block b+1 needs the columns block b updated),
// and block b of the next elimination on the same pivot needs only R's row block b; the
// arithmetic per ib-block is task_pairqrt_resident's.
template <bool kTS>
__device__ void task_pairqrt_split(const ExecParams &p, unsigned char *raw, uint64_t *ph, int i, int piv, int k,
                                   int b) {
  const TileGeom geo{p.m, p.n, kMNB};
  const int ib = p.ib;
  const int c0 = b * kPanelSplitCols;
  ResBufs rb = res_carve(raw, ib, ph);
  Smem<float> &s = rb.s;
  float *A = static_cast<float *>(p.A);
  float *t1 = tile_ptr(A, p.lda, kMNB, piv, k), *t2 = tile_ptr(A, p.lda, kMNB, i, k);
  float *Tt = t_ptr(static_cast<float *>(p.T), p.P, ib, kMNB, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  const int c1 = min(c0 + kPanelSplitCols, kMNB);
  if (c0 >= K) {  // a ragged last tile column: these reflectors do not exist
    for (int cb = c0; cb < c1; cb += ib) store_t(Tt, ib, cb, min(ib, kMNB - cb), s, 0);
    __syncthreads();
    return;
  }
  const int r1 = min(c1, K);                   // R rows of this block: c0 .. r1-1
  const int rows_i = kTS ? mb : min(c1, mb);   // rows of the zeroed tile the block touches
  // resident (local column c - c0; R rows local r - c0)
  load_block_mode(rb.Rp, kMLD, t1 + c0 + static_cast<int64_t>(c0) * p.lda, p.lda, r1 - c0, K - c0,
                  [](int r, int c) { return r <= c ? static_cast<int>(kLoad) : static_cast<int>(kZero); });
  load_block_mode(rb.Ct, kMLD, t2 + static_cast<int64_t>(c0) * p.lda, p.lda, rows_i, K - c0, [c0](int r, int c) {
    return (kTS || r <= c0 + c) ? static_cast<int>(kLoad) : static_cast<int>(kZero);
  });
  __syncthreads();
  phase_mark(s.ph, 3);
  for (int cb = c0; cb < c1; cb += ib) {
    const int width = min(ib, kMNB - cb), kb = max(0, min(ib, K - cb));
    if (kb == 0) {
      store_t(Tt, ib, cb, width, s, 0);
      continue;
    }
    const int rbk = kTS ? mb : min(cb + kb, mb);
    s.V = rb.Ct + (cb - c0) * kMLD;
    s.P1 = rb.Rp + (cb - c0) + (cb - c0) * kMLD;
    panel_factor_dispatch<float, kTS ? 2 : 1>(s, kb, rbk, cb, mb);
    phase_mark(s.ph, 0);
    panel_gram(s, kb, rbk);
    build_t(s, kb);
    store_t(Tt, ib, cb, width, s, kb);
    __syncthreads();
    phase_mark(s.ph, 1);
    for (int cs = cb + kb; cs < K; cs += 32) {
      const int w = min(32, K - cs);
      apply_block(rb.Ct + (cs - c0) * kMLD, kMLD, rbk, rb.Rp + (cb - c0) + (cs - c0) * kMLD, kMLD, w, s.V, kMLD,
                  s.T, s.ldt, kb, s.W, s.ldw, false, s.Wv, s.red);
    }
    phase_mark(s.ph, 2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = c0 + warp; c < K; c += kWarps) {
    for (int r = lane; r < rows_i; r += 32)
      if (kTS || r <= c) t2[r + static_cast<int64_t>(c) * p.lda] = rb.Ct[r + (c - c0) * kMLD];
    for (int r = c0 + lane; r < r1 && r <= c; r += 32)
      t1[r + static_cast<int64_t>(c) * p.lda] = rb.Rp[(r - c0) + (c - c0) * kMLD];
  }
  __syncthreads();
}

// D(128 x 128, FP32 in TMEM) (+)= A (128 x 128) op(B)^T for split operands: the part
// products A_qa B_qb of one "level" s = qa + qb (s < nparts: hi*hi is level 0; hi*lo and
// lo*hi level 1; hi*lo2, mid*mid, lo2*hi level 2) for the k-steps ks0 .. ks1-1 (16 columns
// of K each), levels lvl_hi down to lvl_lo, level-major.  neg_b negates B.  acc: whether
// the first MMA accumulates onto D; set to 1 afterwards.
//
// Order matters for accuracy.  Each MMA adds its products to the FP32 sum held in tensor
// memory; a small part product added to a large sum keeps only the bits that sum can
// hold.  Measured on GB300 with every part product added onto the TMEM copy of the tile,
// the split-bf16 x6 factorization's backward error grew about linearly with n (1.2e-5 at
// 4096 x 1024, against 1.0e-6 for FP32 SIMT updates), the sign of a bias.  The updates
// therefore accumulate into a fresh D (the tile itself is added once, in FP32, by the
// epilogue) and issue every small level over the whole K range before the level-0
// products, so only the 8 level-0 MMAs of a product meet a full-size sum: the same
// factorization's backward error is then 1.8e-6 and grows like the FP32 updates'.
__device__ __forceinline__ void issue_levels(uint32_t d_tmem, const unsigned char *bufA, const unsigned char *bufB,
                                             int nparts, int fmt, int neg_b, uint32_t &acc, int ks0, int ks1,
                                             int lvl_lo, int lvl_hi) {
  const uint32_t idesc = umma::idesc_f16(128, 128, fmt, neg_b);
  const uint32_t a0 = umma::smem_u32(bufA), b0 = umma::smem_u32(bufB);
#pragma unroll 1
  for (int lv = lvl_hi; lv >= lvl_lo; --lv) {
#pragma unroll 1
    for (int ks = ks0; ks < ks1; ++ks) {
      const uint32_t off = (ks >> 2) * (kMNB * 128) + (ks & 3) * 32;
      for (int qa = lv; qa >= 0; --qa) {
        const int qb = lv - qa;
        if (qa >= nparts || qb >= nparts) continue;
        umma::mma_f16(d_tmem, umma::smem_desc(a0 + qa * kImg + off), umma::smem_desc(b0 + qb * kImg + off), idesc,
                      acc);
        acc = 1u;
      }
    }
  }
}

// One K half h (k-steps 4h .. 4h+3) of a fresh product D = A op(B)^T, issued as its
// operand half becomes ready: half 0 issues the small levels of its k-steps; half 1 the
// small levels of its own, then the level-0 products of all eight k-steps.  With one
// part (bf16 / fp16) each half issues its own k-steps.
__device__ __forceinline__ void issue_product_half(uint32_t d_tmem, const unsigned char *bufA,
                                                   const unsigned char *bufB, int nparts, int fmt, int neg_b,
                                                   uint32_t &acc, int h) {
  if (nparts == 1) {
    issue_levels(d_tmem, bufA, bufB, nparts, fmt, neg_b, acc, 4 * h, 4 * h + 4, 0, 0);
    return;
  }
  issue_levels(d_tmem, bufA, bufB, nparts, fmt, neg_b, acc, 4 * h, 4 * h + 4, 1, nparts - 1);
  if (h == 1) issue_levels(d_tmem, bufA, bufB, nparts, fmt, neg_b, acc, 0, 8, 0, 0);
}

// A whole fresh product D = A op(B)^T (both operands resident), in the same order.
__device__ __forceinline__ void issue_product(uint32_t d_tmem, const unsigned char *bufA, const unsigned char *bufB,
                                              int nparts, int fmt, int neg_b) {
  uint32_t acc = 0u;
  issue_product_half(d_tmem, bufA, bufB, nparts, fmt, neg_b, acc, 0);
  issue_product_half(d_tmem, bufA, bufB, nparts, fmt, neg_b, acc, 1);
}

// L2 prefetch hints for the ncols 512-byte columns of a 128-row FP32 tile.
__device__ __forceinline__ void prefetch_tile_l2(const float *C, int64_t ldc, int ncols) {
  for (int c = threadIdx.x; c < ncols; c += kThreads) {
    const char *col = reinterpret_cast<const char *>(C + static_cast<int64_t>(c) * ldc);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(col));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(col + 256));
  }
}

// Split image of C^T (row c, k = r) in shared memory, K half h only (rows r of C in
// 64h .. 64h+63, one 1024-byte-swizzled K atom), one 16-byte chunk (8 rows of one column)
// per thread step; the rows come as two float4 loads when the tile is 16-byte aligned
// (vec4), else one by one.  Each thread issues the loads of its four chunks before
// converting any, so that enough bytes are in flight to hide the memory latency.
__device__ void c_transposed_image(unsigned char *img, const float *C, int64_t ldc, int mb, int ncols, int fmt,
                                   int nparts, bool vec4, int h) {
  constexpr int kU = 4;  // chunks per thread and half
  static_assert(kMNB * kMNB / 16 == kU * kThreads, "one group of chunks per half");
  float x[kU][8];
#pragma unroll
  for (int u = 0; u < kU; ++u) {
    const int ch = threadIdx.x + (4 * h + u) * kThreads;
    const int kb = ch >> 10, rem = ch & 1023, row = rem >> 3, sub = rem & 7;
    const int k0 = kb * 64 + ((sub ^ (row & 7)) << 3);
    const float *colp = C + static_cast<int64_t>(row) * ldc + k0;
    if (row < ncols && vec4 && k0 + 8 <= mb) {
      const float4 a = __ldcg(reinterpret_cast<const float4 *>(colp));
      const float4 b = __ldcg(reinterpret_cast<const float4 *>(colp + 4));
      x[u][0] = a.x; x[u][1] = a.y; x[u][2] = a.z; x[u][3] = a.w;
      x[u][4] = b.x; x[u][5] = b.y; x[u][6] = b.z; x[u][7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[u][j] = (row < ncols && k0 + j < mb) ? __ldcg(colp + j) : 0.f;
    }
  }
  with_parts(nparts, [&](auto np) {
    constexpr int NP = decltype(np)::value;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int ch = threadIdx.x + (4 * h + u) * kThreads;
      uint4 parts[NP];
      split8<NP>(x[u], parts, fmt);
#pragma unroll
      for (int q = 0; q < NP; ++q) reinterpret_cast<uint4 *>(img + q * kImg)[ch] = parts[q];
    }
  });
}

// W^T (TMEM lane c, column a) -> split image of W as a B operand (row c, k = a), K half h
// only (a in 64h .. 64h+63: warps 0-3 take the first 32 columns, warps 4-7 the next 32).
// C1 non-null (TTMQR / TSMQR): W^T(c, a) += C1(a, c) in FP32 first - the identity part of
// the pair's reflectors - with C1(a, c) read from global memory (zero for c >= ncols).
__device__ void w_image_from_tmem(unsigned char *img, uint32_t tmem_w, int fmt, int nparts, int h,
                                  const float *C1 = nullptr, int64_t ldc1 = 0, int ncols = 0, bool vec4 = false) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (warp & 3) * 32 + lane;
  const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
  const int a0 = 64 * h + (warp >> 2) * 32;
  float v[32];
  umma::tmem_ld32(tmem_w + lane_base + a0, v);
  if (C1) {
    const float *col = C1 + static_cast<int64_t>(c) * ldc1 + a0;
    if (c < ncols && vec4) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 q4 = __ldcg(reinterpret_cast<const float4 *>(col) + u);
        v[4 * u] += q4.x;
        v[4 * u + 1] += q4.y;
        v[4 * u + 2] += q4.z;
        v[4 * u + 3] += q4.w;
      }
    } else if (c < ncols) {
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] += __ldcg(col + u);
    }
  }
  with_parts(nparts, [&](auto np) {
    constexpr int NP = decltype(np)::value;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint4 parts[NP];
      split8<NP>(v + 8 * u, parts, fmt);
      const uint32_t off = umma::sw128_offset(c, a0 + 8 * u, kMNB);
#pragma unroll
      for (int q = 0; q < NP; ++q) *reinterpret_cast<uint4 *>(img + q * kImg + off) = parts[q];
    }
  });
}

// C(r, c) = base(r, c) + P(r, c), the update P at tmem_p (lane r, column c) added in FP32 to
// the tile's old values: base at tmem_base (lane r) when tmem_base != 0, else read from C.
__device__ void tile_plus_tmem(float *C, int64_t ldc, int nrows, int ncols, uint32_t tmem_p, uint32_t tmem_base) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = (warp & 3) * 32 + lane;
  const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
  for (int g = 0; g < 2; ++g) {
    const int c0 = (warp >> 2) * 64 + g * 32;
    float v[32], b[32];
    umma::tmem_ld32(tmem_p + lane_base + c0, v);
    if (tmem_base) {
      umma::tmem_ld32(tmem_base + lane_base + c0, b);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        b[j] = (r < nrows && c0 + j < ncols) ? __ldcg(C + r + static_cast<int64_t>(c0 + j) * ldc) : 0.f;
    }
    if (r < nrows) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < ncols) C[r + static_cast<int64_t>(c0 + j) * ldc] = b[j] + v[j];
    }
  }
}

__device__ __forceinline__ void sync_all_tc() {
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
}

// Bounded wait on an mbarrier phase.  On expiry (or when another thread of the block
// already gave up) it records kStatusTimeout in the status word, raises the block's
// failure flag and returns false; the task then stops issuing work at its next block
// barrier (task_failed), its successors are never released and the executor drains the
// tensor-core work in flight before it frees tensor memory.
__device__ __forceinline__ bool wait_or_flag(const ExecParams &p, MixedState &ms, uint64_t *bar,
                                             uint32_t parity) {
  if (*ms.fail) return false;
  if (umma::mbar_wait(bar, parity, static_cast<uint64_t>(p.wait_limit_ns), ms.fail)) return true;
  atomicCAS(p.status, 0, kStatusTimeout | (0x7fffff << 8));
  *ms.fail = 1;
  return false;
}

// Thread 0 waits for the operand copies it issued.
__device__ __forceinline__ bool wait_loads(const ExecParams &p, MixedState &ms) {
  const bool ok = wait_or_flag(p, ms, ms.bar_ld, ms.ld_phase);
  if (ok) ms.ld_pending = false;
  return ok;
}

// Thread 0 issues bulk copies of "bytes" in total on the load barrier.
__device__ __forceinline__ void expect_loads(MixedState &ms, uint32_t bytes) {
  umma::mbar_expect_tx(ms.bar_ld, bytes);
  ms.ld_pending = true;
}

// After a block barrier every thread reads the same failure flag.
__device__ __forceinline__ bool task_failed(const MixedState &ms) { return *ms.fail != 0; }

// Shared-memory operand buffers: X and Y always; a third buffer Zb when the parts of
// three operands fit (nparts <= 2), which lets the second operand load early.
struct OperandBufs {
  unsigned char *X, *Y, *Zb;
  uint32_t bytes;  // nparts images
};

__device__ __forceinline__ OperandBufs operand_bufs(unsigned char *raw, int nparts) {
  unsigned char *base = align1024(raw);
  OperandBufs b;
  b.bytes = static_cast<uint32_t>(nparts) * kImg;
  b.X = base;
  b.Y = base + b.bytes;
  b.Zb = nparts <= 2 ? base + 2 * b.bytes : nullptr;
  return b;
}

// UNMQR(i,k,j) on tensor cores:  W^T = C^T V (TMEM 0..127),  P = Z (-W) (TMEM 128..255),
// C = C_old + P (C_old read again, from L2, and added in FP32).  Each product is issued in
// two K halves: the MMAs of the first half run while the second half of its split operand
// (C^T, then W) is being written.
__device__ void task_unmqr_umma(const ExecParams &p, unsigned char *raw, MixedState &ms, int i, int k, int j) {
  const TileGeom geo{p.m, p.n, kMNB};
  const OperandBufs b = operand_bufs(raw, p.nparts);
  const unsigned char *slot = ops_slot(p, i, k, 0);
  const unsigned char *imgV = slot, *imgZ = slot + b.bytes;
  unsigned char *bufZ = b.Zb ? b.Zb : b.Y;
  if (threadIdx.x == 0) {
    expect_loads(ms, b.Zb ? 2 * b.bytes : b.bytes);
    umma::bulk_g2s(b.Y, imgV, b.bytes, ms.bar_ld);
    if (b.Zb) umma::bulk_g2s(b.Zb, imgZ, b.bytes, ms.bar_ld);
  }
  float *C = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, j);
  const int mb = geo.rows(i), ncols = geo.cols(j);
  prefetch_tile_l2(C, p.lda, ncols);  // read twice more: transposed for the image, then by the epilogue
  uint32_t acc = 0u;
  for (int h = 0; h < 2; ++h) {
    c_transposed_image(b.X, C, p.lda, mb, ncols, p.fmt, p.nparts, p.vec4 != 0, h);
    umma::fence_proxy_async();
    sync_all_tc();
    if (task_failed(ms)) return;
    if (threadIdx.x == 0) {
      const bool ok = h != 0 || wait_loads(p, ms);
      if (ok) {
        umma::fence_after();
        issue_product_half(ms.tmem, b.X, b.Y, p.nparts, p.fmt, 0, acc, h);
        if (h == 1) umma::commit(ms.bar_mma);
      }
    }
  }
  ms.ld_phase ^= 1;
  phase_mark(ms.ph, 0);
  wait_or_flag(p, ms, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  if (!b.Zb && threadIdx.x == 0 && !*ms.fail) {  // Y is free again: fetch Z into it
    expect_loads(ms, b.bytes);
    umma::bulk_g2s(b.Y, imgZ, b.bytes, ms.bar_ld);
  }
  phase_mark(ms.ph, 1);
  acc = 0u;
  for (int h = 0; h < 2; ++h) {
    w_image_from_tmem(b.X, ms.tmem, p.fmt, p.nparts, h);
    umma::fence_proxy_async();
    sync_all_tc();
    if (task_failed(ms)) return;
    if (threadIdx.x == 0) {
      const bool ok = !(h == 0 && !b.Zb) || wait_loads(p, ms);
      if (ok) {
        umma::fence_after();
        issue_product_half(ms.tmem + 128, bufZ, b.X, p.nparts, p.fmt, 1, acc, h);
        if (h == 1) umma::commit(ms.bar_mma);
      }
    }
  }
  if (!b.Zb) ms.ld_phase ^= 1;
  phase_mark(ms.ph, 2);
  wait_or_flag(p, ms, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  sync_all_tc();
  if (task_failed(ms)) return;
  tile_plus_tmem(C, p.lda, mb, ncols, ms.tmem + 128, 0);
  sync_all_tc();
  phase_mark(ms.ph, 3);
}

// TTMQR(i,piv,k,j) / TSMQR (V2 dense):  W^T = C1^T + C2^T V2 (the product fresh in TMEM
// 0..127, C1^T added in FP32 while W's image is written);  P2 = Z2 (-W) (TMEM 128..255),
// P1 = T^T (-W) (256..383);  C2 = C2_old + P2, C1 = C1_old + P1 (the old tiles read again,
// from L2, where the task's first step pulled them).  The first two products are issued in
// two K halves like UNMQR's; with two operand buffers C2 is written while T^T arrives.
__device__ void task_ttmqr_umma(const ExecParams &p, unsigned char *raw, MixedState &ms, int i, int piv, int k,
                                int j) {
  const TileGeom geo{p.m, p.n, kMNB};
  const OperandBufs b = operand_bufs(raw, p.nparts);
  const unsigned char *slot = ops_slot(p, i, k, 1);
  const unsigned char *imgV = slot, *imgZ = slot + b.bytes, *imgT = slot + 2 * b.bytes;
  if (threadIdx.x == 0) {
    expect_loads(ms, b.Zb ? 2 * b.bytes : b.bytes);
    umma::bulk_g2s(b.Y, imgV, b.bytes, ms.bar_ld);
    if (b.Zb) umma::bulk_g2s(b.Zb, imgZ, b.bytes, ms.bar_ld);
  }
  float *C1 = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, piv, j);
  float *C2 = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, j);
  const int mb = geo.rows(i), ncols = geo.cols(j);
  // C2 and C1 are each read twice (transposed for the first product / W, then by the
  // epilogue): pull them into L2 now
  prefetch_tile_l2(C2, p.lda, ncols);
  prefetch_tile_l2(C1, p.lda, ncols);
  uint32_t acc = 0u;
  for (int h = 0; h < 2; ++h) {
    c_transposed_image(b.X, C2, p.lda, mb, ncols, p.fmt, p.nparts, p.vec4 != 0, h);
    umma::fence_proxy_async();
    sync_all_tc();
    if (task_failed(ms)) return;
    if (threadIdx.x == 0) {
      const bool ok = h != 0 || wait_loads(p, ms);
      if (ok) {
        umma::fence_after();
        issue_product_half(ms.tmem, b.X, b.Y, p.nparts, p.fmt, 0, acc, h);
        if (h == 1) umma::commit(ms.bar_mma);
      }
    }
  }
  ms.ld_phase ^= 1;
  phase_mark(ms.ph, 0);
  wait_or_flag(p, ms, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  if (threadIdx.x == 0 && !*ms.fail) {  // Y is free: the next operand (Z2, or T^T when Z2 is resident)
    expect_loads(ms, b.bytes);
    umma::bulk_g2s(b.Y, b.Zb ? imgT : imgZ, b.bytes, ms.bar_ld);
  }
  phase_mark(ms.ph, 1);
  acc = 0u;
  for (int h = 0; h < 2; ++h) {
    w_image_from_tmem(b.X, ms.tmem, p.fmt, p.nparts, h, C1, p.lda, ncols, p.vec4 != 0);
    umma::fence_proxy_async();
    sync_all_tc();
    if (task_failed(ms)) return;
    if (threadIdx.x == 0) {
      if (b.Zb) {
        issue_product_half(ms.tmem + 128, b.Zb, b.X, p.nparts, p.fmt, 1, acc, h);  // P2 = -Z2 W
        if (h == 1 && wait_loads(p, ms)) {                                           // T^T in Y
          umma::fence_after();
          issue_product(ms.tmem + 256, b.Y, b.X, p.nparts, p.fmt, 1);                 // P1 = -T^T W
          umma::commit(ms.bar_mma);
        }
      } else {
        const bool ok = h != 0 || wait_loads(p, ms);                                 // Z2 in Y
        if (ok) {
          umma::fence_after();
          issue_product_half(ms.tmem + 128, b.Y, b.X, p.nparts, p.fmt, 1, acc, h);
          if (h == 1) umma::commit(ms.bar_mma);
        }
      }
    }
  }
  ms.ld_phase ^= 1;
  phase_mark(ms.ph, 2);
  if (!b.Zb) {
    // Y held Z2: wait for that product, bring T^T into Y and write C2 (from P2 and the old
    // tile, both in TMEM) while the copy is in flight; then P1 = -T^T W
    wait_or_flag(p, ms, ms.bar_mma, ms.mma_phase);
    ms.mma_phase ^= 1;
    umma::fence_after();
    sync_all_tc();
    if (task_failed(ms)) return;
    if (threadIdx.x == 0) {
      expect_loads(ms, b.bytes);
      umma::bulk_g2s(b.Y, imgT, b.bytes, ms.bar_ld);
    }
    tile_plus_tmem(C2, p.lda, mb, ncols, ms.tmem + 128, 0);
    if (threadIdx.x == 0 && wait_loads(p, ms)) {
      umma::fence_after();
      issue_product(ms.tmem + 256, b.Y, b.X, p.nparts, p.fmt, 1);
      umma::commit(ms.bar_mma);
    }
    ms.ld_phase ^= 1;
  }
  wait_or_flag(p, ms, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  sync_all_tc();
  if (task_failed(ms)) return;
  if (b.Zb) tile_plus_tmem(C2, p.lda, mb, ncols, ms.tmem + 128, 0);
  tile_plus_tmem(C1, p.lda, kMNB, ncols, ms.tmem + 256, 0);
  sync_all_tc();
  phase_mark(ms.ph, 3);
}

}  // namespace
}  // namespace tqr
