// Mixed-precision tile tasks (included by factor.cu; uses its SIMT helpers).
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
// TTMQR(i,piv,k,j) on [C1; C2]:  W^T = C1^T + C2^T V2 (TMEM initialised with C1^T)
//                                C2 -= Z2 W,  C1 -= T^T W
// Products are bf16 x3 (hi*hi + hi*lo + lo*hi) or a single bf16 / fp16 product, always
// accumulated in FP32 in tensor memory.  The tensor-core tile is nb = 128.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "umma.cuh"

namespace tqr {
namespace {

constexpr int kMNB = 128;                       // tile size of the tensor-core path
constexpr int kMLD = kMNB + 1;                  // padded leading dimension of FP32 smem matrices
constexpr uint32_t kImg = kMNB * kMNB * 2;      // one 16-bit operand image, bytes
constexpr uint32_t kSlotBytes = 6 * kImg;       // operand images of one factored tile
constexpr size_t kMixedSmem = 3 * 2 * kImg + 1024;  // three split operands + alignment

__host__ __device__ inline size_t mixed_smem_bytes() {
  const size_t prep = 3 * static_cast<size_t>(kMNB) * kMLD * sizeof(float) + 1024;
  return prep > kMixedSmem ? prep : kMixedSmem;
}

struct MixedState {
  uint64_t *bar_ld, *bar_mma;
  uint32_t tmem;
  uint32_t ld_phase, mma_phase;
  uint64_t *ph;  // phase clock of the execution trace, or null
};

__device__ __forceinline__ unsigned char *ops_slot(const ExecParams &p, int i, int k, int which) {
  return static_cast<unsigned char *>(p.ops) +
         ((static_cast<size_t>(k) * p.P + i) * 2 + which) * static_cast<size_t>(kSlotBytes);
}

__device__ __forceinline__ unsigned char *align1024(unsigned char *raw) {
  const uint32_t a = umma::smem_u32(raw);
  return raw + ((1024u - (a & 1023u)) & 1023u);
}

// Writes an operand image (hi, and lo when requested) whose element (row, kk) is get().
template <typename F>
__device__ void write_image(unsigned char *hi_img, unsigned char *lo_img, F get, int fmt, bool need_lo) {
  for (int ch = threadIdx.x; ch < kMNB * kMNB / 8; ch += kThreads) {
    const int kb = ch >> 10, rem = ch & 1023, row = rem >> 3, sub = rem & 7;
    const int k0 = kb * 64 + ((sub ^ (row & 7)) << 3);
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = get(row, k0 + j);
    uint4 h, l;
    if (fmt == 1)
      umma::split8_bf16(x, h, l);
    else
      umma::split8_f16(x, h, l);
    reinterpret_cast<uint4 *>(hi_img)[ch] = h;
    if (need_lo) reinterpret_cast<uint4 *>(lo_img)[ch] = l;
  }
}

// G(a, c) = sum_r V(r, a) V(r, c) for a < c over the rows rlo(a0,c0)..rhi, in 4x4 tiles.
template <typename RowRange>
__device__ void gram_upper(float *G, const float *V, RowRange range) {
  for (int t = threadIdx.x; t < 32 * 32; t += kThreads) {
    const int ta = t & 31, tc = t >> 5;
    if (ta > tc) continue;
    const int a0 = ta * 4, c0 = tc * 4;
    int r0, r1;
    range(a0, c0, r0, r1);
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    for (int r = r0; r < r1; ++r) {
      float va[4], vc[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        va[x] = V[r + (a0 + x) * kMLD];
        vc[x] = V[r + (c0 + x) * kMLD];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += va[x] * vc[y];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        if (a0 + x < c0 + y) G[(a0 + x) + (c0 + y) * kMLD] = acc[x][y];
  }
}

// T_full from its ib x ib diagonal blocks (already in Ts) and the Gram matrix (Gs).
// Block column j: X = G(0:c0, blk) T(blk, blk);  T(0:c0, blk) = -T(0:c0, 0:c0) X.
__device__ void assemble_t(float *Ts, float *Gs, int ib) {
  for (int c0 = ib; c0 < kMNB; c0 += ib) {
    const int w = min(ib, kMNB - c0);
    const int nout = c0 * w;
    float reg[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int o = threadIdx.x + s * kThreads;
      reg[s] = 0.f;
      if (o < nout) {
        const int a = o % c0, cc = o / c0;
        float acc = 0.f;
        for (int b = 0; b <= cc; ++b) acc += Gs[a + (c0 + b) * kMLD] * Ts[(c0 + b) + (c0 + cc) * kMLD];
        reg[s] = acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int o = threadIdx.x + s * kThreads;
      if (o < nout) Gs[(o % c0) + (c0 + o / c0) * kMLD] = reg[s];
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int o = threadIdx.x + s * kThreads;
      reg[s] = 0.f;
      if (o < nout) {
        const int a = o % c0, cc = o / c0;
        float acc = 0.f;
        for (int b = a; b < c0; ++b) acc += Ts[a + b * kMLD] * Gs[b + (c0 + cc) * kMLD];
        reg[s] = -acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int o = threadIdx.x + s * kThreads;
      if (o < nout) Ts[(o % c0) + (c0 + o / c0) * kMLD] = reg[s];
    }
    __syncthreads();
  }
}

// Z(r, a) = sum_b V(r, b) T(a, b) (= V T^T), b over [max(a0, blo(r0)), bhi(r0)) in 4x4 tiles.
template <typename Bounds>
__device__ void v_times_tt(float *Z, const float *V, const float *Ts, Bounds bounds) {
  for (int t = threadIdx.x; t < 32 * 32; t += kThreads) {
    const int tr = t & 31, ta = t >> 5;
    const int r0 = tr * 4, a0 = ta * 4;
    int b0, b1;
    bounds(r0, a0, b0, b1);
    float acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
    for (int b = b0; b < b1; ++b) {
      float vr[4], ta4[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        vr[x] = V[(r0 + x) + b * kMLD];
        ta4[x] = Ts[(a0 + x) + b * kMLD];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += vr[x] * ta4[y];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) Z[(r0 + x) + (a0 + y) * kMLD] = acc[x][y];
  }
}

// Loads the ib-blocked T of a factored tile into the block diagonal of Ts (zeros elsewhere).
__device__ void load_t_blocks(float *Ts, const float *Tg, int ib) {
  for (int idx = threadIdx.x; idx < kMNB * kMNB; idx += kThreads) {
    const int c = idx >> 7, a = idx & 127;
    const int cb = (c / ib) * ib;
    float v = 0.f;
    if (a >= cb && a <= c) v = static_cast<float>(ldcg(Tg + (a - cb) + static_cast<int64_t>(c) * ib));
    Ts[a + c * kMLD] = v;
  }
}

// Operand images of GEQRT(i,k): V and Z = V T_full^T.
__device__ void prep_geqrt_ops(const ExecParams &p, unsigned char *raw, int i, int k) {
  const TileGeom geo{p.m, p.n, kMNB};
  float *Vs = reinterpret_cast<float *>(raw);
  float *Ts = Vs + kMNB * kMLD;
  float *Gs = Ts + kMNB * kMLD;
  const float *tile = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, k);
  const float *Tg = t_ptr(static_cast<float *>(p.T), p.P, p.ib, kMNB, i, k, 0);
  const int mb = geo.rows(i), K = min(mb, geo.cols(k));
  for (int idx = threadIdx.x; idx < kMNB * kMNB; idx += kThreads) {
    const int c = idx >> 7, r = idx & 127;
    float v = 0.f;
    if (c < K && r < mb) v = r > c ? static_cast<float>(ldcg(tile + r + static_cast<int64_t>(c) * p.lda)) : (r == c ? 1.f : 0.f);
    Vs[r + c * kMLD] = v;
  }
  load_t_blocks(Ts, Tg, p.ib);
  __syncthreads();
  // G(a, c) = v_a . v_c over rows r >= c (v_c is zero above its diagonal)
  gram_upper(Gs, Vs, [](int a0, int c0, int &r0, int &r1) { r0 = c0; r1 = kMNB; });
  __syncthreads();
  assemble_t(Ts, Gs, p.ib);
  // Z = V T^T: Z(r, a) = sum_{a <= b <= r} V(r, b) T(a, b)
  v_times_tt(Gs, Vs, Ts, [](int r0, int a0, int &b0, int &b1) { b0 = a0; b1 = min(r0 + 4, kMNB); });
  __syncthreads();
  unsigned char *slot = ops_slot(p, i, k, 0);
  const bool lo = p.nprod == 3;
  write_image(slot, slot + kImg, [&](int row, int kk) { return Vs[kk + row * kMLD]; }, p.fmt, lo);
  write_image(slot + 2 * kImg, slot + 3 * kImg, [&](int row, int kk) { return Gs[row + kk * kMLD]; }, p.fmt, lo);
  __syncthreads();
}

// Operand images of TTQRT(i,piv,k): V2 (upper part of tile i), Z2 = V2 T_full^T, T_full^T.
__device__ void prep_ttqrt_ops(const ExecParams &p, unsigned char *raw, int i, int k) {
  const TileGeom geo{p.m, p.n, kMNB};
  float *Vs = reinterpret_cast<float *>(raw);
  float *Ts = Vs + kMNB * kMLD;
  float *Gs = Ts + kMNB * kMLD;
  const float *tile = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, k);
  const float *Tt = t_ptr(static_cast<float *>(p.T), p.P, p.ib, kMNB, i, k, 1);
  const int mb = geo.rows(i), K = geo.cols(k);
  for (int idx = threadIdx.x; idx < kMNB * kMNB; idx += kThreads) {
    const int c = idx >> 7, r = idx & 127;
    float v = 0.f;
    if (c < K && r < mb && r <= c) v = static_cast<float>(ldcg(tile + r + static_cast<int64_t>(c) * p.lda));
    Vs[r + c * kMLD] = v;
  }
  load_t_blocks(Ts, Tt, p.ib);
  __syncthreads();
  // G(a, c) = v_a . v_c over rows r <= a (the tails live in the upper triangle)
  gram_upper(Gs, Vs, [](int a0, int c0, int &r0, int &r1) { r0 = 0; r1 = min(a0 + 4, kMNB); });
  __syncthreads();
  assemble_t(Ts, Gs, p.ib);
  // Z2(r, a) = sum_{b >= max(a, r)} V2(r, b) T(a, b)
  v_times_tt(Gs, Vs, Ts, [](int r0, int a0, int &b0, int &b1) { b0 = min(a0, r0); b1 = kMNB; });
  __syncthreads();
  unsigned char *slot = ops_slot(p, i, k, 1);
  const bool lo = p.nprod == 3;
  write_image(slot, slot + kImg, [&](int row, int kk) { return Vs[kk + row * kMLD]; }, p.fmt, lo);
  write_image(slot + 2 * kImg, slot + 3 * kImg, [&](int row, int kk) { return Gs[row + kk * kMLD]; }, p.fmt, lo);
  write_image(slot + 4 * kImg, slot + 5 * kImg, [&](int row, int kk) { return Ts[kk + row * kMLD]; }, p.fmt, lo);
  __syncthreads();
}

// D(128 x 128, FP32 in TMEM) (+)= A (128 x 128) B^T over K = 128, both split images.
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, const unsigned char *bufA, const unsigned char *bufB,
                                           int nprod, int fmt, uint32_t accumulate_first) {
  const uint32_t idesc = umma::idesc_f16(128, 128, fmt, 0);
  const uint32_t a_hi = umma::smem_u32(bufA), a_lo = a_hi + kImg;
  const uint32_t b_hi = umma::smem_u32(bufB), b_lo = b_hi + kImg;
#pragma unroll 1
  for (int ks = 0; ks < kMNB / 16; ++ks) {
    const uint32_t off = (ks >> 2) * (kMNB * 128) + (ks & 3) * 32;
    const uint32_t acc = (ks > 0 || accumulate_first) ? 1u : 0u;
    if (nprod == 3) {
      umma::mma_f16(d_tmem, umma::smem_desc(a_lo + off), umma::smem_desc(b_hi + off), idesc, acc);
      umma::mma_f16(d_tmem, umma::smem_desc(a_hi + off), umma::smem_desc(b_lo + off), idesc, 1u);
      umma::mma_f16(d_tmem, umma::smem_desc(a_hi + off), umma::smem_desc(b_hi + off), idesc, 1u);
    } else {
      umma::mma_f16(d_tmem, umma::smem_desc(a_hi + off), umma::smem_desc(b_hi + off), idesc, acc);
    }
  }
}

// Writes C^T (row c, k = r) of a tile as a split image into shared memory.
__device__ void c_transposed_image(unsigned char *img, const float *C, int64_t ldc, int mb, int ncols, int fmt,
                                   bool need_lo) {
  for (int ch = threadIdx.x; ch < kMNB * kMNB / 8; ch += kThreads) {
    const int kb = ch >> 10, rem = ch & 1023, row = rem >> 3, sub = rem & 7;
    const int k0 = kb * 64 + ((sub ^ (row & 7)) << 3);
    float x[8];
    const float *col = C + static_cast<int64_t>(row) * ldc;
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (row < ncols && k0 + j < mb) ? __ldcg(col + k0 + j) : 0.f;
    uint4 h, l;
    if (fmt == 1)
      umma::split8_bf16(x, h, l);
    else
      umma::split8_f16(x, h, l);
    reinterpret_cast<uint4 *>(img)[ch] = h;
    if (need_lo) reinterpret_cast<uint4 *>(img + kImg)[ch] = l;
  }
}

// W^T (TMEM lane c, column a) -> split image of W as a B operand (row c, k = a).
__device__ void w_image_from_tmem(unsigned char *img, uint32_t tmem_w, int fmt, bool need_lo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = (warp & 3) * 32 + lane;
  const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
  for (int g = 0; g < 2; ++g) {
    const int a0 = (warp >> 2) * 64 + g * 32;
    float v[32];
    umma::tmem_ld32(tmem_w + lane_base + a0, v);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      uint4 h, l;
      if (fmt == 1)
        umma::split8_bf16(v + 8 * u, h, l);
      else
        umma::split8_f16(v + 8 * u, h, l);
      const uint32_t off = umma::sw128_offset(c, a0 + 8 * u, kMNB);
      *reinterpret_cast<uint4 *>(img + off) = h;
      if (need_lo) *reinterpret_cast<uint4 *>(img + kImg + off) = l;
    }
  }
}

// C(r, c) -= D(r, c) for the accumulator at tmem_d (lane r, column c).
__device__ void subtract_from_tmem(float *C, int64_t ldc, int nrows, int ncols, uint32_t tmem_d) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = (warp & 3) * 32 + lane;
  const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
  for (int g = 0; g < 2; ++g) {
    const int c0 = (warp >> 2) * 64 + g * 32;
    float v[32];
    umma::tmem_ld32(tmem_d + lane_base + c0, v);
    if (r < nrows) {
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        if (c < ncols) {
          float *ptr = C + r + static_cast<int64_t>(c) * ldc;
          *ptr = __ldcg(ptr) - v[j];
        }
      }
    }
  }
}

__device__ __forceinline__ void sync_all_tc() {
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
}

// Records a failed bounded wait in the status word.
__device__ __forceinline__ void wait_or_flag(const ExecParams &p, uint64_t *bar, uint32_t parity) {
  if (!umma::mbar_wait(bar, parity, 1ull << 26)) atomicCAS(p.status, 0, kStatusTimeout | (0x7fffff << 8));
}

__device__ void task_unmqr_umma(const ExecParams &p, unsigned char *raw, MixedState &ms, int i, int k, int j) {
  const TileGeom geo{p.m, p.n, kMNB};
  unsigned char *base = align1024(raw);
  unsigned char *bufA = base, *bufB = base + 2 * kImg, *bufZ = base + 4 * kImg;
  const bool lo = p.nprod == 3;
  const uint32_t nimg = lo ? 2 : 1;
  const unsigned char *slot = ops_slot(p, i, k, 0);
  if (threadIdx.x == 0) {
    umma::mbar_expect_tx(ms.bar_ld, 2 * nimg * kImg);
    umma::bulk_g2s(bufB, slot, nimg * kImg, ms.bar_ld);
    umma::bulk_g2s(bufZ, slot + 2 * kImg, nimg * kImg, ms.bar_ld);
  }
  float *C = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, j);
  const int mb = geo.rows(i), ncols = geo.cols(j);
  c_transposed_image(bufA, C, p.lda, mb, ncols, p.fmt, lo);
  umma::fence_proxy_async();
  sync_all_tc();
  phase_mark(ms.ph, 0);
  if (threadIdx.x == 0) {
    wait_or_flag(p, ms.bar_ld, ms.ld_phase);
    umma::fence_after();
    issue_gemm(ms.tmem, bufA, bufB, p.nprod, p.fmt, 0);
    umma::commit(ms.bar_mma);
  }
  ms.ld_phase ^= 1;
  wait_or_flag(p, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  phase_mark(ms.ph, 1);
  w_image_from_tmem(bufA, ms.tmem, p.fmt, lo);
  umma::fence_proxy_async();
  sync_all_tc();
  phase_mark(ms.ph, 2);
  if (threadIdx.x == 0) {
    issue_gemm(ms.tmem + 128, bufZ, bufA, p.nprod, p.fmt, 0);
    umma::commit(ms.bar_mma);
  }
  wait_or_flag(p, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  subtract_from_tmem(C, p.lda, mb, ncols, ms.tmem + 128);
  sync_all_tc();
  phase_mark(ms.ph, 3);
}

__device__ void task_ttmqr_umma(const ExecParams &p, unsigned char *raw, MixedState &ms, int i, int piv, int k,
                                int j) {
  const TileGeom geo{p.m, p.n, kMNB};
  unsigned char *base = align1024(raw);
  unsigned char *bufA = base, *bufB = base + 2 * kImg, *bufZ = base + 4 * kImg;
  const bool lo = p.nprod == 3;
  const uint32_t nimg = lo ? 2 : 1;
  const unsigned char *slot = ops_slot(p, i, k, 1);
  if (threadIdx.x == 0) {
    umma::mbar_expect_tx(ms.bar_ld, 2 * nimg * kImg);
    umma::bulk_g2s(bufB, slot, nimg * kImg, ms.bar_ld);
    umma::bulk_g2s(bufZ, slot + 2 * kImg, nimg * kImg, ms.bar_ld);
  }
  float *C1 = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, piv, j);
  float *C2 = tile_ptr(static_cast<float *>(p.A), p.lda, kMNB, i, j);
  const int mb = geo.rows(i), ncols = geo.cols(j);
  c_transposed_image(bufA, C2, p.lda, mb, ncols, p.fmt, lo);
  // TMEM D1 (lane c, column a) = C1(a, c): the identity part of the TT reflectors
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = (warp & 3) * 32 + lane;
    const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
    const float *col = C1 + static_cast<int64_t>(c) * p.lda;
    for (int g = 0; g < 2; ++g) {
      const int a0 = (warp >> 2) * 64 + g * 32;
      float v[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) v[u] = c < ncols ? __ldcg(col + a0 + u) : 0.f;
      umma::tmem_st32(ms.tmem + lane_base + a0, v);
    }
    umma::tmem_wait_st();
  }
  umma::fence_proxy_async();
  sync_all_tc();
  phase_mark(ms.ph, 0);
  if (threadIdx.x == 0) {
    wait_or_flag(p, ms.bar_ld, ms.ld_phase);
    umma::fence_after();
    issue_gemm(ms.tmem, bufA, bufB, p.nprod, p.fmt, 1);
    umma::commit(ms.bar_mma);
  }
  ms.ld_phase ^= 1;
  wait_or_flag(p, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  phase_mark(ms.ph, 1);
  w_image_from_tmem(bufA, ms.tmem, p.fmt, lo);
  umma::fence_proxy_async();
  sync_all_tc();
  phase_mark(ms.ph, 2);
  if (threadIdx.x == 0) {
    umma::mbar_expect_tx(ms.bar_ld, nimg * kImg);
    umma::bulk_g2s(bufB, slot + 4 * kImg, nimg * kImg, ms.bar_ld);
    issue_gemm(ms.tmem + 128, bufZ, bufA, p.nprod, p.fmt, 0);
    wait_or_flag(p, ms.bar_ld, ms.ld_phase);
    umma::fence_after();
    issue_gemm(ms.tmem + 256, bufB, bufA, p.nprod, p.fmt, 0);
    umma::commit(ms.bar_mma);
  }
  ms.ld_phase ^= 1;
  wait_or_flag(p, ms.bar_mma, ms.mma_phase);
  ms.mma_phase ^= 1;
  umma::fence_after();
  subtract_from_tmem(C2, p.lda, mb, ncols, ms.tmem + 128);
  subtract_from_tmem(C1, p.lda, kMNB, ncols, ms.tmem + 256);
  sync_all_tc();
  phase_mark(ms.ph, 3);
}

}  // namespace
}  // namespace tqr
