// Double-complex tiled QR (the thesis's second precision, Section 3.3): the persistent
// tile-task executor with complex GEQRT / TTQRT / TSQRT panels and UNMQR / TTMQR / TSMQR
// updates (Table "Kernels for tiled QR"; the update kernels multiply by the unitary Q,
// glossary), plus the complex triangular solve of the least-squares path.
//
// Storage: interleaved complex double (re, im), column-major, leading dimensions in
// complex elements.  The task graph, its claim order and the dependency counters are
// those of the real executor; only the tile kernels differ.
//
// Reflector convention (LAPACK's complex one): H = I - tau v v^H, v(0) = 1, beta =
// -sign(Re alpha) ||[alpha; x]|| (real), tau = (beta - alpha) / beta, v = x / (alpha -
// beta), so H^H [alpha; x] = [beta; 0]; tau = 0 only when x = 0 and alpha is real.  The
// factorization applies H^H to the trailing columns; Q^H B applies the H^H in order, Q B
// the H in reverse.  T of ib reflectors: H_1 ... H_b = I - V T V^H, T upper triangular,
// T(0:c, c) = -tau_c T(0:c, 0:c) (V(:, 0:c)^H v_c), stored ib x nb per factored tile.
//
// The kernels favour simplicity over speed (one block barrier per step of a reflector);
// the complex path has no tensor-core form.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/tqr.h"
#include "tqr_internal.h"

namespace tqr {
namespace {

constexpr int kZThreads = 256;
constexpr int kZWarps = kZThreads / 32;
constexpr int kZChunk = 16;  // columns of an update chunk in shared memory

struct Z {
  double re, im;
};
__device__ __forceinline__ Z zmk(double r, double i) { return Z{r, i}; }
__device__ __forceinline__ Z operator+(Z a, Z b) { return Z{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Z operator-(Z a, Z b) { return Z{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Z operator*(Z a, Z b) {
  return Z{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__device__ __forceinline__ Z conj(Z a) { return Z{a.re, -a.im}; }
__device__ __forceinline__ double abs2(Z a) { return fma(a.re, a.re, a.im * a.im); }
// acc + conj(a) * b
__device__ __forceinline__ Z fma_conj(Z a, Z b, Z acc) {
  return Z{fma(a.re, b.re, fma(a.im, b.im, acc.re)), fma(a.re, b.im, fma(-a.im, b.re, acc.im))};
}
__device__ __forceinline__ Z zld(const Z *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return Z{v.x, v.y};
}

__device__ __forceinline__ double zwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ uint64_t zglobaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared memory of one CTA.
struct ZSmem {
  Z *V, *C, *C1, *W, *T, *G, *P1, *tau;
  double *red;  // [kZWarps] partial sums
  int ldv, ldw, ldt;
};

__host__ __device__ inline size_t zsmem_bytes(int nb, int ib) {
  const size_t ldv = nb + 1, ldw = ib + 1, ldt = ib + 1;
  const size_t elems = ldv * ib + 2 * ldv * kZChunk + ldw * kZChunk + 3 * ldt * ib + ib;
  return elems * sizeof(Z) + kZWarps * sizeof(double);
}

__device__ ZSmem zcarve(unsigned char *raw, int nb, int ib) {
  ZSmem s;
  s.ldv = nb + 1;
  s.ldw = ib + 1;
  s.ldt = ib + 1;
  Z *p = reinterpret_cast<Z *>(raw);
  s.V = p;
  p += s.ldv * ib;
  s.C = p;
  p += s.ldv * kZChunk;
  s.C1 = p;
  p += s.ldv * kZChunk;
  s.W = p;
  p += s.ldw * kZChunk;
  s.T = p;
  p += s.ldt * ib;
  s.G = p;
  p += s.ldt * ib;
  s.P1 = p;
  p += s.ldt * ib;
  s.tau = p;
  p += ib;
  s.red = reinterpret_cast<double *>(p);
  return s;
}

// dst(r, c) = src(r, c) where keep(r, c), zero elsewhere, r < nrows, c < ncols.
template <typename Keep>
__device__ void zload(Z *dst, int ldd, const Z *src, int64_t lds, int nrows, int ncols, Keep keep) {
  for (int idx = threadIdx.x; idx < nrows * ncols; idx += kZThreads) {
    const int c = idx / nrows, r = idx - c * nrows;
    dst[r + c * ldd] = keep(r, c) ? zld(src + r + static_cast<int64_t>(c) * lds) : Z{0.0, 0.0};
  }
}

__device__ void zstore(Z *dst, int64_t ldd, const Z *src, int lds, int nrows, int ncols) {
  for (int idx = threadIdx.x; idx < nrows * ncols; idx += kZThreads) {
    const int c = idx / nrows, r = idx - c * nrows;
    dst[r + static_cast<int64_t>(c) * ldd] = src[r + c * lds];
  }
}

// Block-wide sum of one double per thread (every thread gets the result).
__device__ double zblock_sum(double v, double *red) {
  v = zwarp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();  // red may still be read by the previous sum
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kZWarps; ++w) s += red[w];
  return s;
}

// Householder factorization of a panel block of kb columns in shared memory.
// kind 0 GEQRT: head V(c, c), tail V(c+1 .. rows-1, c).
// kind 1 TT:    head P1(c, c), tail V(0 .. min(c0+c+1, mb)-1, c).
// kind 2 TS:    head P1(c, c), tail V(0 .. rows-1, c).
// Reflector c applies H^H to the later columns of the block; the tails end as v, the
// heads as beta, s.tau holds tau.
__device__ void zpanel(ZSmem &s, int kind, int kb, int rows, int c0, int mb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ Z s_scal;
  for (int c = 0; c < kb; ++c) {
    const int lo = kind == 0 ? c + 1 : 0;
    const int hi = kind == 1 ? min(c0 + c + 1, mb) : rows;
    Z *head_c = kind == 0 ? &s.V[c + c * s.ldv] : &s.P1[c + c * s.ldt];
    Z *x = s.V + c * s.ldv;
    double part = 0.0;
    for (int r = lo + threadIdx.x; r < hi; r += kZThreads) part += abs2(x[r]);
    const double xx = zblock_sum(part, s.red);
    if (threadIdx.x == 0) {
      const Z alpha = *head_c;
      Z tau{0.0, 0.0}, scal{0.0, 0.0};
      double beta = alpha.re;
      if (!(xx == 0.0 && alpha.im == 0.0)) {
        const double nrm = sqrt(abs2(alpha) + xx);
        beta = alpha.re >= 0.0 ? -nrm : nrm;
        tau = Z{(beta - alpha.re) / beta, -alpha.im / beta};
        const Z d{alpha.re - beta, alpha.im};  // scal = 1 / (alpha - beta)
        const double dd = abs2(d);
        scal = Z{d.re / dd, -d.im / dd};
        *head_c = Z{beta, 0.0};
      }
      s.tau[c] = tau;
      s_scal = scal;
    }
    __syncthreads();
    const Z scal = s_scal, tau = s.tau[c];
    for (int r = lo + threadIdx.x; r < hi; r += kZThreads) x[r] = x[r] * scal;
    __syncthreads();
    if (tau.re != 0.0 || tau.im != 0.0) {
      const Z ctau = conj(tau);
      for (int cc = c + 1 + warp; cc < kb; cc += kZWarps) {
        Z *y = s.V + cc * s.ldv;
        Z *head = kind == 0 ? &s.V[c + cc * s.ldv] : &s.P1[c + cc * s.ldt];
        Z acc{0.0, 0.0};
        for (int r = lo + lane; r < hi; r += 32) acc = fma_conj(x[r], y[r], acc);
        acc.re = zwarp_sum(acc.re);
        acc.im = zwarp_sum(acc.im);
        const Z w = *head + acc;  // v^H [head; tail] with v(0) = 1
        const Z tw = ctau * w;
        __syncwarp();
        if (lane == 0) *head = *head - tw;
        for (int r = lo + lane; r < hi; r += 32) y[r] = y[r] - x[r] * tw;
      }
    }
    __syncthreads();
  }
}

// T (kb x kb, upper) of the block's reflectors from their Gram matrix: G(a, c) =
// v_a^H v_c over the tails (the explicit unit entries of GEQRT's vectors are stored in
// s.V; the TT / TS unit entries sit in different rows and are orthogonal).
__device__ void zbuild_t(ZSmem &s, int kb, int nrows) {
  for (int idx = threadIdx.x; idx < kb * kb; idx += kZThreads) {
    const int c = idx / kb, a = idx - c * kb;
    if (a < c) {
      Z acc{0.0, 0.0};
      for (int r = 0; r < nrows; ++r) acc = fma_conj(s.V[r + a * s.ldv], s.V[r + c * s.ldv], acc);
      s.G[a + c * s.ldt] = acc;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int a = threadIdx.x;
    for (int c = 0; c < kb; ++c) {
      // T(a, c) = -tau_c sum_{a <= b < c} T(a, b) G(b, c); T(c, c) = tau_c
      Z v{0.0, 0.0};
      if (a < c) {
        Z acc{0.0, 0.0};
        for (int b = a; b < c; ++b) acc = acc + s.T[a + b * s.ldt] * s.G[b + c * s.ldt];
        const Z t = s.tau[c];
        v = Z{0.0, 0.0} - t * acc;
      } else if (a == c) {
        v = s.tau[c];
      }
      if (a < kb) s.T[a + c * s.ldt] = v;
      __syncwarp();
    }
  }
  __syncthreads();
}

// Block reflector of kb reflectors applied to a chunk of ncols columns:
//   W = [C1(0:kb, :)] + V^H C;  W = T^H W (adjoint: Q^H) or T W (Q);  C1 -= W;  C -= V W.
__device__ void zapply(Z *C, int ldc, int nrows, Z *C1, int ldc1, int ncols, const ZSmem &s, int kb,
                       bool adjoint) {
  for (int idx = threadIdx.x; idx < kb * ncols; idx += kZThreads) {
    const int c = idx / kb, a = idx - c * kb;
    Z acc = C1 ? C1[a + c * ldc1] : Z{0.0, 0.0};
    for (int r = 0; r < nrows; ++r) acc = fma_conj(s.V[r + a * s.ldv], C[r + c * ldc], acc);
    s.W[a + c * s.ldw] = acc;
  }
  __syncthreads();
  Z nw[(32 * kZChunk + kZThreads - 1) / kZThreads];
  int u = 0;
  for (int idx = threadIdx.x; idx < kb * ncols; idx += kZThreads, ++u) {
    const int c = idx / kb, a = idx - c * kb;
    Z acc{0.0, 0.0};
    if (adjoint) {
      for (int b = 0; b <= a; ++b) acc = fma_conj(s.T[b + a * s.ldt], s.W[b + c * s.ldw], acc);
    } else {
      for (int b = a; b < kb; ++b) acc = acc + s.T[a + b * s.ldt] * s.W[b + c * s.ldw];
    }
    nw[u] = acc;
  }
  __syncthreads();
  u = 0;
  for (int idx = threadIdx.x; idx < kb * ncols; idx += kZThreads, ++u) {
    const int c = idx / kb, a = idx - c * kb;
    s.W[a + c * s.ldw] = nw[u];
    if (C1) C1[a + c * ldc1] = C1[a + c * ldc1] - nw[u];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nrows * ncols; idx += kZThreads) {
    const int c = idx / nrows, r = idx - c * nrows;
    Z acc{0.0, 0.0};
    for (int a = 0; a < kb; ++a) acc = acc + s.V[r + a * s.ldv] * s.W[a + c * s.ldw];
    C[r + c * ldc] = C[r + c * ldc] - acc;
  }
  __syncthreads();
}

__device__ __forceinline__ Z *ztile(Z *A, int64_t lda, int nb, int i, int j) {
  return A + static_cast<int64_t>(j) * nb * lda + static_cast<int64_t>(i) * nb;
}
__device__ __forceinline__ Z *zt_ptr(Z *T, int P, int ib, int nb, int i, int k, int which) {
  return T + (static_cast<int64_t>(k) * P + i) * 2 * ib * nb + static_cast<int64_t>(which) * ib * nb;
}
__device__ __forceinline__ int zrows(const ExecParams &p, int i) {
  return static_cast<int>(min(static_cast<int64_t>(p.nb), p.m - static_cast<int64_t>(i) * p.nb));
}
__device__ __forceinline__ int zcols(const ExecParams &p, int j) {
  return static_cast<int>(min(static_cast<int64_t>(p.nb), p.n - static_cast<int64_t>(j) * p.nb));
}

// T slice of reflectors c0 .. c0+width-1 (zeros outside the kb x kb block).
__device__ void zstore_t(Z *Tg, int ib, int c0, int width, const ZSmem &s, int kb) {
  for (int idx = threadIdx.x; idx < ib * width; idx += kZThreads) {
    const int c = idx / ib, a = idx - c * ib;
    Tg[a + static_cast<int64_t>(c0 + c) * ib] = (a < kb && c < kb) ? s.T[a + c * s.ldt] : Z{0.0, 0.0};
  }
}

__device__ void ztask_geqrt(const ExecParams &p, ZSmem &s, int i, int k) {
  const int nb = p.nb, ib = p.ib;
  Z *tile = ztile(static_cast<Z *>(p.A), p.lda, nb, i, k);
  Z *Tg = zt_ptr(static_cast<Z *>(p.T), p.P, ib, nb, i, k, 0);
  const int mb = zrows(p, i), ncol = zcols(p, k), K = min(mb, ncol);
  for (int c0 = 0; c0 < nb; c0 += ib) {
    const int width = min(ib, nb - c0), kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      zstore_t(Tg, ib, c0, width, s, 0);
      continue;
    }
    const int rows = mb - c0;
    Z *blk = tile + c0 + static_cast<int64_t>(c0) * p.lda;
    zload(s.V, s.ldv, blk, p.lda, rows, kb, [](int, int) { return true; });
    __syncthreads();
    zpanel(s, 0, kb, rows, c0, mb);
    zstore(blk, p.lda, s.V, s.ldv, rows, kb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < kb * kb; idx += kZThreads) {  // explicit unit diagonal, zeros above
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) s.V[r + c * s.ldv] = r == c ? Z{1.0, 0.0} : Z{0.0, 0.0};
    }
    __syncthreads();
    zbuild_t(s, kb, rows);
    zstore_t(Tg, ib, c0, width, s, kb);
    for (int cs = c0 + kb; cs < ncol; cs += kZChunk) {
      const int w = min(kZChunk, ncol - cs);
      Z *cb = tile + c0 + static_cast<int64_t>(cs) * p.lda;
      zload(s.C, s.ldv, cb, p.lda, rows, w, [](int, int) { return true; });
      __syncthreads();
      zapply(s.C, s.ldv, rows, nullptr, 0, w, s, kb, true);
      zstore(cb, p.lda, s.C, s.ldv, rows, w);
      __syncthreads();
    }
  }
}

// TTQRT (ts false) / TSQRT (ts true) of tile (i,k) under the triangle of (piv,k).
__device__ void ztask_pair_qrt(const ExecParams &p, ZSmem &s, int i, int piv, int k, bool ts) {
  const int nb = p.nb, ib = p.ib;
  Z *A = static_cast<Z *>(p.A);
  Z *t1 = ztile(A, p.lda, nb, piv, k), *t2 = ztile(A, p.lda, nb, i, k);
  Z *Tt = zt_ptr(static_cast<Z *>(p.T), p.P, ib, nb, i, k, 1);
  const int mb = zrows(p, i), K = zcols(p, k);
  for (int c0 = 0; c0 < nb; c0 += ib) {
    const int width = min(ib, nb - c0), kb = max(0, min(ib, K - c0));
    if (kb == 0) {
      zstore_t(Tt, ib, c0, width, s, 0);
      continue;
    }
    const int rb = ts ? mb : min(c0 + kb, mb);
    zload(s.V, s.ldv, t2 + static_cast<int64_t>(c0) * p.lda, p.lda, rb, kb,
          [c0, ts](int r, int c) { return ts || r <= c0 + c; });
    zload(s.P1, s.ldt, t1 + c0 + static_cast<int64_t>(c0) * p.lda, p.lda, kb, kb, [](int r, int c) { return r <= c; });
    __syncthreads();
    zpanel(s, ts ? 2 : 1, kb, rb, c0, mb);
    zbuild_t(s, kb, rb);
    for (int idx = threadIdx.x; idx < rb * kb; idx += kZThreads) {
      const int c = idx / rb, r = idx - c * rb;
      if (ts || r <= c0 + c) t2[r + static_cast<int64_t>(c0 + c) * p.lda] = s.V[r + c * s.ldv];
    }
    for (int idx = threadIdx.x; idx < kb * kb; idx += kZThreads) {
      const int c = idx / kb, r = idx - c * kb;
      if (r <= c) t1[(c0 + r) + static_cast<int64_t>(c0 + c) * p.lda] = s.P1[r + c * s.ldt];
    }
    zstore_t(Tt, ib, c0, width, s, kb);
    __syncthreads();
    for (int cs = c0 + kb; cs < K; cs += kZChunk) {
      const int w = min(kZChunk, K - cs);
      Z *c1 = t1 + c0 + static_cast<int64_t>(cs) * p.lda, *c2 = t2 + static_cast<int64_t>(cs) * p.lda;
      zload(s.C1, s.ldv, c1, p.lda, kb, w, [](int, int) { return true; });
      zload(s.C, s.ldv, c2, p.lda, rb, w, [](int, int) { return true; });
      __syncthreads();
      zapply(s.C, s.ldv, rb, s.C1, s.ldv, w, s, kb, true);
      zstore(c1, p.lda, s.C1, s.ldv, kb, w);
      zstore(c2, p.lda, s.C, s.ldv, rb, w);
      __syncthreads();
    }
  }
}

// UNMQR: C (mb x ncols at cptr) <- Q^H C (adjoint) or Q C with GEQRT(i,k)'s reflectors.
__device__ void ztask_unmqr(const ExecParams &p, ZSmem &s, int i, int k, Z *cptr, int64_t ldc, int ncols,
                            bool adjoint) {
  const int nb = p.nb, ib = p.ib;
  const Z *vt = ztile(static_cast<Z *>(p.A), p.lda, nb, i, k);
  const Z *Tg = zt_ptr(static_cast<Z *>(p.T), p.P, ib, nb, i, k, 0);
  const int mb = zrows(p, i), K = min(mb, zcols(p, k)), nblk = (K + ib - 1) / ib;
  for (int cs = 0; cs < ncols; cs += kZChunk) {
    const int w = min(kZChunk, ncols - cs);
    Z *cb = cptr + static_cast<int64_t>(cs) * ldc;
    zload(s.C, s.ldv, cb, ldc, mb, w, [](int, int) { return true; });
    for (int bb = 0; bb < nblk; ++bb) {
      const int b = adjoint ? bb : nblk - 1 - bb;
      const int c0 = b * ib, kb = min(ib, K - c0), rows = mb - c0;
      const Z *vb = vt + c0 + static_cast<int64_t>(c0) * p.lda;
      __syncthreads();
      for (int idx = threadIdx.x; idx < rows * kb; idx += kZThreads) {
        const int c = idx / rows, r = idx - c * rows;
        s.V[r + c * s.ldv] = r > c ? zld(vb + r + static_cast<int64_t>(c) * p.lda) : (r == c ? Z{1.0, 0.0} : Z{0.0, 0.0});
      }
      zload(s.T, s.ldt, Tg + static_cast<int64_t>(c0) * ib, ib, kb, kb, [](int, int) { return true; });
      __syncthreads();
      zapply(s.C + c0, s.ldv, rows, nullptr, 0, w, s, kb, adjoint);
    }
    zstore(cb, ldc, s.C, s.ldv, mb, w);
    __syncthreads();
  }
}

// TTMQR / TSMQR on the pair (C1: pivot row's K rows, C2: row i's mb rows).
__device__ void ztask_pair_mqr(const ExecParams &p, ZSmem &s, int i, int k, Z *c1ptr, Z *c2ptr, int64_t ldc,
                               int ncols, bool adjoint, bool ts) {
  const int nb = p.nb, ib = p.ib;
  const Z *vt = ztile(static_cast<Z *>(p.A), p.lda, nb, i, k);
  const Z *Tt = zt_ptr(static_cast<Z *>(p.T), p.P, ib, nb, i, k, 1);
  const int mb = zrows(p, i), K = zcols(p, k), nblk = (K + ib - 1) / ib;
  for (int cs = 0; cs < ncols; cs += kZChunk) {
    const int w = min(kZChunk, ncols - cs);
    Z *b1 = c1ptr + static_cast<int64_t>(cs) * ldc, *b2 = c2ptr + static_cast<int64_t>(cs) * ldc;
    zload(s.C1, s.ldv, b1, ldc, K, w, [](int, int) { return true; });
    zload(s.C, s.ldv, b2, ldc, mb, w, [](int, int) { return true; });
    for (int bb = 0; bb < nblk; ++bb) {
      const int b = adjoint ? bb : nblk - 1 - bb;
      const int c0 = b * ib, kb = min(ib, K - c0), rb = ts ? mb : min(c0 + kb, mb);
      __syncthreads();
      zload(s.V, s.ldv, vt + static_cast<int64_t>(c0) * p.lda, p.lda, rb, kb,
            [c0, ts](int r, int c) { return ts || r <= c0 + c; });
      zload(s.T, s.ldt, Tt + static_cast<int64_t>(c0) * ib, ib, kb, kb, [](int, int) { return true; });
      __syncthreads();
      zapply(s.C, s.ldv, rb, s.C1 + c0, s.ldv, w, s, kb, adjoint);
    }
    zstore(b1, ldc, s.C1, s.ldv, K, w);
    zstore(b2, ldc, s.C, s.ldv, mb, w);
    __syncthreads();
  }
}

// Bounded wait until the task's counter reaches zero; false when this CTA must stop.
__device__ bool zwait_ready(const ExecParams &p, int t) {
  const int32_t *cnt = p.counters + t;
  const uint64_t t0 = zglobaltimer();
  const uint64_t limit = static_cast<uint64_t>(p.wait_limit_ns);
  for (uint64_t it = 0;; ++it) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
    if (v <= 0) return true;
    int st;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(st) : "l"(p.status) : "memory");
    if (st != 0) return false;
    if (zglobaltimer() - t0 > limit || it > (limit >> 4) + 1000000ull) {
      atomicCAS(p.status, 0, kStatusTimeout | (min(t, (1 << 23) - 1) << 8));
      return false;
    }
    __nanosleep(64);
  }
}

__global__ void __launch_bounds__(kZThreads, 1) zexecutor_kernel(ExecParams p) {
  extern __shared__ __align__(16) unsigned char zsmem_raw[];
  __shared__ int s_task, s_stop;
  ZSmem s = zcarve(zsmem_raw, p.nb, p.ib);
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(p.next, 1);
      int st;
      asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(st) : "l"(p.status) : "memory");
      int stop = t >= p.ntask || st != 0;
      if (!stop && !zwait_ready(p, t)) stop = 1;
      s_task = t;
      s_stop = stop;
    }
    __syncthreads();
    if (s_stop) break;
    const int t = s_task;
    const Task task = p.tasks[t];
    Z *A = static_cast<Z *>(p.A);
    Z *B = reinterpret_cast<Z *>(p.B);
    const int nb = p.nb;
    switch (task.kind) {
      case kGeqrt: ztask_geqrt(p, s, task.i, task.k); break;
      case kTtqrt: ztask_pair_qrt(p, s, task.i, task.piv, task.k, false); break;
      case kTsqrt: ztask_pair_qrt(p, s, task.i, task.piv, task.k, true); break;
      case kUnmqr:
        ztask_unmqr(p, s, task.i, task.k, ztile(A, p.lda, nb, task.i, task.j), p.lda, zcols(p, task.j), true);
        break;
      case kTtmqr:
      case kTsmqr:
        ztask_pair_mqr(p, s, task.i, task.k, ztile(A, p.lda, nb, task.piv, task.j), ztile(A, p.lda, nb, task.i, task.j),
                       p.lda, zcols(p, task.j), true, task.kind == kTsmqr);
        break;
      case kUnmqrB:
        ztask_unmqr(p, s, task.i, task.k, B + static_cast<int64_t>(task.i) * nb, p.ldb, static_cast<int>(p.nrhs),
                    p.trans == 0);
        break;
      case kTtmqrB:
      case kTsmqrB:
        ztask_pair_mqr(p, s, task.i, task.k, B + static_cast<int64_t>(task.piv) * nb,
                       B + static_cast<int64_t>(task.i) * nb, p.ldb, static_cast<int>(p.nrhs), p.trans == 0,
                       task.kind == kTsmqrB);
        break;
      default:
        break;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      for (int e = p.succ_ptr[t]; e < p.succ_ptr[t + 1]; ++e) atomicSub(p.counters + p.succ_idx[e], 1);
    }
  }
}

// R X = B for the n x n upper-triangular complex R (lda), B n x nrhs (ldb): one CTA per
// right-hand side, 32-row blocks from the bottom: warp 0 solves the diagonal block by
// substitution, then every thread subtracts the block's contribution from the rows above.
__global__ void __launch_bounds__(kZThreads) ztrsm_kernel(int64_t n, const Z *R, int64_t lda, Z *B, int64_t ldb) {
  Z *b = B + static_cast<int64_t>(blockIdx.x) * ldb;
  __shared__ Z xs[32];
  const int64_t nblk = (n + 31) / 32;
  for (int64_t blk = nblk - 1; blk >= 0; --blk) {
    const int64_t r0 = blk * 32;
    const int rows = static_cast<int>(n - r0 < 32 ? n - r0 : 32);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      Z x = lane < rows ? b[r0 + lane] : Z{0.0, 0.0};
      for (int j = rows - 1; j >= 0; --j) {
        // x_j = (b_j - sum_{c > j} R(j, c) x_c) / R(j, j): lane j finishes, then broadcasts
        if (lane == j) {
          const Z d = R[(r0 + j) + (r0 + j) * lda];
          const double dd = abs2(d);
          x = x * Z{d.re / dd, -d.im / dd};
        }
        const Z xj{__shfl_sync(0xffffffffu, x.re, j), __shfl_sync(0xffffffffu, x.im, j)};
        if (lane < j) x = x - R[(r0 + lane) + (r0 + j) * lda] * xj;
      }
      if (lane < rows) xs[lane] = x;
    }
    __syncthreads();
    if (threadIdx.x < rows) b[r0 + threadIdx.x] = xs[threadIdx.x];
    for (int64_t r = threadIdx.x; r < r0; r += kZThreads) {
      Z acc{0.0, 0.0};
      for (int c = 0; c < rows; ++c) acc = acc + R[r + (r0 + c) * lda] * xs[c];
      b[r] = b[r] - acc;
    }
    __syncthreads();
  }
}

}  // namespace

size_t zexecutor_smem_bytes(int nb, int ib) {
  const size_t b = zsmem_bytes(nb, ib);
  return b <= 227 * 1024 ? b : 0;
}

int zexec_launch(const ExecParams &p, void *stream) {
  const size_t smem = zsmem_bytes(p.nb, p.ib);
  cudaError_t e = cudaFuncSetAttribute(zexecutor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return static_cast<int>(e);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zexecutor_kernel, kZThreads, smem);
  if (e != cudaSuccess) return static_cast<int>(e);
  int grid = nsm * (per_sm < 1 ? 1 : per_sm);
  if (grid > p.ntask) grid = p.ntask;
  if (grid < 1) grid = 1;
  zexecutor_kernel<<<grid, kZThreads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  count_launch();
  return static_cast<int>(cudaGetLastError());
}

int zexec_slots(int nb, int ib) {
  const size_t smem = zsmem_bytes(nb, ib);
  if (cudaFuncSetAttribute(zexecutor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
      cudaSuccess)
    return 0;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zexecutor_kernel, kZThreads, smem) != cudaSuccess)
    return 0;
  return nsm * (per_sm < 1 ? 1 : per_sm);
}

int launch_ztrsm(int64_t n, const void *R, int64_t lda, void *B, int64_t ldb, int64_t nrhs, void *stream) {
  if (nrhs <= 0) return 0;
  ztrsm_kernel<<<static_cast<unsigned>(nrhs), kZThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      n, static_cast<const Z *>(R), lda, static_cast<Z *>(B), ldb);
  count_launch();
  return static_cast<int>(cudaGetLastError());
}

}  // namespace tqr
