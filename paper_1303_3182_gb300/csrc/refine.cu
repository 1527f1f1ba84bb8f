// FP64 iterative refinement of a least-squares solution with a low-precision tiled QR.
//
// The tensor-core factorization gives R with a backward error far above FP64 rounding.
// Each outer step computes, in FP64, the residual r = b - A x of the current solution
// and its optimality ||A^T r|| / (||A||_F ||r||); it stops when that is <= tol, else it
// solves min || A dx - r || with LSQR (Paige & Saunders, ACM TOMS 8(1), 1982)
// right-preconditioned by the computed R (y = R dx, operator A R^{-1}) and sets
// x += dx.  Restarting from the true residual makes the stopping test independent of
// LSQR's internal estimates, which drift when the preconditioner is weak.  A products,
// residuals, the Krylov vectors and every scalar recurrence are FP64; the triangular
// solves read the low-precision R (FP32) and compute in FP64; the two products with A inside
// an LSQR iteration use A split into FP32 pairs with double-float arithmetic (below).  All
// scalar state lives in device memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tqr_internal.h"

namespace tqr {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double per thread; result valid in thread 0.
__device__ double block_sum(double v) {
  __shared__ double part[kT / 32];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < kT / 32 ? part[threadIdx.x] : 0.0;
    s = warp_sum_d(s);
  }
  __syncthreads();
  return s;
}

// Y(:, r) = sy(r) * Y(:, r) + A X(:, r)  for r < nrhs, rows [row0, row0 + 256) of this CTA,
// columns [c0, c1) of A; partial sums are added atomically.  sy(r) is applied by the CTAs
// of the first column chunk only.  ssq(r) += ||Y(:, r)||^2 is NOT formed here.
__global__ void gemv_n(int64_t m, int64_t n, const double *A, int64_t lda, const double *X, int64_t ldx,
                       double *Y, int64_t ldy, int nrhs, int64_t chunk) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x;
  const int64_t c0 = blockIdx.y * chunk, c1 = c0 + chunk < n ? c0 + chunk : n;
  if (i >= m) return;
  for (int r = 0; r < nrhs; ++r) {
    const double *x = X + r * ldx;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t j = c0;
    for (; j + 4 <= c1; j += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(A[i + (j + u) * lda], x[j + u], acc[u]);
    }
    for (; j < c1; ++j) acc[0] = fma(A[i + j * lda], x[j], acc[0]);
    atomicAdd(Y + i + r * ldy, (acc[0] + acc[1]) + (acc[2] + acc[3]));
  }
}

// Y(j, r) = sum_i A(i, j) X(i, r) * scale(r): one warp per column j.
__global__ void gemv_t(int64_t m, int64_t n, const double *A, int64_t lda, const double *X, int64_t ldx,
                       double *Y, int64_t ldy, int nrhs, const double *scale) {
  const int warp = (blockIdx.x * kT + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const double *col = A + warp * lda;
  for (int r = 0; r < nrhs; ++r) {
    const double *x = X + r * ldx;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int64_t i = lane;
    for (; i + 96 < m; i += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(col[i + 32 * u], x[i + 32 * u], acc[u]);
    }
    for (; i < m; i += 32) acc[0] = fma(col[i], x[i], acc[0]);
    const double s = warp_sum_d((acc[0] + acc[1]) + (acc[2] + acc[3]));
    if (lane == 0) Y[warp + r * ldy] = s * (scale ? scale[r] : 1.0);
  }
}

// ---- inner-solve products with A held as FP32 pairs ---------------------------------
// The LSQR correction solve needs A v and A^T u only to the accuracy of a correction, but
// its FP64 GEMVs are bound by this GPU's FP64 rate (m n DFMA, about twice the time the
// 8 m n bytes of A take to stream).  For them A is split once per solve into FP32 pairs
// a = a_hi + a_lo (a_lo the FP32 rounding of a - a_hi, 8 bytes per entry like the FP64
// matrix), the vector likewise, and each product is formed in double-float FP32 arithmetic:
// a x = a_hi x_hi (exact as p + e by an FMA) + (a_hi x_lo + a_lo x_hi), the sum kept as an
// unevaluated pair with Knuth's TwoSum - about 2^-47 relative per term, against 2^-53 for
// FP64, with FP32 instructions only.  The residual r = b - A x and A^T r of the outer
// refinement stay in FP64.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ void df_acc(DF &s, float ah, float al, float xh, float xl) {
  const float p = ah * xh;
  const float e = fmaf(ah, xh, -p) + fmaf(ah, xl, al * xh);
  const float t = s.hi + p;
  const float bb = t - s.hi;
  const float err = (s.hi - (t - bb)) + (p - bb);
  s.hi = t;
  s.lo += err + e;
}

__device__ __forceinline__ DF df_sum(DF a, DF b) {
  const float t = a.hi + b.hi;
  const float bb = t - a.hi;
  const float err = (a.hi - (t - bb)) + (b.hi - bb);
  return DF{t, a.lo + b.lo + err};
}

// One pass over A before the factorization: F = fl32(A) (the matrix the tensor-core
// factorization overwrites), P = A as FP32 pairs (column-major, ld m; hi is F's value, lo
// the FP32 rounding of a - hi; split_pair, in integer instructions) and ||A||_F^2 added to
// *anorm2, accumulated per thread in double-float (hi^2 exactly as p + e, plus 2 hi lo;
// about 2^-44 relative, ample for the stopping tests that use it).  Four columns per
// thread step, so that four loads are in flight before the first store.
__global__ void __launch_bounds__(kT) prepare_a(int64_t m, int64_t n, const double *__restrict__ A, int64_t lda,
                                                float *__restrict__ F, int64_t ldf, float2 *__restrict__ P,
                                                double *anorm2) {
  DF acc{0.f, 0.f};
  const int64_t i0 = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x;
  const int64_t istep = static_cast<int64_t>(gridDim.x) * kT;
  for (int64_t j0 = static_cast<int64_t>(blockIdx.y) * 4; j0 < n; j0 += static_cast<int64_t>(gridDim.y) * 4) {
    for (int64_t i = i0; i < m; i += istep) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = j0 + u < n ? A[i + (j0 + u) * lda] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (j0 + u < n) {
          float hi, lo;
          split_pair(v[u], hi, lo);
          F[i + (j0 + u) * ldf] = hi;
          P[i + (j0 + u) * m] = make_float2(hi, lo);
          const float pp = hi * hi;
          const float t = acc.hi + pp;
          const float bb = t - acc.hi;
          const float err = (acc.hi - (t - bb)) + (pp - bb);
          acc.lo += err + fmaf(hi, hi, -pp) + 2.f * hi * lo;
          acc.hi = t;
        }
      }
    }
  }
  const double s = block_sum(static_cast<double>(acc.hi) + static_cast<double>(acc.lo));
  if (threadIdx.x == 0) atomicAdd(anorm2, s);
}

// Xp(:, r) = pair split of X(:, r), r < nrhs.
__global__ void split_vec(int64_t len, const double *X, int64_t ldx, float2 *Xp, int nrhs) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < len;
       i += static_cast<int64_t>(gridDim.x) * kT) {
    const double a = X[i + r * ldx];
    const float hi = static_cast<float>(a);
    Xp[i + r * len] = make_float2(hi, static_cast<float>(a - static_cast<double>(hi)));
  }
}

// Y(:, r) += A X(:, r) with A and X as pairs (rows of this CTA, columns [c0, c1)); four
// columns per step with their own accumulators, so that four loads of A are in flight.
__global__ void __launch_bounds__(kT) gemv_n_pairs(int64_t m, int64_t n, const float2 *__restrict__ P,
                                                   const float2 *__restrict__ Xp, double *Y, int64_t ldy, int nrhs,
                                                   int64_t chunk) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x;
  const int64_t c0 = blockIdx.y * chunk, c1 = c0 + chunk < n ? c0 + chunk : n;
  if (i >= m) return;
  for (int r = 0; r < nrhs; ++r) {
    const float2 *x = Xp + r * n;
    DF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int64_t j = c0;
    for (; j + 4 <= c1; j += 4) {
      float2 a[4], xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = P[i + (j + u) * m];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = x[j + u];
#pragma unroll
      for (int u = 0; u < 4; ++u) df_acc(s[u], a[u].x, a[u].y, xv[u].x, xv[u].y);
    }
    for (; j < c1; ++j) {
      const float2 a0 = P[i + j * m], x0 = x[j];
      df_acc(s[0], a0.x, a0.y, x0.x, x0.y);
    }
    const DF t = df_sum(df_sum(s[0], s[1]), df_sum(s[2], s[3]));
    atomicAdd(Y + i + r * ldy, static_cast<double>(t.hi) + static_cast<double>(t.lo));
  }
}

// Y(j, r) = scale(r) sum_i A(i, j) U(i, r) with A and U as pairs: one warp per column j.
// Every column reads all of U, so a CTA (kT / 32 columns) stages U through shared memory
// in chunks of kTChunk rows, read from L2 once per CTA instead of once per warp; each lane
// then takes two rows per float4 of A (m even and 16-byte aligned pair arrays: vec), else
// one row per load.
constexpr int kTChunk = 4096;
__global__ void __launch_bounds__(kT) gemv_t_pairs(int64_t m, int64_t n, const float2 *__restrict__ P,
                                                   const float2 *__restrict__ Up, double *Y, int64_t ldy, int nrhs,
                                                   const double *scale, int vec) {
  __shared__ __align__(16) float2 us[kTChunk];
  const int lane = threadIdx.x & 31;
  const int64_t col = (static_cast<int64_t>(blockIdx.x) * kT + threadIdx.x) >> 5;
  const bool active = col < n;
  const float2 *cp = P + (active ? col : 0) * m;
  for (int r = 0; r < nrhs; ++r) {
    const float2 *u = Up + r * m;
    DF s[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int64_t r0 = 0; r0 < m; r0 += kTChunk) {
      const int len = static_cast<int>(m - r0 < kTChunk ? m - r0 : kTChunk);
      __syncthreads();  // the previous chunk is no longer read
      if (vec) {
        const float4 *u4 = reinterpret_cast<const float4 *>(u + r0);
        for (int x = threadIdx.x; x < len / 2; x += kT) reinterpret_cast<float4 *>(us)[x] = u4[x];
        if ((len & 1) && threadIdx.x == 0) us[len - 1] = u[r0 + len - 1];
      } else {
        for (int x = threadIdx.x; x < len; x += kT) us[x] = u[r0 + x];
      }
      __syncthreads();
      if (!active) continue;
      const float2 *c = cp + r0;
      int i = 0;
      if (vec) {
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
        const float4 *w4 = reinterpret_cast<const float4 *>(us);
#pragma unroll 2
        for (; i + 256 <= len; i += 256) {
          float4 a[4], w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a[q] = c4[(i >> 1) + 32 * q + lane];
#pragma unroll
          for (int q = 0; q < 4; ++q) w[q] = w4[(i >> 1) + 32 * q + lane];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            df_acc(s[q], a[q].x, a[q].y, w[q].x, w[q].y);
            df_acc(s[q], a[q].z, a[q].w, w[q].z, w[q].w);
          }
        }
      }
      for (i += lane; i < len; i += 32) {
        const float2 a0 = c[i], u0 = us[i];
        df_acc(s[0], a0.x, a0.y, u0.x, u0.y);
      }
    }
    if (!active) continue;
    DF t = df_sum(df_sum(s[0], s[1]), df_sum(s[2], s[3]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const DF v{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)};
      t = df_sum(t, v);
    }
    if (lane == 0)
      Y[col + r * ldy] = (static_cast<double>(t.hi) + static_cast<double>(t.lo)) * (scale ? scale[r] : 1.0);
  }
}

// LSQR scalar state of one right-hand side (double-buffered by iteration parity).
struct LsqrScalars {
  double alpha, beta, rhobar, phibar, anorm2, conv;
};

// Residual start: U = B - A X0 (U pre-filled with B), then per rhs beta = ||U||.
__global__ void colnorm(int64_t rows, const double *U, int64_t ldu, double *out, int nrhs) {
  const int r = blockIdx.y;
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < rows;
       i += static_cast<int64_t>(gridDim.x) * kT) {
    const double v = U[i + r * ldu];
    s += v * v;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(out + r, s);
}

// v(:, r) = z(:, r) - beta(r) * vold(:, r) when vold given, else z; per-rhs ||v||^2.
__global__ void axpy_norm(int64_t n, double *Z, int64_t ldz, const double *Vold, int64_t ldv, const double *beta,
                          double *ssq, int nrhs) {
  const int r = blockIdx.y;
  double s = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kT) {
    double z = Z[i + r * ldz];
    if (Vold) z -= beta[r] * Vold[i + r * ldv];
    Z[i + r * ldz] = z;
    s += z * z;
  }
  s = block_sum(s);
  if (threadIdx.x == 0) atomicAdd(ssq + r, s);
}


// One fused scalar + vector step after alpha_new^2 (ssq_a) and beta_new (stored) are known:
//   alpha = sqrt(ssq_a); v = z / alpha; rho = hypot(rhobar, beta); c = rhobar/rho;
//   s = beta/rho; theta = s*alpha; rhobar' = -c*alpha; phi = c*phibar; phibar' = s*phibar;
//   y += (phi/rho) w;  w = v - (theta/rho) w
__global__ void lsqr_step(int64_t n, double *Z, int64_t ldz, double *V, double *W, double *Y, int64_t ld,
                          const double *ssq_a, const double *beta_new, const LsqrScalars *in, LsqrScalars *outs,
                          int nrhs, double tol) {
  const int r = blockIdx.y;
  const LsqrScalars st = in[r];
  const double alpha = sqrt(ssq_a[r]);
  const double beta = beta_new[r];
  const double rho = hypot(st.rhobar, beta);
  const double c = st.rhobar / rho, s = beta / rho;
  const double theta = s * alpha;
  const double phi = c * st.phibar;
  const double inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
  const double f_y = phi / rho, f_w = theta / rho;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kT) {
    const double v = Z[i + r * ldz] * inv_alpha;
    const double w = W[i + r * ld];
    V[i + r * ld] = v;
    Y[i + r * ld] += f_y * w;
    W[i + r * ld] = v - f_w * w;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    LsqrScalars o;
    o.alpha = alpha;
    o.beta = beta;
    o.rhobar = -c * alpha;
    o.phibar = s * st.phibar;
    o.anorm2 = st.anorm2 + alpha * alpha + beta * beta;
    // ||(A M)^T r|| / ||r|| = alpha |c| (Paige & Saunders); since A^T r = R^T (A M)^T r
    // and ||R|| ~ ||A||, this bounds ||A^T r|| / (||A|| ||r||) of the unpreconditioned
    // problem, the quantity the FP64 target is stated for
    o.conv = alpha * fabs(c);
    outs[r] = o;
  }
}

// Start of LSQR: beta = ||u||, alpha = ||z|| known; v = z/alpha, w = v, y = 0.
__global__ void lsqr_init(int64_t n, double *Z, int64_t ldz, double *V, double *W, double *Y, int64_t ld,
                          const double *ssq_a, const double *ssq_b, LsqrScalars *outs, int nrhs) {
  const int r = blockIdx.y;
  const double alpha = sqrt(ssq_a[r]), beta = sqrt(ssq_b[r]);
  const double inv_alpha = alpha > 0.0 ? 1.0 / alpha : 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kT) {
    const double v = Z[i + r * ldz] * inv_alpha;
    V[i + r * ld] = v;
    W[i + r * ld] = v;
    Y[i + r * ld] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    LsqrScalars o;
    o.alpha = alpha;
    o.beta = beta;
    o.rhobar = alpha;
    o.phibar = beta;
    o.anorm2 = alpha * alpha;
    o.conv = beta > 0.0 ? 1.0 : 0.0;
    outs[r] = o;
  }
}

// U = U * (-alpha / beta_old) ... prepares u' accumulation: U_new = A t - alpha * u,
// with u = U_old / beta_old: scale U_old in place by -alpha/beta_old before the atomics.
__global__ void scale_u(int64_t m, double *U, int64_t ldu, const LsqrScalars *st, int nrhs) {
  const int r = blockIdx.y;
  const double f = st[r].beta > 0.0 ? -st[r].alpha / st[r].beta : 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * kT)
    U[i + r * ldu] *= f;
}

// inv[r] = 1 / sqrt(ssq[r]); out_beta[r] = sqrt(ssq[r])
__global__ void finish_norm(const double *ssq, double *inv, double *out_beta, int nrhs) {
  const int r = threadIdx.x;
  if (r < nrhs) {
    const double b = sqrt(ssq[r]);
    inv[r] = b > 0.0 ? 1.0 / b : 0.0;
    out_beta[r] = b;
  }
}

__global__ void add_into(int64_t n, double *X, int64_t ldx, const double *D, int64_t ldd, int nrhs) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kT)
    X[i + r * ldx] += D[i + r * ldd];
}

// D(:, r) = f * S(:, r)
__global__ void copy_scaled(int64_t n, double *D, int64_t ldd, const double *S, int64_t lds, double f, int nrhs) {
  const int r = blockIdx.y;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(kT) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kT)
    D[i + r * ldd] = f * S[i + r * lds];
}

dim3 vgrid(int64_t len, int nrhs) {
  int64_t b = (len + kT - 1) / kT;
  if (b > 1024) b = 1024;
  return dim3(static_cast<unsigned>(b), static_cast<unsigned>(nrhs));
}

}  // namespace

// Workspace (doubles).  Fixed part, set up once per least-squares call: ||A||_F^2 (padded to
// two), A as FP32 pairs (one double's worth per entry), the inverses of R's 64 x 64
// diagonal blocks and the preconditioner's set-up.  Per block of right-hand sides: U (m)
// and V, W, Y, Z, Tt (n) per right-hand side, the scalar arrays, two LSQR state sets, and
// the pair splits of one n- and one m-vector per right-hand side (16-byte aligned).
namespace {
struct FixedLayout {
  double *anorm2;
  float2 *Apair;
  double *Dinv, *Pw;
  double *end;
};
FixedLayout fixed_layout(int64_t m, int64_t n, double *work) {
  FixedLayout l;
  l.anorm2 = work;
  l.Apair = reinterpret_cast<float2 *>(work + 2);
  l.Dinv = work + 2 + static_cast<size_t>(m) * n;
  l.Pw = l.Dinv + static_cast<size_t>((n + 63) / 64) * 64 * 64;
  l.end = l.Pw + precond_work_doubles(n, false);
  return l;
}
size_t even(size_t x) { return (x + 1) & ~static_cast<size_t>(1); }
}  // namespace

size_t lsqr_work_doubles(int64_t m, int64_t n, int nrhs) {
  const size_t nblk = static_cast<size_t>((n + 63) / 64);
  const size_t fixed = 2 + static_cast<size_t>(m) * n + nblk * 64 * 64 + precond_work_doubles(n, false);
  const size_t per = static_cast<size_t>(nrhs) * (m + 5 * n) + 8 * static_cast<size_t>(nrhs) + 8 +
                     2 * (sizeof(LsqrScalars) / sizeof(double)) * static_cast<size_t>(nrhs) +
                     static_cast<size_t>(nrhs) * (m + n) + 8;
  return fixed + per;
}

int lsqr_prepare(int64_t m, int64_t n, const double *A, int64_t lda, float *F, int64_t ldf, double *work,
                 void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const FixedLayout fl = fixed_layout(m, n, work);
  cudaError_t e = cudaMemsetAsync(fl.anorm2, 0, sizeof(double), st);
  if (e != cudaSuccess) return static_cast<int>(e);
  const int64_t gx = (m + kT - 1) / kT;
  const int64_t gy = (n + 3) / 4;
  const dim3 grid(static_cast<unsigned>(gx < 128 ? gx : 128), static_cast<unsigned>(gy < 64 ? gy : 64));
  prepare_a<<<grid, kT, 0, st>>>(m, n, A, lda, F, ldf, fl.Apair, fl.anorm2);
  count_launch();
  return static_cast<int>(cudaGetLastError());
}

int lsqr_refine(int64_t m, int64_t n, int nrhs, const double *A, int64_t lda, const float *R, int64_t ldr,
                const double *B, int64_t ldb, double *X, int64_t ldx, double tol, int max_iter, int *iters_out,
                bool setup, bool x_zero, double *work, int32_t *flags, int32_t *status, int64_t wait_limit_ns,
                void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const FixedLayout fl = fixed_layout(m, n, work);
  const float2 *Apair = fl.Apair;
  double *Dinv = fl.Dinv, *Pw = fl.Pw;
  double *U = fl.end;
  double *V = U + static_cast<size_t>(m) * nrhs;
  double *W = V + static_cast<size_t>(n) * nrhs;
  double *Y = W + static_cast<size_t>(n) * nrhs;
  double *Z = Y + static_cast<size_t>(n) * nrhs;
  double *Tt = Z + static_cast<size_t>(n) * nrhs;
  double *ssq_a = Tt + static_cast<size_t>(n) * nrhs;  // [nrhs]
  double *ssq_b = ssq_a + nrhs;                         // [nrhs]
  double *inv_b = ssq_b + nrhs;                         // [nrhs]
  double *betas = inv_b + nrhs;                         // [nrhs]
  double *anorm2 = betas + nrhs;                        // [1]  ||A||_F^2 (copied from the fixed part)
  double *eta2 = anorm2 + 1;                            // [nrhs] ||A^T u||^2, u = r / ||r||
  LsqrScalars *sc = reinterpret_cast<LsqrScalars *>(eta2 + nrhs + ((nrhs + 1) & 1));  // [2][nrhs]
  double *bn2 = reinterpret_cast<double *>(sc + 2 * nrhs);                         // [nrhs] ||b||^2
  double *xn2 = bn2 + nrhs;                                                       // [nrhs] ||x||^2
  // the pair splits of the inner products' vectors, 16-byte aligned for float4 loads
  const size_t pv = even(static_cast<size_t>((xn2 + nrhs) - work));
  float2 *Vpair = reinterpret_cast<float2 *>(work + pv);                           // n x nrhs
  float2 *Upair = reinterpret_cast<float2 *>(work + even(pv + static_cast<size_t>(n) * nrhs));  // m x nrhs
  const int vec = (m % 2 == 0) ? 1 : 0;
  const int64_t chunk = 512;
  const dim3 ggrid(static_cast<unsigned>((m + kT - 1) / kT), static_cast<unsigned>((n + chunk - 1) / chunk));
  const unsigned tgrid = static_cast<unsigned>((n * 32 + kT - 1) / kT);
  cudaError_t e = cudaSuccess;
  int rc = 0;
#define TQR_CK(x)                                       \
  do {                                                  \
    e = (x);                                            \
    if (e != cudaSuccess) return static_cast<int>(e);   \
  } while (0)
#define TQR_CKL()                                       \
  do {                                                  \
    count_launch();                                     \
    e = cudaGetLastError();                             \
    if (e != cudaSuccess) return static_cast<int>(e);   \
  } while (0)
  TQR_CK(cudaMemcpyAsync(anorm2, fl.anorm2, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (setup) {
    if ((rc = launch_diag_inverse(n, R, ldr, false, Dinv, stream)) != 0) return rc;
    if ((rc = precond_setup(n, R, ldr, false, Dinv, Pw, stream)) != 0) return rc;
  }
  // R^{-1} and R^{-T} applied with the inverses of R's 1024 x 1024 diagonal blocks
  auto solve_r = [&](double *Vec, bool lower_t) -> int {
    return precond_solve(n, R, ldr, false, Pw, Vec, n, nrhs, flags, status, wait_limit_ns, stream, lower_t);
  };
  std::vector<double> host_eta(nrhs + 1), host_rn2(nrhs), host_xn2(nrhs), host_bn2(nrhs), thr(nrhs);
  std::vector<LsqrScalars> host(nrhs);
  TQR_CK(cudaMemsetAsync(bn2, 0, sizeof(double) * nrhs, st));
  colnorm<<<vgrid(m, nrhs), kT, 0, st>>>(m, B, ldb, bn2, nrhs);
  TQR_CKL();
  TQR_CK(cudaMemcpyAsync(host_bn2.data(), bn2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
  int total_it = 0;
  bool converged = false;
  double prev_eta = 1e300, prev_omega = 1e300;
  const bool debug = std::getenv("TQR_DEBUG_REFINE") != nullptr;
  const int max_outer = 12;
  for (int outer = 0; outer < max_outer; ++outer) {
    // FP64 residual of the current solution: u = r = B - A X, beta = ||r||
    TQR_CK(cudaMemcpy2DAsync(U, m * sizeof(double), B, ldb * sizeof(double), m * sizeof(double), nrhs,
                             cudaMemcpyDeviceToDevice, st));
    if (outer > 0 || !x_zero) {  // a zero start has the residual B itself
      copy_scaled<<<vgrid(n, nrhs), kT, 0, st>>>(n, Tt, n, X, ldx, -1.0, nrhs);
      TQR_CKL();
      gemv_n<<<ggrid, kT, 0, st>>>(m, n, A, lda, Tt, n, U, m, nrhs, chunk);
      TQR_CKL();
    }
    TQR_CK(cudaMemsetAsync(ssq_a, 0, sizeof(double) * 2 * nrhs, st));
    TQR_CK(cudaMemsetAsync(eta2, 0, sizeof(double) * nrhs, st));
    colnorm<<<vgrid(m, nrhs), kT, 0, st>>>(m, U, m, ssq_b, nrhs);
    TQR_CKL();
    finish_norm<<<1, 64, 0, st>>>(ssq_b, inv_b, betas, nrhs);
    TQR_CKL();
    // A^T u in FP64 and the optimality ||A^T r|| / (||A||_F ||r||) of the current X
    gemv_t<<<tgrid, kT, 0, st>>>(m, n, A, lda, U, m, Z, n, nrhs, inv_b);
    TQR_CKL();
    axpy_norm<<<vgrid(n, nrhs), kT, 0, st>>>(n, Z, n, nullptr, n, nullptr, eta2, nrhs);
    TQR_CKL();
    // ||x|| of the current solution for the backward error of a consistent system
    TQR_CK(cudaMemsetAsync(xn2, 0, sizeof(double) * nrhs, st));
    colnorm<<<vgrid(n, nrhs), kT, 0, st>>>(n, X, ldx, xn2, nrhs);
    TQR_CKL();
    TQR_CK(cudaMemcpyAsync(host_eta.data(), anorm2, sizeof(double) * (nrhs + 1), cudaMemcpyDeviceToHost, st));
    TQR_CK(cudaMemcpyAsync(host_rn2.data(), ssq_b, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    TQR_CK(cudaMemcpyAsync(host_xn2.data(), xn2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    TQR_CK(cudaStreamSynchronize(st));
    // A right-hand side is done when X is least-squares optimal to tol (||A^T r|| small)
    // or, for a consistent system, when the normwise backward error
    // ||r|| / (||A||_F ||x|| + ||b||) is below tol.
    const double anorm = sqrt(host_eta[0]);
    double worst_eta = 0.0, worst_omega = 0.0;
    bool all_done = true;
    for (int r = 0; r < nrhs; ++r) {
      const double eta = sqrt(host_eta[1 + r] / host_eta[0]);
      const double scale = anorm * sqrt(host_xn2[r]) + sqrt(host_bn2[r]);
      const double omega = scale > 0.0 ? sqrt(host_rn2[r]) / scale : 0.0;
      worst_eta = fmax(worst_eta, eta);
      worst_omega = fmax(worst_omega, omega);
      all_done = all_done && (!(eta > tol) || !(omega > tol));
      thr[r] = 0.1 * tol * scale;
    }
    if (debug)
      std::fprintf(stderr, "[tqr refine] outer %d: optimality %.3e backward error %.3e after %d LSQR iterations\n",
                   outer, worst_eta, worst_omega, total_it);
    if (all_done) {
      converged = true;
      break;
    }
    // an outer step that halves neither the optimality nor the backward error has reached
    // the level FP64 rounding allows for this problem (as LAPACK's refinement stops):
    // converged.  (A least-squares problem stalls on the optimality; a consistent system,
    // whose optimality ratio is rounding noise, on the backward error.)
    if (worst_eta > 0.5 * prev_eta && worst_omega > 0.5 * prev_omega) {
      converged = true;
      break;
    }
    if (total_it >= max_iter) break;
    prev_eta = worst_eta;
    prev_omega = worst_omega;
    // LSQR on min || (A R^-1) y - r ||, then X += R^{-1} y
    if ((rc = solve_r(Z, true)) != 0) return rc;
    axpy_norm<<<vgrid(n, nrhs), kT, 0, st>>>(n, Z, n, nullptr, n, nullptr, ssq_a, nrhs);
    TQR_CKL();
    lsqr_init<<<vgrid(n, nrhs), kT, 0, st>>>(n, Z, n, V, W, Y, n, ssq_a, ssq_b, sc, nrhs);
    TQR_CKL();
    for (int it = 0; it < 64 && total_it < max_iter; ++it, ++total_it) {
      LsqrScalars *cur = sc + (it & 1) * nrhs, *nxt = sc + ((it + 1) & 1) * nrhs;
      TQR_CK(cudaMemcpyAsync(Tt, V, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
      if ((rc = solve_r(Tt, false)) != 0) return rc;
      scale_u<<<vgrid(m, nrhs), kT, 0, st>>>(m, U, m, cur, nrhs);
      TQR_CKL();
      split_vec<<<vgrid(n, nrhs), kT, 0, st>>>(n, Tt, n, Vpair, nrhs);
      TQR_CKL();
      gemv_n_pairs<<<ggrid, kT, 0, st>>>(m, n, Apair, Vpair, U, m, nrhs, chunk);
      TQR_CKL();
      TQR_CK(cudaMemsetAsync(ssq_a, 0, sizeof(double) * 2 * nrhs, st));
      colnorm<<<vgrid(m, nrhs), kT, 0, st>>>(m, U, m, ssq_b, nrhs);
      TQR_CKL();
      finish_norm<<<1, 64, 0, st>>>(ssq_b, inv_b, betas, nrhs);
      TQR_CKL();
      split_vec<<<vgrid(m, nrhs), kT, 0, st>>>(m, U, m, Upair, nrhs);
      TQR_CKL();
      gemv_t_pairs<<<tgrid, kT, 0, st>>>(m, n, Apair, Upair, Z, n, nrhs, inv_b, vec);
      TQR_CKL();
      if ((rc = solve_r(Z, true)) != 0) return rc;
      axpy_norm<<<vgrid(n, nrhs), kT, 0, st>>>(n, Z, n, V, n, betas, ssq_a, nrhs);
      TQR_CKL();
      lsqr_step<<<vgrid(n, nrhs), kT, 0, st>>>(n, Z, n, V, W, Y, n, ssq_a, betas, cur, nxt, nrhs, tol);
      TQR_CKL();
      TQR_CK(cudaMemcpyAsync(host.data(), nxt, sizeof(LsqrScalars) * nrhs, cudaMemcpyDeviceToHost, st));
      TQR_CK(cudaStreamSynchronize(st));
      // LSQR's two stopping rules per right-hand side: the normal-equation estimate
      // (inconsistent systems) or the residual estimate phibar against the backward-error
      // threshold of the outer solution (consistent systems)
      bool inner_done = true;
      for (int r = 0; r < nrhs; ++r)
        inner_done = inner_done && (!(host[r].conv > 0.1 * tol) || !(host[r].phibar > thr[r]));
      if (inner_done) {
        ++total_it;
        break;
      }
    }
    TQR_CK(cudaMemcpyAsync(Tt, Y, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, st));
    if ((rc = solve_r(Tt, false)) != 0) return rc;
    add_into<<<vgrid(n, nrhs), kT, 0, st>>>(n, X, ldx, Tt, n, nrhs);
    TQR_CKL();
  }
  if (iters_out) *iters_out = total_it;
#undef TQR_CK
#undef TQR_CKL
  return converged ? 0 : -1;
}

}  // namespace tqr
