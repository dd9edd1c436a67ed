// Shared-A multi-right-hand-side solver: R problems  min tau_j ||x_j||_1 + 1/2 ||A x_j - b_j||^2
// with one dense A stored as bf16 times a per-tensor scale (MFIPM_PREC_BF16_A).  All right-hand
// sides run the single-corrector IPM of Sec. 5.1 in lockstep, each with its own scalars (mu,
// sigma, step lengths, corrector decision, stop flag); a column that has converged keeps its
// iterate.  Every PCG operator product (Sec. 4) needs A^T A w for all columns at once, so A is
// read once per product for all R columns:
//     T = A W,  Y = A^T T      (two GEMMs, bf16 operands, float32 accumulation)
// where W (and T) are split into bf16 high and low halves, W = W_hi + W_lo, which keeps the
// product accurate to ~2^-16 at the cost of doubling the GEMM's N (the GEMMs are bounded by
// reading A, not by the tensor rate).  A transposed copy of A in the workspace makes both
// GEMMs K-major.  The outer loop is float64: the residual A^T (A x - b) is formed on the float32
// pipes with a biased accumulator that captures every rounding error exactly (resid_gemm).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "large_dct.h"
#include "lockstep.h"
#include "mrhs.h"

namespace mfipm {
namespace mr {

constexpr int kT = 256;       // threads per block of the per-column passes
constexpr int kIdx = 2048;    // indices per block (8 per thread)
constexpr int kPart = 8;      // partial sums per (column, block)

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// P^-1 r for one index (Eq. eq:ne2_P), float32
__device__ __forceinline__ float2 precond2(float2 d, float2 r, float rho) {
  const float a = d.x + rho, c = d.y + rho;
  const float inv = 1.f / (d.x * d.y + rho * (d.x + d.y));
  return make_float2((c * r.x + rho * r.y) * inv, (rho * r.x + a * r.y) * inv);
}

// block sum of up to kPart values; thread 0 writes part[(col * nb + blk) * kPart + k]
// Per-block totals of K per-thread values: warp sums in the values' own type (float32 for
// the positive sums of the float32 passes, so that no float64 instruction runs per thread),
// the warps' totals in float64.
template <int K, class V>
__device__ __forceinline__ void block_partials(const V (&v)[K], double* part, int col, int nb, int blk) {
  __shared__ double red[kT / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const V w = warp_sum(v[k]);
    if (lane == 0) red[warp][k] = (double)w;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += red[w][threadIdx.x];
    part[((int64_t)col * nb + blk) * kPart + threadIdx.x] = s;
  }
}
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// per-block minima (exact in any precision: the warp minima stay in the values' type)
template <int K, class V>
__device__ __forceinline__ void block_minima(const V (&v)[K], double* part, int col, int nb, int blk) {
  __shared__ double red[kT / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    V w = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = vmin(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (lane == 0) red[warp][k] = (double)w;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = INFINITY;
    for (int w = 0; w < kT / 32; ++w) s = fmin(s, red[w][threadIdx.x]);
    part[((int64_t)col * nb + blk) * kPart + threadIdx.x] = s;
  }
}
// column total of partial k over the nb block partials, computed by a whole block of kT
// threads (every thread gets the result; fixed order, so deterministic)
__device__ double block_col_total(const double* part, int col, int nb, int k, bool is_min = false) {
  __shared__ double red[kT / 32];
  __shared__ double out;
  double s = is_min ? INFINITY : 0.0;
  for (int b = threadIdx.x; b < nb; b += kT) {
    const double v = part[((int64_t)col * nb + b) * kPart + k];
    s = is_min ? fmin(s, v) : s + v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double t = __shfl_xor_sync(0xffffffffu, s, o);
    s = is_min ? fmin(s, t) : s + t;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = is_min ? INFINITY : 0.0;
    for (int w = 0; w < kT / 32; ++w) t = is_min ? fmin(t, red[w]) : t + red[w];
    out = t;
  }
  __syncthreads();
  return out;
}
// column total of partial k (fixed order: deterministic)
__device__ __forceinline__ double col_total(const double* part, int col, int nb, int k, bool is_min = false) {
  double s = is_min ? INFINITY : 0.0;
  for (int b = 0; b < nb; ++b) {
    const double v = part[((int64_t)col * nb + b) * kPart + k];
    s = is_min ? fmin(s, v) : s + v;
  }
  return s;
}

// ------------------------------------------------------------------ setup
__global__ void transpose_bf16(const __nv_bfloat16* __restrict__ A, int64_t lda, __nv_bfloat16* __restrict__ At,
                               int m, int n) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = by + r, k = bx + threadIdx.x;
    if (i < m && k < n) tile[r][threadIdx.x] = A[(int64_t)i * lda + k];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = bx + r, i = by + threadIdx.x;
    if (k < n && i < m) At[(int64_t)k * m + i] = tile[threadIdx.x][r];
  }
}

__global__ void gather_b(const double* const* __restrict__ bptr, double* __restrict__ Bm, int m) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    Bm[(int64_t)j * m + i] = bptr[j][i];
}

// ------------------------------------------------------------------ GEMMs
// C[c][r] = sum_k Aop[r][k] * Bop[c][k]   (Aop: rows x K bf16, Bop: N x K bf16, C: N x rows f32)
// Plain CUDA-core tile (64 x 64 outputs per block, float32 accumulation).
__global__ void gemm_bf16_simple(const __nv_bfloat16* __restrict__ Aop, const __nv_bfloat16* __restrict__ Bop,
                                 float* __restrict__ C, int rows, int N, int K) {
  __shared__ float As[32][65];
  __shared__ float Bs[32][65];
  const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += kT) {
      const int rr = e / 32, kk = e % 32;
      As[kk][rr] = (r0 + rr < rows && k0 + kk < K) ? bf(Aop[(int64_t)(r0 + rr) * K + k0 + kk]) : 0.f;
      Bs[kk][rr] = (c0 + rr < N && k0 + kk < K) ? bf(Bop[(int64_t)(c0 + rr) * K + k0 + kk]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty * 4 + q];
        b[q] = Bs[kk][tx * 4 + q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + ty * 4 + p, c = c0 + tx * 4 + q;
      if (r < rows && c < N) C[(int64_t)c * rows + r] = acc[p][q];
    }
}

// ------------------------------------------------------------------ float64-grade residual GEMMs
// Out[j][r] = scale * sum_k Aop[r][k] X[j][k] (- Bsub[j][r]) for the outer residual
// A^T (A x - b) of Eq. fzfs.  bf16 A is exact in float32 and x = xh + xl is carried as two
// float32 halves.  Each output keeps a biased float32 accumulator H that starts at
// H0 = 1.5 * 2^E, with 2^E >= 4 ||a_r|| ||x_j|| over the block's K range (Cauchy-Schwarz),
// so H never leaves the binade [2^E, 2^(E+1)).  For a term t = a * xh:
//     H' = fma(a, xh, H)            (one rounding)
//     q  = H' - H                   (exact: H, H' in one binade)
//     e  = fma(a, xh, -q)           (the rounding error of H', exact when a * xh fits
//                                    24 bits below ulp(H); else rounded at 2^-24 |e|)
// and the small remainders e + a * xl accumulate in float32 c, folded every K-tile into a
// double-float sum.  Five float32 operations per term; the result H - H0 + sum(c) carries
// ~2^-40 of ||a|| ||x||, which is what the float64 outer loop of Sec. 5.1 needs.
constexpr int kRB = 64;   // rows per block
constexpr int kJB = 64;   // columns (right-hand sides) per block
constexpr int kKB = 32;   // K per tile
constexpr int kMaxRsplit = 32;

// K range [k0, k1) of split s out of S (whole tiles of kKB, identical in every kernel)
__host__ __device__ __forceinline__ void split_range(int K, int S, int s, int* k0, int* k1) {
  const int64_t T = (K + kKB - 1) / kKB;
  const int t0 = (int)((int64_t)s * T / S), t1 = (int)((int64_t)(s + 1) * T / S);
  *k0 = t0 * kKB;
  *k1 = min(K, t1 * kKB);
}
// smallest power of two >= v, clamped to [2^-50, 2^50]
__device__ __forceinline__ float pow2_ceil(float v) {
  if (!(v > 0x1p-50f)) return 0x1p-50f;
  if (v >= 0x1p50f) return 0x1p50f;
  int e;
  const float f = frexpf(v, &e);  // v = f 2^e, f in [0.5, 1)
  return f == 0.5f ? ldexpf(1.f, e - 1) : ldexpf(1.f, e);
}

// pw[s * rows + r] >= ||Aop[r][range s]||_2, one warp per (row, split)
__global__ void k_rowpow(const __nv_bfloat16* __restrict__ Aop, int64_t lda, int rows, int K, int S,
                         float* __restrict__ pw) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)rows * S) return;
  const int r = (int)(w / S), s = (int)(w % S);
  int k0, k1;
  split_range(K, S, s, &k0, &k1);
  float acc = 0.f;
  for (int k = k0 + lane; k < k1; k += 32) {
    const float v = bf(Aop[(int64_t)r * lda + k]);
    acc = fmaf(v, v, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) pw[(int64_t)s * rows + r] = pow2_ceil(sqrtf(acc) * 1.0001f);
}

// cp[s * R + j] >= ||x_j[range s]||_2 for the double-float X (R x K).  Block (s, j).
__global__ void k_xbound(const float2* __restrict__ X, float* __restrict__ cp, int K, int R, int S) {
  const int s = blockIdx.x, j = blockIdx.y;
  int k0, k1;
  split_range(K, S, s, &k0, &k1);
  float acc = 0.f;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const float h = X[(int64_t)j * K + k].x;
    acc = fmaf(h, h, acc);
  }
  __shared__ float red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cp[(int64_t)s * R + j] = pow2_ceil(sqrtf(t) * 1.0001f);
  }
}

// Part[s][j][r] (double-float) = sum over K range s of Aop[r][k] * (xh + xl)[j][k].
// Block (row tile, column tile, split); 256 threads, 4 x 4 outputs each.  K tiles are double
// buffered: A through registers (converted to float32 in shared memory), X by cp.async.
// vecA: Aop rows and base 16-byte aligned with lda % 8 == 0.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__global__ void __launch_bounds__(256, 2)
resid_gemm(const __nv_bfloat16* __restrict__ Aop, int64_t lda, const float* __restrict__ rp,
           const float2* __restrict__ Xf, const float* __restrict__ cp, float2* __restrict__ Part, int rows, int R,
           int K, int S, int vecA) {
  __shared__ __align__(16) float As[2][kKB][kRB];
  __shared__ __align__(16) float2 Xs[2][kKB][kJB];
  const int r0 = blockIdx.x * kRB, j0 = blockIdx.y * kJB, s = blockIdx.z;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int k0, k1;
  split_range(K, S, s, &k0, &k1);
  // loader coordinates: 8 consecutive k of one row (A) / one column (X)
  const int lrow = threadIdx.x >> 2, lk = (threadIdx.x & 3) * 8;
  uint4 ra;
  auto fetchA = [&](int kb) {
    const int k = kb + lk, r = r0 + lrow;
    if (r < rows && vecA && k + 8 <= k1) {
      ra = *reinterpret_cast<const uint4*>(Aop + (int64_t)r * lda + k);
    } else {
      __nv_bfloat16 t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
        t[i] = (r < rows && k + i < k1) ? Aop[(int64_t)r * lda + k + i] : __float2bfloat16_rn(0.f);
      ra = *reinterpret_cast<const uint4*>(t);
    }
  };
  auto stashA = [&](int buf) {
    const __nv_bfloat16* t = reinterpret_cast<const __nv_bfloat16*>(&ra);
#pragma unroll
    for (int i = 0; i < 8; ++i) As[buf][lk + i][lrow] = bf(t[i]);
  };
  auto copyX = [&](int kb, int buf) {
    const int k = kb + lk, j = j0 + lrow;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const bool ok = j < R && k + i < k1;
      cp_async8(&Xs[buf][lk + i][lrow], ok ? (const void*)(Xf + (int64_t)j * K + k + i) : (const void*)Xf, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  // H0 = 1.5 * 2^E with 2^E = 4 rp cp (exact: rp, cp are powers of two)
  auto bias = [&](int p, int q) {
    const int r = min(r0 + ty * 4 + p, rows - 1), j = min(j0 + tx * 4 + q, R - 1);
    return 6.f * rp[(int64_t)s * rows + r] * cp[(int64_t)s * R + j];
  };
  float H[4][4], c[4][4], Sh[4][4], Sl[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      H[p][q] = bias(p, q);
      c[p][q] = Sh[p][q] = Sl[p][q] = 0.f;
    }
  if (k0 < k1) {
    copyX(k0, 0);
    fetchA(k0);
    stashA(0);
    cp_async_wait_all();
  }
  __syncthreads();
  int buf = 0;
  for (int kb = k0; kb < k1; kb += kKB) {
    const bool more = kb + kKB < k1;
    if (more) {
      copyX(kb + kKB, buf ^ 1);
      fetchA(kb + kKB);
    }
#pragma unroll 4
    for (int kk = 0; kk < kKB; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 x01 = *reinterpret_cast<const float4*>(&Xs[buf][kk][tx * 4]);
      const float4 x23 = *reinterpret_cast<const float4*>(&Xs[buf][kk][tx * 4 + 2]);
      const float a[4] = {a4.x, a4.y, a4.z, a4.w};
      const float xh[4] = {x01.x, x01.z, x23.x, x23.z};
      const float xl[4] = {x01.y, x01.w, x23.y, x23.w};
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float hn = __fmaf_rn(a[p], xh[q], H[p][q]);
          const float qv = __fsub_rn(hn, H[p][q]);
          const float e = __fmaf_rn(a[p], xh[q], -qv);
          c[p][q] = __fmaf_rn(a[p], xl[q], __fadd_rn(c[p][q], e));
          H[p][q] = hn;
        }
    }
    // fold the tile's remainders into the double-float sum
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const df t = df_two_sum(Sh[p][q], c[p][q]);
        Sh[p][q] = t.hi;
        Sl[p][q] = __fadd_rn(Sl[p][q], t.lo);
        c[p][q] = 0.f;
      }
    if (more) {
      stashA(buf ^ 1);
      cp_async_wait_all();
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + ty * 4 + p, j = j0 + tx * 4 + q;
      if (r < rows && j < R) {
        const df v = df(__fsub_rn(H[p][q], bias(p, q))) + df(Sh[p][q], Sl[p][q]);
        Part[((int64_t)s * R + j) * rows + r] = make_float2(v.hi, v.lo);
      }
    }
}

// Rr = scale * sum_s Part1 - Bm (float64), its (hi, lo) split for the second GEMM, and
// cp2[s2 * R + j] >= ||Rr_j[range s2]||.  Block (s2, j) over the K ranges of the second GEMM.
__global__ void k_fin1(const float2* __restrict__ Part, int S1, const double* __restrict__ Bm, double scale,
                       double* __restrict__ Rr, float2* __restrict__ Rf, float* __restrict__ cp2, int m, int R,
                       int S2) {
  const int s2 = blockIdx.x, j = blockIdx.y;
  int k0, k1;
  split_range(m, S2, s2, &k0, &k1);
  float acc = 0.f;
  for (int r = k0 + threadIdx.x; r < k1; r += blockDim.x) {
    df v(0.f);
    for (int s = 0; s < S1; ++s) {
      const float2 t = Part[((int64_t)s * R + j) * m + r];
      v = v + df(t.x, t.y);
    }
    const int64_t gi = (int64_t)j * m + r;
    const double rv = scale * to_double(v) - Bm[gi];
    Rr[gi] = rv;
    const float h = __double2float_rn(rv);
    Rf[gi] = make_float2(h, __double2float_rn(rv - (double)h));
    acc = fmaf(h, h, acc);
  }
  __shared__ float red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cp2[(int64_t)s2 * R + j] = pow2_ceil(sqrtf(t) * 1.0001f);
  }
}
// Gr = scale * sum_s Part2 (float64)
__global__ void k_fin2(const float2* __restrict__ Part, int S2, double scale, float2* __restrict__ Gr, int n, int R) {
  const int64_t total = (int64_t)R * n;
  const df sc = to_df(scale);
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
       gi += (int64_t)gridDim.x * blockDim.x) {
    df v(0.f);
    for (int s = 0; s < S2; ++s) {
      const float2 t = Part[(int64_t)s * total + gi];
      v = v + df(t.x, t.y);
    }
    const df g = sc * v;
    Gr[gi] = make_float2(g.hi, g.lo);
  }
}

// ------------------------------------------------------------------ residual on the tensor cores
// The same float64-grade products A x and A^T r on the tcgen05 GEMM by error-free splitting
// into integer digit slices (the splitting of Ozaki et al. for accurate products on
// low-precision units): per row r of A and per column j of x, with 2^E bounding the largest
// magnitude,
//     a = 2^(Er - 7) sum_t D_t 2^(-7t),   x = 2^(Ej - 7) sum_s X_s 2^(-7s),
// digits |D_0|, |X_0| <= 128 and |D_t|, |X_s| <= 65 after the first: every digit is an integer
// exact in bf16, every product of two digits is below 2^14 and a sum of 1024 of them below
// 2^24, so the GEMM's float32 accumulation over a split-K chunk of 1024 is exact.  The integer
// chunk sums are combined in double-float with the weights 2^(Er + Ej - 14 - 7(t + s)) for all
// pairs t + s <= kPairMax.  kSlA = 5 slices carry 35 bits of A (bf16 A needs 8 bits within
// 2^-27 of the row maximum: exact but for entries below that), kSlX = 6 carry 42 bits of x.
constexpr int kSlA = 5, kSlX = 6, kPairMax = 6, kChunkK = 1024;

__device__ __forceinline__ int exp_above(float mx) {  // 2^E > mx (frexp: mx = f 2^E, f in [0.5, 1))
  if (!(mx > 0.f)) return -60;
  int e;
  frexpf(mx, &e);
  return e;
}
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// A (rows x K, lda) -> digit slices S[t][r][k] and row exponents E[r]; one block per row
__global__ void k_slice_rows(const __nv_bfloat16* __restrict__ A, int64_t lda, int rows, int K,
                             __nv_bfloat16* __restrict__ S, int* __restrict__ E) {
  __shared__ float red[33];
  const int r = blockIdx.x;
  const __nv_bfloat16* a = A + (int64_t)r * lda;
  float mx = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmaxf(mx, fabsf(bf(a[k])));
  const int e = exp_above(block_max(mx, red));
  if (threadIdx.x == 0) E[r] = e;
  const float sc = ldexpf(1.f, 7 - e);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    float v = bf(a[k]) * sc;  // |v| < 128, exact
#pragma unroll
    for (int t = 0; t < kSlA; ++t) {
      const float dg = rintf(v);
      S[((int64_t)t * rows + r) * K + k] = __float2bfloat16_rn(dg);
      v = (v - dg) * 128.f;  // exact
    }
  }
}

__device__ __forceinline__ df load_dfv(const float2* X, int64_t i) { return df(X[i].x, X[i].y); }
__device__ __forceinline__ df load_dfv(const double* X, int64_t i) { return to_df(X[i]); }
__device__ __forceinline__ df scale2(df v, float p2) { return df(v.hi * p2, v.lo * p2); }  // exact: power of two

// X (R x K, double-float or float64) -> digit slices S[s][j][k] and column exponents E[j];
// one block per column
template <class T>
__global__ void k_slice_cols(const T* __restrict__ X, int R, int K, __nv_bfloat16* __restrict__ S,
                             int* __restrict__ E) {
  __shared__ float red[33];
  const int j = blockIdx.x;
  float mx = 0.f;
  for (int k = threadIdx.x; k < K; k += blockDim.x) mx = fmaxf(mx, fabsf(load_dfv(X, (int64_t)j * K + k).hi));
  // |x| <= |hi| (1 + 2^-24): a bound just above the largest hi covers it
  const int e = exp_above(block_max(mx, red) * 1.0001f);
  if (threadIdx.x == 0) E[j] = e;
  const float sc = ldexpf(1.f, 7 - e);
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    df v = scale2(load_dfv(X, (int64_t)j * K + k), sc);
#pragma unroll
    for (int s = 0; s < kSlX; ++s) {
      const float dg = rintf(v.hi);
      S[((int64_t)s * R + j) * K + k] = __float2bfloat16_rn(dg);
      v = scale2(v - df(dg), 128.f);
    }
  }
}

// Acc[j][r] (+)= sum over the c slices s0.. of one GEMM call: weight(t, s) * (integer chunk sums)
__global__ void k_slice_acc(const float* __restrict__ C, int splits, int c, int R, int rows, int t, int s0,
                            const int* __restrict__ Er, const int* __restrict__ Ej, float2* __restrict__ Acc,
                            int first) {
  const int64_t total = (int64_t)R * rows, N = (int64_t)c * R;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
       gi += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(gi / rows), r = (int)(gi % rows);
    df acc = first ? df(0.f) : df(Acc[gi].x, Acc[gi].y);
    for (int sl = 0; sl < c; ++sl) {
      int isum = 0;  // exact: chunk sums are integers below 2^24, their sum below 2^28
      for (int sp = 0; sp < splits; ++sp) isum += __float2int_rn(C[((int64_t)sp * N + sl * R + j) * rows + r]);
      const float hi = __int2float_rn(isum);
      const df term(hi, __int2float_rn(isum - __float2int_rn(hi)));
      acc = acc + scale2(term, ldexpf(1.f, Er[r] + Ej[j] - 14 - 7 * (t + s0 + sl)));
    }
    Acc[gi] = make_float2(acc.hi, acc.lo);
  }
}
// Rr = scale Acc - Bm (float64), first product of the residual
__global__ void k_fin1_tc(const float2* __restrict__ Acc, const double* __restrict__ Bm, double scale,
                          double* __restrict__ Rr, int64_t total) {
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x)
    Rr[gi] = scale * ((double)Acc[gi].x + (double)Acc[gi].y) - Bm[gi];
}
// Gr = scale Acc (double-float)
__global__ void k_fin2_tc(const float2* __restrict__ Acc, double scale, float2* __restrict__ Gr, int64_t total) {
  const df sc = to_df(scale);
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const df g = sc * df(Acc[gi].x, Acc[gi].y);
    Gr[gi] = make_float2(g.hi, g.lo);
  }
}

// The residual of the outer loop's large-gap iterations (reading R17) in float32-grade
// arithmetic on the tensor cores: a value v as three bf16 pieces v0 + v1 + v2 (24 significant
// bits; every piece times a bf16 entry of A is exact in float32, the GEMM sums in float32).
__device__ __forceinline__ void bf16_pieces3(float f, __nv_bfloat16* S, int64_t stride, int64_t at) {
  const __nv_bfloat16 p0 = __float2bfloat16_rn(f);
  const float r1 = f - __bfloat162float(p0);
  const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
  S[at] = p0;
  S[at + stride] = p1;
  S[at + 2 * stride] = __float2bfloat16_rn(r1 - __bfloat162float(p1));
}
// x (R x K, double-float) -> S[piece][j][k]
__global__ void k_pieces_x(const float2* __restrict__ X, int R, int K, __nv_bfloat16* __restrict__ S) {
  const int64_t total = (int64_t)R * K;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = X[gi];
    // hi - bf16(hi) is exact in float32; lo lies below hi's last bit
    const __nv_bfloat16 p0 = __float2bfloat16_rn(v.x);
    const float r1 = (v.x - __bfloat162float(p0)) + v.y;
    const __nv_bfloat16 p1 = __float2bfloat16_rn(r1);
    S[gi] = p0;
    S[gi + total] = p1;
    S[gi + 2 * total] = __float2bfloat16_rn(r1 - __bfloat162float(p1));
  }
}
// after T = A x (C: splits x 3R x m): Rr = scale T - b (float64) and the pieces of Rr
__global__ void k_pieces_mid(const float* __restrict__ C, int splits, int R, int m, const double* __restrict__ Bm,
                             double scale, double* __restrict__ Rr, __nv_bfloat16* __restrict__ S) {
  const int64_t total = (int64_t)R * m, N = 3 * (int64_t)R;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = gi / m, i = gi % m;
    float t = 0.f;
    for (int sp = 0; sp < splits; ++sp)
      for (int pc = 0; pc < 3; ++pc) t += C[(sp * N + pc * R + j) * m + i];
    const double r = scale * (double)t - Bm[gi];
    Rr[gi] = r;
    bf16_pieces3((float)r, S, total, gi);
  }
}
// after A^T r (C: splits x 3R x n): Gr = scale sum (double-float)
__global__ void k_pieces_fin(const float* __restrict__ C, int splits, int R, int n, double scale,
                             float2* __restrict__ Gr) {
  const int64_t total = (int64_t)R * n, N = 3 * (int64_t)R;
  const float sc = (float)scale;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total; gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = gi / n, k = gi % n;
    float t = 0.f;
    for (int sp = 0; sp < splits; ++sp)
      for (int pc = 0; pc < 3; ++pc) t += C[(sp * N + pc * R + j) * n + k];
    Gr[gi] = make_float2(sc * t, 0.f);
  }
}

// ------------------------------------------------------------------ per-column state
struct Dev {
  int m, n, R, nb;                 // nb: blocks per column of the index passes
  int op;                          // OP_SHARED_BF16 or OP_LARGE_DCT
  int nb2;                         // blocks per column of the operator's partial sums (part2)
  double a_scale, rho;
  float* Yv;                       // R x n   A^T A w (OP_LARGE_DCT)
  const __nv_bfloat16* A;          // m x n (lda)
  int64_t lda;
  const __nv_bfloat16* At;         // n x m
  float2* X;                       // R x n   residual input (x or trial x), double-float
  double* Rr;                      // R x m   A x - b
  float2* Gr;                      // R x n   A^T (A x - b), double-float
  double* Bm;                      // R x m
  float4* zs;                      // R x n x 2 {u, v}, {s_u, s_v} as double-float pairs
  float2 *X1, *X2, *Rv, *Pv, *Dv;  // R x n each
  __nv_bfloat16* W;                // 2R x n
  __nv_bfloat16* Tb;               // 2R x m
  float* C1;                       // s1 x 2R x m  (split-K slices)
  float* C2;                       // s2 x 2R x n
  int s1, s2;
  double* part;                    // R x nb x kPart
  Col* col;
  int* counters;                   // [0] active PCG columns, [1] unfinished columns, [2] corrector columns
  SolveParams prm;
};

// dz, ds of one index from the PCG pairs (Eq. redNewtonB; corrector reading R6).  Precision
// split: the direction, Theta^-1 = s/z, sigma mu / z and the step-to-boundary ratios only steer
// the iteration and are float32 (the PCG precision); the iterate (z, s), its update
// z + alpha dz, x = u - v, the residual and the gap sums stay float64.  The ratio test and the
// update evaluate the direction by the same function from the same inputs, so the
// fraction-to-boundary rule keeps z, s > 0.
struct Steer {
  float smu, s3mut, ap1, ad1;
  bool corr;
};
__device__ __forceinline__ Steer steer(const Col& c, double sigma3, bool corr) {
  return Steer{(float)(c.sigma * c.mu), (float)(sigma3 * c.mu_t), (float)c.alpha_p1, (float)c.alpha_d1, corr};
}
struct D2 {
  float dz, ds;
};
__device__ __forceinline__ D2 dirn(float z, float s, float dz1, float dz2, const Steer& c) {
  const float rz = __frcp_rn(z), d = s * rz;
  const float ds1 = (c.smu * rz - s) - d * dz1;
  D2 r{dz1, ds1};
  if (c.corr) {
    const float zt = z + c.ap1 * dz1, st = s + c.ad1 * ds1;
    r.dz = dz1 + dz2;
    r.ds = ds1 + ((c.s3mut - zt * st) * rz - d * dz2);
  }
  return r;
}

// The iterate in double-float (about 48 significant bits on the float32 pipes; float64 runs
// at 1/64 of the float32 rate on this part): per index {u, v} and {s_u, s_v} as (hi, lo)
// pairs, 32 bytes.  x and the residual g are double-float too.
struct St {
  df u, v, su, sv;
};
__device__ __forceinline__ St load_st(const float4* zs, int64_t gi) {
  const float4 a = zs[2 * gi], b = zs[2 * gi + 1];
  return St{df(a.x, a.y), df(a.z, a.w), df(b.x, b.y), df(b.z, b.w)};
}
__device__ __forceinline__ void store_st(float4* zs, int64_t gi, const St& q) {
  zs[2 * gi] = make_float4(q.u.hi, q.u.lo, q.v.hi, q.v.lo);
  zs[2 * gi + 1] = make_float4(q.su.hi, q.su.lo, q.sv.hi, q.sv.lo);
}
__device__ __forceinline__ df axpy(df z, df a, float d) { return z + a * df(d); }
__device__ __forceinline__ float2 f2(df a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ df d2(float2 a) { return df(a.x, a.y); }

// iterate update (previous direction) and x = u - v; partials z.s, 1^T z, ||x||^2
__global__ void k_update(Dev d, int first) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  const bool done = c.done, corr = c.corr;
  const Steer sc = steer(c, d.prm.sigma3, corr);
  const df ap = to_df(c.alpha_p), ad = to_df(c.alpha_d), keep = to_df(1.0 - d.prm.eta);
  float a[3] = {0.f, 0.f, 0.f};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    St st;
    if (first) {
      st = St{df(1.f), df(1.f), df(1.f), df(1.f)};  // reading R3
    } else {
      st = load_st(d.zs, gi);
      if (!done) {
        const float2 x1 = d.X1[gi];
        const float2 x2 = corr ? d.X2[gi] : make_float2(0.f, 0.f);
        const D2 du = dirn(st.u.hi, st.su.hi, x1.x, x2.x, sc);
        const D2 dv = dirn(st.v.hi, st.sv.hi, x1.y, x2.y, sc);
        const St o = st;
        st.u = axpy(o.u, ap, du.dz);
        st.v = axpy(o.v, ap, dv.dz);
        st.su = axpy(o.su, ad, du.ds);
        st.sv = axpy(o.sv, ad, dv.ds);
        if (!(st.u.hi > 0.f)) st.u = o.u * keep;
        if (!(st.v.hi > 0.f)) st.v = o.v * keep;
        if (!(st.su.hi > 0.f)) st.su = o.su * keep;
        if (!(st.sv.hi > 0.f)) st.sv = o.sv * keep;
      }
    }
    store_st(d.zs, gi, st);
    const df x = st.u - st.v;
    d.X[gi] = f2(x);
    // float32 terms of positive sums (no cancellation), float64 across threads
    a[0] += st.u.hi * st.su.hi + st.v.hi * st.sv.hi;
    a[1] += st.u.hi + st.v.hi;
    a[2] += x.hi * x.hi;
  }
  block_partials<3>(a, d.part, j, d.nb, blk);
}

// sum of squares of a double-float vector, per block
__global__ void k_colnorm2_df(const float2* __restrict__ V, int len, double* part, int nb) {
  const int j = blockIdx.y, blk = blockIdx.x;
  float a = 0.f;
  const int per = (len + nb - 1) / nb;
  for (int i = blk * per + threadIdx.x; i < min(len, (blk + 1) * per); i += kT) {
    const float t = V[(int64_t)j * len + i].x;
    a = fmaf(t, t, a);
  }
  const float v[1] = {a};
  block_partials<1>(v, part, j, nb, blk);
}

__global__ void k_colnorm2(const double* __restrict__ V, int len, double* part, int nb) {
  const int j = blockIdx.y, blk = blockIdx.x;
  double v[1] = {0.0};
  const int per = (len + nb - 1) / nb;
  for (int i = blk * per + threadIdx.x; i < min(len, (blk + 1) * per); i += kT) {
    const double t = V[(int64_t)j * len + i];
    v[0] += t * t;
  }
  block_partials<1>(v, part, j, nb, blk);
}

// gap test, mu, sigma (one thread per column)
// one block of kT threads per column
// lowp: the residual came from the float32-grade chain; a column that would stop, or whose gap
// has reached prm.f32_gap, is counted in counters[3] instead (the driver then recomputes the
// residual in full precision and runs this kernel again), so no stop rests on it.
__global__ void k_stats(Dev d, int it, const double* part2, int lowp) {
  const int j = blockIdx.x;
  Col& c = d.col[j];
  if (c.done) return;
  const double zts = block_col_total(d.part, j, d.nb, 0), l1 = block_col_total(d.part, j, d.nb, 1);
  const double res2 = block_col_total(part2, j, d.nb2, 0);
  if (threadIdx.x) return;
  c.res2 = res2;
  c.mu = zts / (2.0 * d.n);
  c.P_obj = c.tau * l1 + 0.5 * res2;
  c.rel_gap = zts / (1.0 + fabs(c.P_obj));
  c.corr = 0;
  c.ipm_iters = it - 1;
  const bool stop_now = !isfinite(c.rel_gap) || c.rel_gap <= d.prm.tol || it > d.prm.max_iter;
  if (lowp && (stop_now || !(c.rel_gap > d.prm.f32_gap))) atomicAdd(&d.counters[3], 1);
  else if (!isfinite(c.rel_gap)) { c.stop = MFIPM_NUMERIC; c.done = 1; }
  else if (c.rel_gap <= d.prm.tol) { c.stop = MFIPM_OK; c.done = 1; }
  else if (it > d.prm.max_iter) { c.stop = MFIPM_NOT_CONVERGED; c.done = 1; }
  c.sigma = (it != 1 && (c.prev_ap <= d.prm.alpha_bar || c.prev_ad <= d.prm.alpha_bar)) ? d.prm.sigma2 : d.prm.sigma1;
  c.nmat += 2;
  if (!c.done) atomicAdd(&d.counters[1], 1);
}

// PCG initialisation.  corr = 0: rhs = sigma mu / z - [tau + g; tau - g], writes Theta^-1.
// corr = 1: rhs~ = f_z~ + Z^-1 f_s~ at the trial point (reading R6), only for columns that
// take a corrector.  Columns that are done (or take no corrector) get rhs = 0.
__global__ void k_pcg_init(Dev d, int corr) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  const bool live = !c.done && (!corr || c.corr_next);
  const Steer sc = steer(c, d.prm.sigma3, false);
  const df tau = to_df(c.tau), ap1 = to_df(c.alpha_p1), ad1 = to_df(c.alpha_d1);
  const float s3mu = (float)(d.prm.sigma3 * c.mu_t);
  float v[2] = {0.f, 0.f};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const St st = load_st(d.zs, gi);
    float2 dd;
    if (!corr) {
      dd = make_float2(__fdiv_rn(st.su.hi, st.u.hi), __fdiv_rn(st.sv.hi, st.v.hi));
      d.Dv[gi] = dd;
    } else {
      dd = d.Dv[gi];
    }
    float2 r = make_float2(0.f, 0.f);
    if (live) {
      const df g = d2(d.Gr[gi]);
      const df tpg = tau + g, tmg = tau - g;
      if (!corr) {
        r.x = sc.smu * __frcp_rn(st.u.hi) - tpg.hi;
        r.y = sc.smu * __frcp_rn(st.v.hi) - tmg.hi;
      } else {
        // f_z~ at the trial point in double-float, Z^-1 f_s~ in float32
        const float2 x1 = d.X1[gi];
        const D2 du = dirn(st.u.hi, st.su.hi, x1.x, 0.f, sc);
        const D2 dv = dirn(st.v.hi, st.sv.hi, x1.y, 0.f, sc);
        const df zu = axpy(st.u, ap1, du.dz), zv = axpy(st.v, ap1, dv.dz);
        const df tsu = axpy(st.su, ad1, du.ds), tsv = axpy(st.sv, ad1, dv.ds);
        r.x = (tsu - tpg).hi + (s3mu - zu.hi * tsu.hi) * __frcp_rn(st.u.hi);
        r.y = (tsv - tmg).hi + (s3mu - zv.hi * tsv.hi) * __frcp_rn(st.v.hi);
      }
    }
    const float2 p = precond2(dd, r, (float)c.rho);
    d.Rv[gi] = r;
    d.Pv[gi] = p;
    if (d.op == OP_SHARED_BF16) {
      const float w = p.x - p.y;
      const __nv_bfloat16 wh = __float2bfloat16_rn(w);
      d.W[(int64_t)j * d.n + i] = wh;
      d.W[(int64_t)(d.R + j) * d.n + i] = __float2bfloat16_rn(w - __bfloat162float(wh));
    }
    v[0] += r.x * p.x + r.y * p.y;
    v[1] += dd.x * p.x * p.x + dd.y * p.y * p.y;
  }
  block_partials<2>(v, d.part, j, d.nb, blk);
}

// T = a_scale (C1_hi + C1_lo) -> bf16 hi/lo halves; partial ||T_j||^2 = ||A w_j||^2
__global__ void k_split_t(Dev d, double* part2) {
  const int j = blockIdx.y, blk = blockIdx.x;
  float v[1] = {0.f};
  const int per = (d.m + d.nb - 1) / d.nb;
  for (int i = blk * per + threadIdx.x; i < min(d.m, (blk + 1) * per); i += kT) {
    float acc = 0.f;
    for (int sp = 0; sp < d.s1; ++sp) {
      const float* C = d.C1 + (int64_t)sp * 2 * d.R * d.m;
      acc += C[(int64_t)j * d.m + i] + C[(int64_t)(d.R + j) * d.m + i];
    }
    const float t = (float)d.a_scale * acc;
    const __nv_bfloat16 th = __float2bfloat16_rn(t);
    d.Tb[(int64_t)j * d.m + i] = th;
    d.Tb[(int64_t)(d.R + j) * d.m + i] = __float2bfloat16_rn(t - __bfloat162float(th));
    v[0] += t * t;
  }
  block_partials<1>(v, part2, j, d.nb, blk);
}

// alpha = r.P^-1 r / (p.Theta^-1 p + ||A w||^2); first iteration records rz0
// one block of kT threads per column
__global__ void k_alpha(Dev d, int first, const double* part2) {
  const int j = blockIdx.x;
  Col& c = d.col[j];
  const double pdp = block_col_total(d.part, j, d.nb, 1), aw2 = block_col_total(part2, j, d.nb2, 0);
  const double rz = first ? block_col_total(d.part, j, d.nb, 0) : 0.0;
  if (threadIdx.x) return;
  if (first) {
    c.rz0 = c.rz = rz;
    c.active = rz > 0.0 && isfinite(rz);
  }
  // breakdown guard: p^T H p not positive and finite ends this column's solve with its last
  // iterate (on the first iteration: zero)
  const double php = pdp + aw2, a = c.rz / php;
  if (c.active && (!(php > 0.0) || !isfinite(php) || !isfinite(a) || !isfinite((double)(float)a))) c.active = 0;
  c.alpha = c.active ? (float)a : 0.f;
  if (c.active) c.nmat += 2;
}

// at most 64 registers: four blocks per SM for this memory-bound pass (measured faster than
// its unbounded 128 registers and than three blocks, despite a small spill)
__global__ void __launch_bounds__(kT, 4) k_pcg_D(Dev d, float2* __restrict__ Xo, int first) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  // a column whose PCG has stopped has alpha = 0: nothing would change (its partial is not
  // read); on the first iteration every column writes its x = 0
  if (!first && !c.active) return;
  const float alpha = c.alpha, rho = (float)c.rho, sc = (float)d.a_scale;
  float v[1] = {0.f};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    float2 x = first ? make_float2(0.f, 0.f) : Xo[gi];
    float2 r = d.Rv[gi];
    const float2 p = d.Pv[gi], dd = d.Dv[gi];
    float y;
    if (d.op == OP_SHARED_BF16) {
      float yacc = 0.f;
      for (int sp = 0; sp < d.s2; ++sp) {
        const float* C = d.C2 + (int64_t)sp * 2 * d.R * d.n;
        yacc += C[(int64_t)j * d.n + i] + C[(int64_t)(d.R + j) * d.n + i];
      }
      y = sc * yacc;
    } else {
      y = d.Yv[gi];
    }
    x.x += alpha * p.x;
    x.y += alpha * p.y;
    r.x -= alpha * (dd.x * p.x + y);
    r.y -= alpha * (dd.y * p.y - y);
    const float2 zz = precond2(dd, r, rho);
    v[0] += r.x * zz.x + r.y * zz.y;
    Xo[gi] = x;
    d.Rv[gi] = r;
  }
  block_partials<1>(v, d.part, j, d.nb, blk);
}

// one block of kT threads per column
__global__ void k_beta(Dev d, int k) {
  const int j = blockIdx.x;
  Col& c = d.col[j];
  if (!c.active) {
    if (threadIdx.x == 0) c.beta = 0.f;
    return;
  }
  const double rzn = block_col_total(d.part, j, d.nb, 0);
  if (threadIdx.x) return;
  c.pcg_iters += 1;
  const bool stop = !(rzn > d.prm.tol_pcg * d.prm.tol_pcg * c.rz0) || k >= d.prm.max_iter_pcg || !isfinite(rzn);
  c.beta = (float)(rzn / c.rz);
  c.rz = rzn;
  if (stop) c.active = 0;
  else atomicAdd(&d.counters[0], 1);
}

__global__ void k_pcg_E(Dev d) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  // a stopped column keeps its direction and its partials go unread; the bf16 path still
  // zeroes its GEMM input below
  if (!c.active && d.op != OP_SHARED_BF16) return;
  const float beta = c.beta, rho = (float)c.rho;
  float v[2] = {0.f, 0.f};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const float2 dd = d.Dv[gi], r = d.Rv[gi];
    float2 p = d.Pv[gi];
    if (c.active) {
      const float2 zz = precond2(dd, r, rho);
      p.x = zz.x + beta * p.x;
      p.y = zz.y + beta * p.y;
      d.Pv[gi] = p;
    } else {
      p = make_float2(0.f, 0.f);  // finished column: no further change
    }
    if (d.op == OP_SHARED_BF16) {
      const float w = p.x - p.y;
      const __nv_bfloat16 wh = __float2bfloat16_rn(w);
      d.W[(int64_t)j * d.n + i] = wh;
      d.W[(int64_t)(d.R + j) * d.n + i] = __float2bfloat16_rn(w - __bfloat162float(wh));
    }
    v[1] += dd.x * p.x * p.x + dd.y * p.y * p.y;
  }
  block_partials<2>(v, d.part, j, d.nb, blk);
}

// fraction-to-boundary ratios (reading R4)
__global__ void k_steps(Dev d, int corr) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  const Steer sc = steer(c, d.prm.sigma3, corr);
  float v[2] = {INFINITY, INFINITY};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const St st = load_st(d.zs, gi);
    const float2 x1 = d.X1[gi];
    const float2 x2 = corr ? d.X2[gi] : make_float2(0.f, 0.f);
    const D2 du = dirn(st.u.hi, st.su.hi, x1.x, x2.x, sc);
    const D2 dv = dirn(st.v.hi, st.sv.hi, x1.y, x2.y, sc);
    // ratios in float32: eta < 1 leaves a margin far above their rounding
    if (du.dz < 0.f) v[0] = fminf(v[0], -st.u.hi * __frcp_rn(du.dz));
    if (dv.dz < 0.f) v[0] = fminf(v[0], -st.v.hi * __frcp_rn(dv.dz));
    if (du.ds < 0.f) v[1] = fminf(v[1], -st.su.hi * __frcp_rn(du.ds));
    if (dv.ds < 0.f) v[1] = fminf(v[1], -st.sv.hi * __frcp_rn(dv.ds));
  }
  block_minima<2>(v, d.part, j, d.nb, blk);
}

// one block of kT threads per column
__global__ void k_steps_fin(Dev d, int corr) {
  const int j = blockIdx.x;
  Col& c = d.col[j];
  if (c.done) {
    if (threadIdx.x == 0) {
      c.alpha_p = c.alpha_d = 0.0;
      c.corr_next = 0;
    }
    return;
  }
  if (corr && !c.corr_next) return;  // keeps its predictor steps
  const double rp = block_col_total(d.part, j, d.nb, 0, true), rd = block_col_total(d.part, j, d.nb, 1, true);
  if (threadIdx.x) return;
  double ap = fmin(1.0, d.prm.eta * rp);
  double ad = fmin(1.0, d.prm.eta * rd);
  if (d.prm.equal_steps) ap = ad = fmin(ap, ad);
  c.alpha_p = ap;
  c.alpha_d = ad;
  if (!corr) {
    c.corr_next = (ap <= d.prm.alpha_tilde || ad <= d.prm.alpha_tilde);
    if (c.corr_next) {
      c.alpha_p1 = ap;
      c.alpha_d1 = ad;
      ++c.correctors;
      atomicAdd(&d.counters[2], 1);
    }
  } else {
    c.corr = 1;
  }
  c.prev_ap = ap;
  c.prev_ad = ad;
}

// trial point x~ = z~_u - z~_v of the corrector columns; partial z~.s~
__global__ void k_trial(Dev d) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  const Steer sc = steer(c, d.prm.sigma3, false);
  const df ap1 = to_df(c.alpha_p1), ad1 = to_df(c.alpha_d1);
  float a = 0.f;
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const St st = load_st(d.zs, gi);
    const float2 x1 = d.X1[gi];
    const D2 du = dirn(st.u.hi, st.su.hi, x1.x, 0.f, sc);
    const D2 dv = dirn(st.v.hi, st.sv.hi, x1.y, 0.f, sc);
    const df zu = axpy(st.u, ap1, du.dz), zv = axpy(st.v, ap1, dv.dz);
    const df su = axpy(st.su, ad1, du.ds), sv = axpy(st.sv, ad1, dv.ds);
    d.X[gi] = f2(zu - zv);
    a += zu.hi * su.hi + zv.hi * sv.hi;
  }
  const float v[1] = {a};
  block_partials<1>(v, d.part, j, d.nb, blk);
}

// one block of kT threads per column
__global__ void k_mu_t(Dev d) {
  const int j = blockIdx.x;
  Col& c = d.col[j];
  if (c.corr_next) {
    const double zts = block_col_total(d.part, j, d.nb, 0);
    if (threadIdx.x) return;
    c.mu_t = zts / (2.0 * d.n);
    c.nmat += 2;
  }
}

// ||c||: with x = 0 the residual kernel gives Gr = -A^T b
// one block of kT threads per column
__global__ void k_setup_cols(Dev d, const double* __restrict__ taus, const double* __restrict__ rhos) {
  const int j = blockIdx.x;
  const double atb2 = block_col_total(d.part, j, d.nb, 0);
  if (threadIdx.x) return;
  Col c{};
  c.tau = taus[j];
  c.rho = rhos ? rhos[j] : d.rho;
  c.alpha_p = c.alpha_d = c.prev_ap = c.prev_ad = 1.0;
  c.cn = sqrt(2.0 * d.n * c.tau * c.tau + 2.0 * atb2);
  c.nmat = 1;
  d.col[j] = c;
}

// the float32-grade residual errs by ~1e-6 ||A^T b||_inf: counters[4] counts the columns
// with tau < 1e-3 ||A^T b||_inf, for which it must not be used (Gr = -A^T b at this point)
__global__ void k_lowp_gate(Dev d) {
  __shared__ float red[33];
  const int j = blockIdx.x;
  float mx = 0.f;
  for (int i = threadIdx.x; i < d.n; i += blockDim.x) mx = fmaxf(mx, fabsf(d.Gr[(int64_t)j * d.n + i].x));
  mx = block_max(mx, red);
  if (threadIdx.x == 0 && !(d.col[j].tau >= 1e-3 * (double)mx)) atomicAdd(&d.counters[4], 1);
}

// outputs in natural order and the float64 certificates (Gr holds the final residual)
__global__ void k_exit(Dev d, double* const* __restrict__ xout, double* const* __restrict__ zsout) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const double tau = d.col[j].tau;
  double v[3] = {0, 0, 0};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const St q = load_st(d.zs, gi);
    const double zp[4] = {to_double(q.u), to_double(q.v), to_double(q.su), to_double(q.sv)};
    const double g = to_double(d2(d.Gr[gi]));
    const double fzu = zp[2] - (tau + g), fzv = zp[3] - (tau - g);
    const double x = to_double(q.u - q.v);
    const double y = x - g;
    const double st = copysign(fmax(fabs(y) - tau, 0.0), y);
    v[0] += fzu * fzu + fzv * fzv;
    v[1] += (x - st) * (x - st);
    v[2] += x * x;
    xout[j][i] = x;
    if (zsout && zsout[j]) {
      zsout[j][i] = zp[0];
      zsout[j][d.n + i] = zp[1];
      zsout[j][2 * d.n + i] = zp[2];
      zsout[j][3 * d.n + i] = zp[3];
    }
  }
  block_partials<3>(v, d.part, j, d.nb, blk);
}

// one block of kT threads per column
__global__ void k_info(Dev d, mfipm_info* infos) {
  const int j = blockIdx.x;
  const Col& c = d.col[j];
  const double fz2 = block_col_total(d.part, j, d.nb, 0), kk2 = block_col_total(d.part, j, d.nb, 1),
               x2 = block_col_total(d.part, j, d.nb, 2);
  if (threadIdx.x) return;
  mfipm_info info{};
  info.ipm_iters = c.ipm_iters;
  info.correctors = c.correctors;
  info.pcg_iters = c.pcg_iters;
  info.n_mat = c.nmat;
  info.rel_gap = c.rel_gap;
  info.dual_res = sqrt(fz2) / (1.0 + c.cn);
  info.kkt_rel = sqrt(kk2) / (1.0 + sqrt(x2));
  // converged: the gap test (reading R7) and a KKT residual of x within sqrt(tol)
  info.status = c.done ? c.stop : MFIPM_NOT_CONVERGED;
  if (info.status == MFIPM_OK && !(info.kkt_rel <= sqrt(d.prm.tol))) info.status = MFIPM_NOT_CONVERGED;
  info.primal_obj = c.P_obj;
  infos[j] = info;
}

}  // namespace mr

// ------------------------------------------------------------------ host orchestration
namespace {
int slice_splits(int64_t K) { return (int)(((K + 63) / 64 + 15) / 16); }  // chunks of <= 1024 = 16 x 64
size_t tc_resid_cbuf(int64_t m, int64_t n) {
  return (size_t)std::max<int64_t>(slice_splits(n) * m, slice_splits(m) * n) * 256 * 4;
}
size_t tc_resid_bytes(int64_t m, int64_t n, int R) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int64_t mx = std::max(m, n);
  return al((size_t)mr::kSlA * m * n * 2) * 2 + al((size_t)mr::kSlX * R * mx * 2) + al(tc_resid_cbuf(m, n)) +
         al((size_t)R * mx * 8) + al((size_t)(m + n) * 4) + al((size_t)R * 8);
}
}  // namespace

bool mrhs_resid_tc_supported(int64_t m, int64_t n, int R) {
  return R >= 1 && R <= 256 && m % 8 == 0 && n % 8 == 0 && tc_gemm_supported((int)m, R, (int)n) &&
         tc_gemm_supported((int)n, R, (int)m);
}

size_t mrhs_workspace_bytes(int64_t m, int64_t n, int R) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int nb = (int)((n + mr::kIdx - 1) / mr::kIdx);
  size_t b = 0;
  b += al((size_t)n * m * 2);             // At
  b += al((size_t)R * n * 8) * 2;         // X, Gr
  b += al((size_t)R * m * 8) * 2;         // Rr, Bm
  b += al((size_t)R * n * 32);            // zs
  b += al((size_t)R * n * 8) * 5;         // PCG pairs
  b += al((size_t)2 * R * n * 2);         // W
  b += al((size_t)2 * R * m * 2);         // Tb
  b += al((size_t)kMaxSplits * 2 * R * m * 4);  // C1
  b += al((size_t)kMaxSplits * 2 * R * n * 4);  // C2
  b += al((size_t)R * nb * mr::kPart * 8) * 2;  // part, part2
  b += al(sizeof(Col) * R);
  b += al(256);                           // counters
  b += al((size_t)R * 8) * 3;             // taus, b / x / zs pointer arrays
  b += al(sizeof(void*) * R);
  b += al((size_t)R * m * 8);                                              // Rf
  b += al((size_t)mr::kMaxRsplit * m * 4) + al((size_t)mr::kMaxRsplit * n * 4);  // row bounds
  b += al((size_t)mr::kMaxRsplit * R * 4) * 2;                             // column bounds
  if (mrhs_resid_tc_supported(m, n, R)) b += tc_resid_bytes(m, n, R);
  return b;
}

namespace {
// kernels launched by the last lockstep solve on this thread (reported with the operator timing)
thread_local int64_t g_nlaunch = 0;

// split count S <= cap (and <= K tiles) whose tiles * S blocks fill whole waves best
int pick_rsplit(int64_t tiles, int ktiles, int64_t slots, int cap) {
  cap = std::max(1, std::min(cap, ktiles));
  int best = 1;
  double best_eff = 0.0;
  for (int S = 1; S <= cap; ++S) {
    const int64_t blocks = tiles * S, waves = (blocks + slots - 1) / slots;
    const double eff = (double)blocks / (double)(waves * slots);
    if (eff > best_eff + 1e-9) {
      best = S;
      best_eff = eff;
    }
  }
  return best;
}
int mr_fail(cudaError_t e, std::string* msg, const char* where) {
  *msg = std::string(where) + ": " + cudaGetErrorString(e);
  return MFIPM_CUDA;
}

// The single-corrector IPM of Sec. 5.1 for all R problems in lockstep, each with its own
// scalars.  residual(gate, lowp) computes Gr = A^T (A X - b) and part2 slot 0 = ||A X - b||^2
// (lowp: by the float32-grade chain of the large-gap iterations, reading R17, where the
// operator has one; allow_lowp says so); normal(k, nprob) computes A^T A (p_u - p_v) for PCG
// iteration k (nprob: problems it covers) and part2 slot 0 = ||A w||^2.
template <class Resid, class Normal>
int lockstep_run(mr::Dev& d, double* part2, const double* taus, const double* rhos, Resid& residual, Normal& normal,
                 double* const* xptr, double* const* zptr, mfipm_info* infos, cudaStream_t st, std::string* msg,
                 bool allow_lowp = false) {
  using namespace mr;
  const int R = d.R, nb = d.nb;
  const dim3 gIdx(nb, R);
  cudaError_t e;
  int live = R, active = R;  // problems covered by the next operator product (host view)
  // The host reads the active count (one stream synchronisation) only from half the
  // iteration count at which the previous PCG solve of the same kind (predictor, corrector)
  // ended; the iterations launched before that without a check change nothing for problems
  // that have stopped (every pass skips them, their alpha and beta are 0), and a solve that
  // ends sooner than half its predecessor wastes at most those launches.
  int prev_iters[2] = {0, 0};
  auto pcg = [&](float2* Xo) -> cudaError_t {
    const int kind = Xo == d.X1 ? 0 : 1;
    const int first_check = prev_iters[kind] / 2;
    for (int k = 0;; ++k) {
      if ((e = normal(k, k == 0 ? live : active))) return e;
      k_alpha<<<R, kT, 0, st>>>(d, k == 0, part2);
      ++g_nlaunch;
      k_pcg_D<<<gIdx, kT, 0, st>>>(d, Xo, k == 0);
      ++g_nlaunch;
      if ((e = cudaMemsetAsync(d.counters, 0, 4, st))) return e;
      k_beta<<<R, kT, 0, st>>>(d, k + 1);
      ++g_nlaunch;
      if (k + 1 >= first_check || k + 1 >= d.prm.max_iter_pcg) {
        active = 0;
        if ((e = cudaMemcpyAsync(&active, d.counters, 4, cudaMemcpyDeviceToHost, st))) return e;
        if ((e = cudaStreamSynchronize(st))) return e;
        if (active == 0) {
          prev_iters[kind] = k + 1;
          return cudaSuccess;
        }
      }
      k_pcg_E<<<gIdx, kT, 0, st>>>(d);
      ++g_nlaunch;
    }
  };

  // setup: ||A^T b|| for ||c||
  if ((e = cudaMemsetAsync(d.X, 0, (size_t)R * d.n * 8, st))) return mr_fail(e, msg, "clear x");
  if ((e = residual(GATE_ALL, false))) return mr_fail(e, msg, "residual");
  k_colnorm2_df<<<gIdx, kT, 0, st>>>(d.Gr, d.n, d.part, nb);
  ++g_nlaunch;
  k_setup_cols<<<R, kT, 0, st>>>(d, taus, rhos);
  ++g_nlaunch;
  // the float32-grade residual while every problem's gap exceeds f32_gap, if every problem
  // passes its gate (tau >= 1e-3 ||A^T b||_inf); from the first iterate at or below it, and
  // before any stop, the residual is recomputed in full precision, which later iterations keep
  bool lowp = false;
  if (allow_lowp && d.prm.f32_gap > 0.0) {
    int failing = 0;
    if ((e = cudaMemsetAsync(d.counters + 4, 0, 4, st))) return mr_fail(e, msg, "counters");
    k_lowp_gate<<<R, kT, 0, st>>>(d);
    ++g_nlaunch;
    if ((e = cudaMemcpyAsync(&failing, d.counters + 4, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return mr_fail(e, msg, "residual gate");
    lowp = failing == 0;
  }
  for (int it = 1;; ++it) {
    k_update<<<gIdx, kT, 0, st>>>(d, it == 1);
    ++g_nlaunch;
    int unfinished = 0;
    for (;;) {
      if ((e = residual(GATE_LIVE, lowp))) return mr_fail(e, msg, "residual");
      if ((e = cudaMemsetAsync(d.counters, 0, 16, st))) return mr_fail(e, msg, "counters");
      k_stats<<<R, kT, 0, st>>>(d, it, part2, lowp ? 1 : 0);
      ++g_nlaunch;
      int cnt[3] = {0, 0, 0};  // unfinished, corrector columns, full precision needed
      if ((e = cudaMemcpyAsync(cnt, d.counters + 1, 12, cudaMemcpyDeviceToHost, st)) ||
          (e = cudaStreamSynchronize(st)))
        return mr_fail(e, msg, "gap test");
      unfinished = cnt[0];
      if (!(lowp && cnt[2] > 0)) break;
      lowp = false;  // this iterate's residual again, in full precision
    }
    if (unfinished == 0) break;
    live = unfinished;
    k_pcg_init<<<gIdx, kT, 0, st>>>(d, 0);
    ++g_nlaunch;
    if ((e = pcg(d.X1))) return mr_fail(e, msg, "predictor PCG");
    k_steps<<<gIdx, kT, 0, st>>>(d, 0);
    ++g_nlaunch;
    k_steps_fin<<<R, kT, 0, st>>>(d, 0);
    ++g_nlaunch;
    int ncorr = 0;
    if ((e = cudaMemcpyAsync(&ncorr, d.counters + 2, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return mr_fail(e, msg, "step lengths");
    if (ncorr > 0) {
      k_trial<<<gIdx, kT, 0, st>>>(d);
      ++g_nlaunch;
      k_mu_t<<<R, kT, 0, st>>>(d);
      ++g_nlaunch;
      if ((e = residual(GATE_LIVE, lowp))) return mr_fail(e, msg, "trial residual");
      k_pcg_init<<<gIdx, kT, 0, st>>>(d, 1);
      ++g_nlaunch;
      if ((e = pcg(d.X2))) return mr_fail(e, msg, "corrector PCG");
      k_steps<<<gIdx, kT, 0, st>>>(d, 1);
      ++g_nlaunch;
      k_steps_fin<<<R, kT, 0, st>>>(d, 1);
      ++g_nlaunch;
    }
  }
  k_exit<<<gIdx, kT, 0, st>>>(d, xptr, zptr);
  ++g_nlaunch;
  k_info<<<R, kT, 0, st>>>(d, infos);
  ++g_nlaunch;
  if ((e = cudaGetLastError())) return mr_fail(e, msg, "exit");
  return MFIPM_OK;
}
}  // namespace

int mrhs_solve(const MrhsCall& call, std::string* msg) {
  using namespace mr;
  const int64_t m = call.m, n = call.n;
  const int R = call.R;
  cudaStream_t st = call.stream;
  char* ws = static_cast<char*>(call.workspace);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const int nb = (int)((n + kIdx - 1) / kIdx);
  Dev d{};
  d.m = (int)m;
  d.n = (int)n;
  d.R = R;
  d.nb = nb;
  d.op = OP_SHARED_BF16;
  d.nb2 = nb;
  d.a_scale = call.a_scale;
  d.A = static_cast<const __nv_bfloat16*>(call.A);
  d.lda = call.lda;
  d.prm = call.prm;
  size_t o = 0;
  auto take = [&](size_t bytes) { char* p = ws + o; o += al(bytes); return p; };
  __nv_bfloat16* At = reinterpret_cast<__nv_bfloat16*>(take((size_t)n * m * 2));
  d.At = At;
  d.X = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.Gr = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.Rr = reinterpret_cast<double*>(take((size_t)R * m * 8));
  d.Bm = reinterpret_cast<double*>(take((size_t)R * m * 8));
  d.zs = reinterpret_cast<float4*>(take((size_t)R * n * 32));
  d.X1 = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.X2 = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.Rv = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.Pv = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.Dv = reinterpret_cast<float2*>(take((size_t)R * n * 8));
  d.W = reinterpret_cast<__nv_bfloat16*>(take((size_t)2 * R * n * 2));
  d.Tb = reinterpret_cast<__nv_bfloat16*>(take((size_t)2 * R * m * 2));
  d.C1 = reinterpret_cast<float*>(take((size_t)kMaxSplits * 2 * R * m * 4));
  d.C2 = reinterpret_cast<float*>(take((size_t)kMaxSplits * 2 * R * n * 4));
  d.s1 = std::min(call.splits1, kMaxSplits);
  d.s2 = std::min(call.splits2, kMaxSplits);
  d.part = reinterpret_cast<double*>(take((size_t)R * nb * kPart * 8));
  double* part2 = reinterpret_cast<double*>(take((size_t)R * nb * kPart * 8));
  d.col = reinterpret_cast<Col*>(take(sizeof(Col) * R));
  d.counters = reinterpret_cast<int*>(take(256));
  double* taus = reinterpret_cast<double*>(take((size_t)R * 8));
  const double** bptr = reinterpret_cast<const double**>(take((size_t)R * 8));
  double** xptr = reinterpret_cast<double**>(take((size_t)R * 8));
  double** zptr = reinterpret_cast<double**>(take(sizeof(void*) * R));
  float2* Rf = reinterpret_cast<float2*>(take((size_t)R * m * 8));
  float* rp1 = reinterpret_cast<float*>(take((size_t)kMaxRsplit * m * 4));
  float* rp2 = reinterpret_cast<float*>(take((size_t)kMaxRsplit * n * 4));
  float* cp1 = reinterpret_cast<float*>(take((size_t)kMaxRsplit * R * 4));
  float* cp2 = reinterpret_cast<float*>(take((size_t)kMaxRsplit * R * 4));
  const bool rtc = call.resid_tc && mrhs_resid_tc_supported(m, n, R);
  __nv_bfloat16 *SA = nullptr, *SAt = nullptr, *XS = nullptr;
  float* Cb = nullptr;
  float2* Acc = nullptr;
  int *EA = nullptr, *EAt = nullptr, *Ex1 = nullptr, *Ex2 = nullptr;
  if (rtc) {
    const int64_t mx = std::max(m, n);
    SA = reinterpret_cast<__nv_bfloat16*>(take((size_t)kSlA * m * n * 2));
    SAt = reinterpret_cast<__nv_bfloat16*>(take((size_t)kSlA * m * n * 2));
    XS = reinterpret_cast<__nv_bfloat16*>(take((size_t)kSlX * R * mx * 2));
    Cb = reinterpret_cast<float*>(take(tc_resid_cbuf(m, n)));
    Acc = reinterpret_cast<float2*>(take((size_t)R * mx * 8));
    EA = reinterpret_cast<int*>(take((size_t)(m + n) * 4));
    EAt = EA + m;
    Ex1 = reinterpret_cast<int*>(take((size_t)R * 8));
    Ex2 = Ex1 + R;
  }
  if (o > call.ws_bytes) {
    *msg = "workspace too small for the shared-A solver";
    return MFIPM_INVALID_ARG;
  }
  cudaError_t e;
  std::vector<void*> hz(R, nullptr);
  for (int j = 0; j < R; ++j) hz[j] = call.zs_out ? call.zs_out[j] : nullptr;
  if ((e = cudaMemcpyAsync(taus, call.tau, R * 8, cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(bptr, call.b, R * sizeof(void*), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(xptr, call.x, R * sizeof(void*), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(zptr, hz.data(), R * sizeof(void*), cudaMemcpyHostToDevice, st)))
    return mr_fail(e, msg, "upload arguments");
  // d.prm.rho: the Frobenius-closest multiple of I to A^T A (reading R2) is supplied by the caller
  d.rho = call.rho;

  transpose_bf16<<<dim3((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32)), dim3(32, 8), 0, st>>>(d.A, d.lda, At,
                                                                                                   (int)m, (int)n);
  gather_b<<<dim3(8, R), 256, 0, st>>>(bptr, d.Bm, (int)m);
  if ((e = cudaGetLastError())) return mr_fail(e, msg, "setup kernels");

  // residual GEMM splits: fill whole waves of resident blocks
  int sms = 0, occ = 0, dev = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, resid_gemm, 256, 0)))
    return mr_fail(e, msg, "residual occupancy");
  const int64_t slots = (int64_t)sms * std::max(occ, 1);
  const int64_t part_cap = (int64_t)kMaxSplits * 2 * R * n * 4;  // bytes of C2, reused for the partials
  const int jt = (R + kJB - 1) / kJB;
  const int S1 = pick_rsplit((int64_t)((m + kRB - 1) / kRB) * jt, (int)((n + kKB - 1) / kKB), slots,
                             (int)std::min<int64_t>(kMaxRsplit, part_cap / ((int64_t)R * m * 8)));
  const int S2 = pick_rsplit((int64_t)((n + kRB - 1) / kRB) * jt, (int)((m + kKB - 1) / kKB), slots,
                             (int)std::min<int64_t>(kMaxRsplit, part_cap / ((int64_t)R * n * 8)));
  float2* Part = reinterpret_cast<float2*>(d.C2);
  const bool vecA1 = (reinterpret_cast<uintptr_t>(d.A) & 15) == 0 && d.lda % 8 == 0;
  const bool vecA2 = m % 8 == 0;
  k_rowpow<<<(unsigned)(((int64_t)m * S1 * 32 + 255) / 256), 256, 0, st>>>(d.A, d.lda, (int)m, (int)n, S1, rp1);
  k_rowpow<<<(unsigned)(((int64_t)n * S2 * 32 + 255) / 256), 256, 0, st>>>(At, m, (int)n, (int)m, S2, rp2);
  g_nlaunch += 4;  // transpose, gather of b, two row-bound passes
  if ((e = cudaGetLastError())) return mr_fail(e, msg, "row bounds");

  auto residual = [&]() -> cudaError_t {
    // Rr = a_scale A X - B ; Gr = a_scale A^T Rr
    k_xbound<<<dim3(S1, R), 256, 0, st>>>(d.X, cp1, (int)n, R, S1);
    resid_gemm<<<dim3((unsigned)((m + kRB - 1) / kRB), jt, S1), 256, 0, st>>>(d.A, d.lda, rp1, d.X, cp1, Part, (int)m,
                                                                            R, (int)n, S1, vecA1);
    k_fin1<<<dim3(S2, R), 256, 0, st>>>(Part, S1, d.Bm, d.a_scale, d.Rr, Rf, cp2, (int)m, R, S2);
    resid_gemm<<<dim3((unsigned)((n + kRB - 1) / kRB), jt, S2), 256, 0, st>>>(At, m, rp2, Rf, cp2, Part, (int)n, R,
                                                                            (int)m, S2, vecA2);
    k_fin2<<<(unsigned)std::min<int64_t>(((int64_t)R * n + 255) / 256, 4096), 256, 0, st>>>(Part, S2, d.a_scale,
                                                                                           d.Gr, (int)n, R);
    k_colnorm2<<<dim3(nb, R), kT, 0, st>>>(d.Rr, (int)m, part2, nb);
    g_nlaunch += 6;
    return cudaGetLastError();
  };
  auto normal = [&](int, int) -> cudaError_t {
    g_nlaunch += 3;
    e = call.gemm(call.gemm_ctx, d.A, d.W, d.C1, (int)m, 2 * R, (int)n, d.s1, st, call.stages1);
    if (e) return e;
    k_split_t<<<dim3(nb, R), kT, 0, st>>>(d, part2);
    e = call.gemm(call.gemm_ctx, At, d.Tb, d.C2, (int)n, 2 * R, (int)m, d.s2, st, call.stages2);
    if (e) return e;
    return cudaGetLastError();
  };
  // the same residual by exact digit slices on the tensor cores (slices of A and A^T once)
  if (rtc) {
    k_slice_rows<<<(unsigned)m, 256, 0, st>>>(d.A, d.lda, (int)m, (int)n, SA, EA);
    k_slice_rows<<<(unsigned)n, 256, 0, st>>>(At, m, (int)n, (int)m, SAt, EAt);
    g_nlaunch += 2;
    if ((e = cudaGetLastError())) return mr_fail(e, msg, "digit slices of A");
  }
  const int per_call = std::max(1, 256 / R);  // x slices per GEMM (N = slices x R <= 256)
  auto slice_product = [&](const __nv_bfloat16* S, const int* Er, int rows, int K, const int* Ej) -> cudaError_t {
    const int splits = slice_splits(K);
    const unsigned ga = (unsigned)std::min<int64_t>(((int64_t)R * rows + 255) / 256, 4096);
    bool first = true;
    for (int t = 0; t < kSlA; ++t) {
      const int smax = std::min(kSlX - 1, kPairMax - t);
      for (int s0 = 0; s0 <= smax; s0 += per_call) {
        const int c = std::min(per_call, smax - s0 + 1);
        cudaError_t r = tc_gemm(S + (size_t)t * rows * K, XS + (size_t)s0 * R * K, Cb, rows, c * R, K, splits,
                                call.err_dev, st);
        if (r) return r;
        k_slice_acc<<<ga, 256, 0, st>>>(Cb, splits, c, R, rows, t, s0, Er, Ej, Acc, first ? 1 : 0);
        first = false;
        g_nlaunch += 2;
      }
    }
    return cudaGetLastError();
  };
  auto residual_tc = [&]() -> cudaError_t {
    const unsigned g1 = (unsigned)std::min<int64_t>(((int64_t)R * m + 255) / 256, 4096);
    const unsigned g2 = (unsigned)std::min<int64_t>(((int64_t)R * n + 255) / 256, 4096);
    cudaError_t r;
    k_slice_cols<float2><<<R, 256, 0, st>>>(d.X, R, (int)n, XS, Ex1);
    if ((r = slice_product(SA, EA, (int)m, (int)n, Ex1))) return r;
    k_fin1_tc<<<g1, 256, 0, st>>>(Acc, d.Bm, d.a_scale, d.Rr, (int64_t)R * m);
    k_slice_cols<double><<<R, 256, 0, st>>>(d.Rr, R, (int)m, XS, Ex2);
    if ((r = slice_product(SAt, EAt, (int)n, (int)m, Ex2))) return r;
    k_fin2_tc<<<g2, 256, 0, st>>>(Acc, d.a_scale, d.Gr, (int64_t)R * n);
    k_colnorm2<<<dim3(nb, R), kT, 0, st>>>(d.Rr, (int)m, part2, nb);
    g_nlaunch += 5;
    return cudaGetLastError();
  };
  // the large-gap residual: A x and A^T r with x and r as three bf16 pieces (tensor cores,
  // float32 sums), split-K capped by the chunk-sum buffer
  auto residual_lowp = [&]() -> cudaError_t {
    const size_t cap = tc_resid_cbuf(m, n);
    auto fit = [&](int sp, int64_t rows) {
      const int64_t lim = (int64_t)(cap / ((size_t)3 * R * rows * 4));
      return (int)std::max<int64_t>(1, std::min<int64_t>(sp, lim));
    };
    const int sa = fit(d.s1, m), sb = fit(d.s2, n);
    const unsigned gm = (unsigned)std::min<int64_t>(((int64_t)R * m + 255) / 256, 4096);
    const unsigned gn = (unsigned)std::min<int64_t>(((int64_t)R * n + 255) / 256, 4096);
    cudaError_t r;
    k_pieces_x<<<gn, 256, 0, st>>>(d.X, R, (int)n, XS);
    if ((r = call.gemm(call.gemm_ctx, d.A, XS, Cb, (int)m, 3 * R, (int)n, sa, st, call.stages1))) return r;
    k_pieces_mid<<<gm, 256, 0, st>>>(Cb, sa, R, (int)m, d.Bm, d.a_scale, d.Rr, XS);
    if ((r = call.gemm(call.gemm_ctx, At, XS, Cb, (int)n, 3 * R, (int)m, sb, st, call.stages2))) return r;
    k_pieces_fin<<<gn, 256, 0, st>>>(Cb, sb, R, (int)n, d.a_scale, d.Gr);
    k_colnorm2<<<dim3(nb, R), kT, 0, st>>>(d.Rr, (int)m, part2, nb);
    g_nlaunch += 6;
    return cudaGetLastError();
  };
  // the pieces need the digit-slice buffers and N = 3R <= 256 for one GEMM
  const bool lowp_ok = rtc && 3 * R <= 256 && tc_gemm_supported((int)m, 3 * R, (int)n) &&
                       tc_gemm_supported((int)n, 3 * R, (int)m);
  auto resid = [&](int, bool lowp) -> cudaError_t {
    if (lowp) return residual_lowp();
    return rtc ? residual_tc() : residual();
  };
  return lockstep_run(d, part2, taus, nullptr, resid, normal, xptr, zptr, call.infos_dev, st, msg, lowp_ok);
}

// ------------------------------------------------------------------ large partial DCT
namespace mr {
// adjoint solve H y = [g_x; -g_x] at the forward solution's final iterate (the derivative of
// the perturbed KKT system of Eq. fzfs at fixed mu): Theta^-1 = s / z, y0 = 0
__global__ void k_bwd_init(Dev d, const double* const* __restrict__ zs_in, const double* const* __restrict__ gx) {
  const int j = blockIdx.y, blk = blockIdx.x;
  const Col& c = d.col[j];
  const double* z = zs_in[j];
  double v[2] = {0, 0};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const double u = z[i], vv = z[d.n + i], su = z[2 * (int64_t)d.n + i], sv = z[3 * (int64_t)d.n + i];
    const float2 dd = make_float2((float)(su / u), (float)(sv / vv));
    const float g = (float)gx[j][i];
    const float2 r = make_float2(g, -g);
    const float2 p = precond2(dd, r, (float)c.rho);
    d.Dv[gi] = dd;
    d.Rv[gi] = r;
    d.Pv[gi] = p;
    v[0] += (double)(r.x * p.x + r.y * p.y);
    v[1] += (double)(dd.x * p.x * p.x + dd.y * p.y * p.y);
  }
  block_partials<2>(v, d.part, j, d.nb, blk);
}
__global__ void k_bwd_cols(Dev d, const double* __restrict__ rhos) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.R) return;
  Col c{};
  c.rho = rhos[j];
  d.col[j] = c;
}
// w = y_u - y_v (float64) for the forward transform, and sum(y_u + y_v)
__global__ void k_bwd_w(Dev d) {
  const int j = blockIdx.y, blk = blockIdx.x;
  double v[1] = {0.0};
  for (int i = blk * kIdx + threadIdx.x; i < min(d.n, (blk + 1) * kIdx); i += kT) {
    const int64_t gi = (int64_t)j * d.n + i;
    const float2 y = d.X1[gi];
    const df w = df_two_sum(y.x, -y.y);  // exact
    d.X[gi] = make_float2(w.hi, w.lo);
    v[0] += (double)y.x + (double)y.y;
  }
  block_partials<1>(v, d.part, j, d.nb, blk);
}
// grad_b = A w = (C w)[rows], grad_tau = -sum(y_u + y_v), info
__global__ void k_bwd_out(Dev d, const int64_t* const* __restrict__ rows, const int64_t* __restrict__ ms,
                          double* const* __restrict__ grad_b, double* __restrict__ gtau, mfipm_info* infos) {
  const int j = blockIdx.y;
  const int64_t m = ms[j];
  double* gb = grad_b[j];
  if (gb)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
      gb[i] = reinterpret_cast<const double*>(d.Gr)[(int64_t)j * d.n + rows[j][i]];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const Col& c = d.col[j];
    gtau[j] = -col_total(d.part, j, d.nb, 0);
    mfipm_info info{};
    info.status = MFIPM_OK;
    info.pcg_iters = c.pcg_iters;
    info.n_mat = c.nmat + 1;
    infos[j] = info;
  }
}
}  // namespace mr

namespace {
// Device time of the multi-pass operator products (mfipm_set_timing): CUDA events on the
// solve's stream around every A^T A w, read after the solve's final synchronisation.
struct OpTimer {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<double> units;  // problems x n per recorded product
  size_t used = 0;
  double ms = -1.0, bytes = 0.0;
  int64_t products = 0;
  cudaError_t begin(cudaStream_t st) {
    if (used + 2 > ev.size()) {
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r) return r;
        ev.push_back(e);
      }
    }
    return cudaEventRecord(ev[used], st);
  }
  cudaError_t end(cudaStream_t st, double u) {
    cudaError_t r = cudaEventRecord(ev[used + 1], st);
    used += 2;
    units.push_back(u);
    return r;
  }
  void reset() {
    used = 0;
    units.clear();
    ms = -1.0;
    bytes = 0.0;
    products = 0;
  }
  // after the stream has been synchronised; algorithmic bytes: w read and y written, 8 per index
  void collect() {
    if (!on) return;
    double t = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
      float x = 0.f;
      if (cudaEventElapsedTime(&x, ev[i], ev[i + 1]) == cudaSuccess) t += x;
    }
    ms = t;
    bytes = 0.0;
    for (double u : units) bytes += 8.0 * u;
    products = (int64_t)units.size();
  }
};
thread_local OpTimer g_optimer;

struct LdLayout {
  int nb, nb2;
  LdShape sh;
  int log2_tw;
  size_t total;
};
LdLayout ld_layout(int64_t n, int R) {
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  LdLayout L{};
  L.sh = ld_shape(n);
  L.nb = (int)((n + mr::kIdx - 1) / mr::kIdx);
  L.nb2 = 1 << (L.sh.logN1 - 1);
  L.log2_tw = L.sh.logN + 2;
  const size_t Rn = (size_t)R * n;
  size_t b = 0;
  b += al(Rn * 8) * 2;                  // X, Gr
  b += al(Rn * 32);                     // zs
  b += al(Rn * 8) * 5;                  // X1 X2 Rv Pv Dv
  b += al(Rn * 4);                      // Yv
  b += al(Rn * 8);                      // intermediate (L double-float complex)
  b += al(Rn) + al(Rn * 8) * 2;         // mask, bsu, bsu_df
  b += al((size_t)R * std::max(L.nb, L.nb2) * mr::kPart * 8) * 2;  // part, part2
  b += al(sizeof(Col) * R) + al(256);   // col, counters
  b += al((size_t)R * 8) * 10;          // taus, rhos, ms, grad_tau, pointer arrays
  b += al(sizeof(ProbDesc) * R) + al(256);  // descriptors, error word
  b += al(((size_t)2 << L.log2_tw) * 8) + al(((size_t)2 << L.log2_tw) * 16);  // twiddles
  b += al((size_t)R * sizeof(mfipm_info));
  b += al(ld_mask_code_bytes(n, R));
  L.total = b;
  return L;
}

struct LdState {
  mr::Dev d;
  double* part2;
  double *taus, *rhos, *gtau;
  int64_t* ms;
  double **xptr, **zptr, **gbptr;
  const double **zinptr, **gxptr;
  const int64_t** rowsptr;
  mfipm_info* infos_dev;
  LdArgs base;
};

// carve the workspace, upload per-problem arguments, build mask / b_u and the twiddles
int ld_setup(const LdCall& call, LdState& S, std::string* msg) {
  using namespace mr;
  const int64_t n = call.n;
  const int R = call.R;
  cudaStream_t st = call.stream;
  const LdLayout L = ld_layout(n, R);
  if (call.ws_bytes < L.total) {
    *msg = "workspace too small for the multi-pass partial-DCT solver";
    return MFIPM_INVALID_ARG;
  }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* ws = static_cast<char*>(call.workspace);
  size_t o = 0;
  auto take = [&](size_t bytes) { char* p = ws + o; o += al(bytes); return p; };
  const size_t Rn = (size_t)R * n;
  Dev& d = S.d;
  d = Dev{};
  d.n = (int)n;
  d.R = R;
  d.nb = L.nb;
  d.nb2 = L.nb2;
  d.op = OP_LARGE_DCT;
  d.a_scale = 1.0;
  d.prm = call.prm;
  d.X = reinterpret_cast<float2*>(take(Rn * 8));
  d.Gr = reinterpret_cast<float2*>(take(Rn * 8));
  d.zs = reinterpret_cast<float4*>(take(Rn * 32));
  d.X1 = reinterpret_cast<float2*>(take(Rn * 8));
  d.X2 = reinterpret_cast<float2*>(take(Rn * 8));
  d.Rv = reinterpret_cast<float2*>(take(Rn * 8));
  d.Pv = reinterpret_cast<float2*>(take(Rn * 8));
  d.Dv = reinterpret_cast<float2*>(take(Rn * 8));
  d.Yv = reinterpret_cast<float*>(take(Rn * 4));
  void* inter = take(Rn * 8);
  uint8_t* mask = reinterpret_cast<uint8_t*>(take(Rn));
  double* bsu = reinterpret_cast<double*>(take(Rn * 8));
  float2* bsu_df = reinterpret_cast<float2*>(take(Rn * 8));
  const size_t partb = (size_t)R * std::max(L.nb, L.nb2) * kPart * 8;
  d.part = reinterpret_cast<double*>(take(partb));
  S.part2 = reinterpret_cast<double*>(take(partb));
  d.col = reinterpret_cast<Col*>(take(sizeof(Col) * R));
  d.counters = reinterpret_cast<int*>(take(256));
  S.taus = reinterpret_cast<double*>(take((size_t)R * 8));
  S.rhos = reinterpret_cast<double*>(take((size_t)R * 8));
  S.gtau = reinterpret_cast<double*>(take((size_t)R * 8));
  S.ms = reinterpret_cast<int64_t*>(take((size_t)R * 8));
  S.xptr = reinterpret_cast<double**>(take((size_t)R * 8));
  S.zptr = reinterpret_cast<double**>(take((size_t)R * 8));
  S.gbptr = reinterpret_cast<double**>(take((size_t)R * 8));
  S.zinptr = reinterpret_cast<const double**>(take((size_t)R * 8));
  S.gxptr = reinterpret_cast<const double**>(take((size_t)R * 8));
  S.rowsptr = reinterpret_cast<const int64_t**>(take((size_t)R * 8));
  ProbDesc* probs = reinterpret_cast<ProbDesc*>(take(sizeof(ProbDesc) * R));
  int* err = reinterpret_cast<int*>(take(256));
  float2* tw32 = reinterpret_cast<float2*>(take(((size_t)2 << L.log2_tw) * 8));
  float4* twdf = reinterpret_cast<float4*>(take(((size_t)2 << L.log2_tw) * 16));
  S.infos_dev = reinterpret_cast<mfipm_info*>(take((size_t)R * sizeof(mfipm_info)));
  uint8_t* mcode = reinterpret_cast<uint8_t*>(take(ld_mask_code_bytes(n, R)));

  std::vector<ProbDesc> desc(R);
  std::vector<double> rh(R), taus(R, 1.0);
  std::vector<const void*> xs(R, nullptr), zo(R, nullptr), gb(R, nullptr), zi(R, nullptr), gx(R, nullptr),
      rw(R, nullptr);
  for (int j = 0; j < R; ++j) {
    ProbDesc& pd = desc[j];
    memset(&pd, 0, sizeof(pd));
    pd.n = n;
    pd.m = call.m[j];
    pd.kind = MFIPM_OP_PARTIAL_DCT;
    pd.log2n = L.sh.logN;
    pd.b = call.b[j];
    pd.rows = call.rows[j];
    pd.mask = mask + (size_t)j * n;
    pd.bsu = bsu + (size_t)j * n;
    pd.bsu_df = bsu_df + (size_t)j * n;
    rh[j] = (double)call.m[j] / (double)n;  // reading R2: A A^T = I, ||A||_F^2 = m
    if (call.tau) taus[j] = call.tau[j];
    xs[j] = call.x ? call.x[j] : nullptr;
    zo[j] = call.zs_out ? call.zs_out[j] : nullptr;
    gb[j] = call.grad_b ? call.grad_b[j] : nullptr;
    zi[j] = call.zs_in ? call.zs_in[j] : nullptr;
    gx[j] = call.gx ? call.gx[j] : nullptr;
    rw[j] = call.rows[j];
  }
  cudaError_t e;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (!e) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  e = cudaSuccess;
  up(probs, desc.data(), sizeof(ProbDesc) * R);
  up(S.taus, taus.data(), (size_t)R * 8);
  up(S.rhos, rh.data(), (size_t)R * 8);
  up(S.ms, call.m, (size_t)R * 8);
  up(S.xptr, xs.data(), (size_t)R * 8);
  up(S.zptr, zo.data(), (size_t)R * 8);
  up(S.gbptr, gb.data(), (size_t)R * 8);
  up(S.zinptr, zi.data(), (size_t)R * 8);
  up(S.gxptr, gx.data(), (size_t)R * 8);
  up(S.rowsptr, rw.data(), (size_t)R * 8);
  if (e) return mr_fail(e, msg, "upload arguments");
  if ((e = cudaMemsetAsync(err, 0, 4, st)) || (e = cudaMemsetAsync(d.Yv, 0, Rn * 4, st)) ||
      (e = cudaMemsetAsync(S.part2, 0, partb, st)) ||
      (e = launch_twiddles(nullptr, tw32, twdf, L.log2_tw, st)) || (e = launch_dct_setup(probs, R, n, err, st)))
    return mr_fail(e, msg, "setup kernels");
  g_nlaunch += 3;
  int herr = 0;
  if ((e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
    return mr_fail(e, msg, "setup kernels");
  if (herr == -1) {
    *msg = "rows must be distinct, ascending and inside [0, n)";
    return MFIPM_INVALID_ARG;
  }
  if (herr == -2) {
    *msg = "b contains a non-finite value";
    return MFIPM_NUMERIC;
  }
  LdArgs& a = S.base;
  a = LdArgs{};
  a.logN = L.sh.logN;
  a.logL = L.sh.logL;
  a.logN1 = L.sh.logN1;
  a.logN2 = L.sh.logN2;
  a.log2_tw = L.log2_tw;
  a.col = d.col;
  a.inter = inter;
  a.mask = mask;
  a.bsu = bsu;
  a.bsu_df = bsu_df;
  a.part2 = S.part2;
  a.nb2 = L.nb2;
  a.kpart = kPart;
  a.tw32 = tw32;
  a.twdf = twdf;
  a.mcode = mcode;
  if ((e = ld_mask_codes(a, R, st))) return mr_fail(e, msg, "mask codes");
  ++g_nlaunch;
  return MFIPM_OK;
}

int ld_read_infos(const LdCall& call, const LdState& S, std::string* msg) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(call.infos, S.infos_dev, sizeof(mfipm_info) * call.R, cudaMemcpyDeviceToHost,
                           call.stream)) ||
      (e = cudaStreamSynchronize(call.stream)))
    return mr_fail(e, msg, "read infos");
  return MFIPM_OK;
}
}  // namespace

size_t large_dct_workspace_bytes(int64_t n, int R) { return ld_layout(n, R).total; }

int large_dct_solve(const LdCall& call, std::string* msg) {
  LdState S;
  int rc = ld_setup(call, S, msg);
  if (rc) return rc;
  mr::Dev& d = S.d;
  cudaStream_t st = call.stream;
  auto residual = [&](int gate, bool lowp) -> cudaError_t {
    LdArgs a = S.base;
    a.gate = gate;
    a.din = d.X;
    a.dout = d.Gr;
    g_nlaunch += 3;
    return lowp ? ld_resid_f32(a, d.R, st) : ld_resid(a, d.R, st);
  };
  OpTimer& T = g_optimer;
  T.reset();
  auto normal = [&](int k, int nprob) -> cudaError_t {
    LdArgs a = S.base;
    // the first product of a PCG solve precedes its activity test
    a.gate = k == 0 ? GATE_LIVE : GATE_ACTIVE;
    a.pin = d.Pv;
    a.yout = d.Yv;
    cudaError_t r;
    if (T.on && (r = T.begin(st))) return r;
    if ((r = ld_normal(a, d.R, st))) return r;
    g_nlaunch += 3;
    return T.on ? T.end(st, (double)nprob * (double)call.n) : cudaSuccess;
  };
  rc = lockstep_run(d, S.part2, S.taus, S.rhos, residual, normal, S.xptr, S.zptr, S.infos_dev, st, msg, true);
  if (rc) return rc;
  rc = ld_read_infos(call, S, msg);
  T.collect();
  return rc;
}

int large_dct_backward(const LdCall& call, std::string* msg) {
  using namespace mr;
  LdState S;
  int rc = ld_setup(call, S, msg);
  if (rc) return rc;
  Dev& d = S.d;
  // the derivative needs a tighter solve than a Newton direction
  d.prm.tol_pcg = std::min(d.prm.tol_pcg, 1e-6);
  cudaStream_t st = call.stream;
  const dim3 gIdx(d.nb, d.R);
  const int colBlocks = (d.R + 127) / 128;
  cudaError_t e;
  k_bwd_cols<<<colBlocks, 128, 0, st>>>(d, S.rhos);
  ++g_nlaunch;
  k_bwd_init<<<gIdx, kT, 0, st>>>(d, S.zinptr, S.gxptr);
  ++g_nlaunch;
  if ((e = cudaGetLastError())) return mr_fail(e, msg, "adjoint setup");
  // PCG as in the solve, with every problem live
  OpTimer& T = g_optimer;
  T.reset();
  int active = d.R;
  for (int k = 0;; ++k) {
    LdArgs a = S.base;
    a.gate = k == 0 ? GATE_ALL : GATE_ACTIVE;
    a.pin = d.Pv;
    a.yout = d.Yv;
    if (T.on && (e = T.begin(st))) return mr_fail(e, msg, "timing event");
    if ((e = ld_normal(a, d.R, st))) return mr_fail(e, msg, "adjoint PCG");
    g_nlaunch += 3;
    if (T.on && (e = T.end(st, (double)active * (double)call.n))) return mr_fail(e, msg, "timing event");
    k_alpha<<<d.R, kT, 0, st>>>(d, k == 0, S.part2);
    ++g_nlaunch;
    k_pcg_D<<<gIdx, kT, 0, st>>>(d, d.X1, k == 0);
    ++g_nlaunch;
    if ((e = cudaMemsetAsync(d.counters, 0, 4, st))) return mr_fail(e, msg, "adjoint PCG");
    k_beta<<<d.R, kT, 0, st>>>(d, k + 1);
    ++g_nlaunch;
    active = 0;
    if ((e = cudaMemcpyAsync(&active, d.counters, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return mr_fail(e, msg, "adjoint PCG");
    if (active == 0) break;
    k_pcg_E<<<gIdx, kT, 0, st>>>(d);
    ++g_nlaunch;
  }
  k_bwd_w<<<gIdx, kT, 0, st>>>(d);
  ++g_nlaunch;
  LdArgs a = S.base;
  a.gate = GATE_ALL;
  a.din = d.X;
  a.fwd = reinterpret_cast<double*>(d.Gr);  // the forward coefficients reuse Gr's memory
  if ((e = ld_forward(a, d.R, st))) return mr_fail(e, msg, "A w");
  g_nlaunch += 2;
  k_bwd_out<<<dim3(64, d.R), 256, 0, st>>>(d, S.rowsptr, S.ms, S.gbptr, S.gtau, S.infos_dev);
  ++g_nlaunch;
  if ((e = cudaGetLastError())) return mr_fail(e, msg, "adjoint outputs");
  if (call.grad_tau && (e = cudaMemcpyAsync(call.grad_tau, S.gtau, (size_t)d.R * 8, cudaMemcpyDeviceToHost, st)))
    return mr_fail(e, msg, "read grad_tau");
  rc = ld_read_infos(call, S, msg);
  T.collect();
  return rc;
}

void large_dct_set_timing(bool on) {
  g_optimer.on = on;
  g_optimer.reset();
}
void lockstep_stats_reset() {
  g_nlaunch = 0;
  g_optimer.reset();
}
void note_launches(int64_t n) { g_nlaunch += n; }

void large_dct_timing(double* ms, double* bytes, int64_t* products, int64_t* launches) {
  *ms = g_optimer.ms;
  *bytes = g_optimer.bytes;
  *products = g_optimer.products;
  *launches = g_nlaunch;
}

namespace mr {
__global__ void k_fro2(const __nv_bfloat16* __restrict__ A, int64_t m, int64_t n, int64_t lda, double* out) {
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * n; e += (int64_t)gridDim.x * blockDim.x) {
    const double a = bf(A[(e / n) * lda + e % n]);
    s += a * a;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}
}  // namespace mr

cudaError_t bf16_fro2(const void* A, int64_t m, int64_t n, int64_t lda, double* out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 8, st);
  if (e) return e;
  mr::k_fro2<<<1024, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(A), m, n, lda, out);
  ++g_nlaunch;
  return cudaGetLastError();
}

cudaError_t gemm_simple(void*, const void* Aop, const void* Bop, float* C, int rows, int N, int K, int splits,
                        cudaStream_t st, int) {
  if (splits != 1) return cudaErrorInvalidValue;
  mr::gemm_bf16_simple<<<dim3((unsigned)((rows + 63) / 64), (unsigned)((N + 63) / 64)), mr::kT, 0, st>>>(
      static_cast<const __nv_bfloat16*>(Aop), static_cast<const __nv_bfloat16*>(Bop), C, rows, N, K);
  return cudaGetLastError();
}

}  // namespace mfipm
