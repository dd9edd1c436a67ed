// Matrix-free products with A (the only use the method makes of A, Sec. 1) and the KKT
// residual of a candidate x, float64 in and out, behind mfipm_apply_A / mfipm_apply_At /
// mfipm_kkt_residual.
//   partial DCT, n >= 1024: the multi-pass chain of large_dct.cu in double-float:
//       A x     = (C x)[rows]                       (forward transform, rows gathered)
//       A^T y   = -(A^T (A 0 - y))                  (the residual chain at x = 0, b = y)
//       g(x)    = A^T (A x - b)                     (the residual chain)
//   partial DCT, n < 1024: direct sums with C[r][k] = a_r cos(pi r (2k + 1) / (2n));
//   dense (float64 or bf16 times a_scale): one warp per row (A x), one thread per column (A^T y).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "device_common.cuh"
#include "internal.h"
#include "large_dct.h"
#include "mrhs.h"

namespace mfipm {
namespace ap {

constexpr int kT = 256;

__device__ __forceinline__ double a_at(const void* A, int dtype, int64_t idx) {
  return dtype == MFIPM_A_BF16 ? (double)__bfloat162float(static_cast<const __nv_bfloat16*>(A)[idx])
                               : static_cast<const double*>(A)[idx];
}

// y_i = a_scale sum_k A[i][k] x_k (one warp per row)
__global__ void gemv_rows(const void* A, int dtype, double a_scale, int64_t lda, const double* __restrict__ x,
                          double* __restrict__ y, int64_t m, int64_t n) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double s = 0.0;
  for (int64_t k = lane; k < n; k += 32) s = fma(a_at(A, dtype, i * lda + k), x[k], s);
  s = warp_sum(s);
  if (lane == 0) y[i] = a_scale * s;
}
// x_k = a_scale sum_i A[i][k] y_i (one thread per column: consecutive threads, consecutive k)
__global__ void gemv_cols(const void* A, int dtype, double a_scale, int64_t lda, const double* __restrict__ y,
                          double* __restrict__ x, int64_t m, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s = fma(a_at(A, dtype, i * lda + k), y[i], s);
  x[k] = a_scale * s;
}
// partial DCT by direct sums (short signals)
__device__ __forceinline__ double dct_entry(int64_t r, int64_t k, int64_t n) {
  const double a = r == 0 ? sqrt(1.0 / (double)n) : sqrt(2.0 / (double)n);
  // cos(pi r (2k+1) / (2n)); the argument reduced mod 4n keeps cospi's input small
  const int64_t q = (r * (2 * k + 1)) % (4 * n);
  return a * cospi((double)q / (double)(2 * n));
}
__global__ void dct_rows_direct(const double* __restrict__ x, const int64_t* __restrict__ rows,
                                double* __restrict__ y, int64_t m, int64_t n) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t r = rows[i];
  double s = 0.0;
  for (int64_t k = lane; k < n; k += 32) s = fma(dct_entry(r, k, n), x[k], s);
  s = warp_sum(s);
  if (lane == 0) y[i] = s;
}
__global__ void dct_rows_t_direct(const double* __restrict__ y, const int64_t* __restrict__ rows,
                                  double* __restrict__ x, int64_t m, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s = fma(dct_entry(rows[i], k, n), y[i], s);
  x[k] = s;
}
// Partial orthonormal Haar (row 0 = 1/sqrt(n); row 2^j + k = +-2^(j/2)/sqrt(n) on the halves
// of [k n/2^j, (k+1) n/2^j)), evaluated directly from its definition: one warp per row for
// A x; for A^T y each column sums its log2(n) + 1 rows, found by binary search in rows.
__device__ __forceinline__ int ilog2_64(int64_t v) { return 63 - __clzll((unsigned long long)v); }
__global__ void haar_rows_direct(const double* __restrict__ x, const int64_t* __restrict__ rows,
                                 double* __restrict__ y, int64_t m, int64_t n) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  const int64_t r = rows[i];
  const double rn = rsqrt((double)n);
  double s = 0.0;
  if (r == 0) {
    for (int64_t k = lane; k < n; k += 32) s += x[k];
    s = warp_sum(s) * rn;
  } else {
    const int j = ilog2_64(r);
    const int64_t w = n >> j, k0 = (r - ((int64_t)1 << j)) * w, h = w >> 1;
    for (int64_t k = lane; k < w; k += 32) s += k < h ? x[k0 + k] : -x[k0 + k];
    s = warp_sum(s) * rn * exp2(0.5 * j);
  }
  if (lane == 0) y[i] = s;
}
__global__ void haar_rows_t_direct(const double* __restrict__ y, const int64_t* __restrict__ rows,
                                   double* __restrict__ x, int64_t m, int64_t n) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int logn = ilog2_64(n);
  const double rn = rsqrt((double)n);
  auto find = [&](int64_t idx) -> int64_t {  // position of idx in the ascending rows, or -1
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rows[mid] < idx) lo = mid + 1; else hi = mid;
    }
    return (lo < m && rows[lo] == idx) ? lo : -1;
  };
  double s = 0.0;
  int64_t p = find(0);
  if (p >= 0) s += y[p] * rn;
  for (int j = 0; j < logn; ++j) {
    const int64_t k = c >> (logn - j);
    p = find(((int64_t)1 << j) + k);
    if (p < 0) continue;
    const bool upper = (c >> (logn - j - 1)) & 1;
    const double v = rn * exp2(0.5 * j);
    s += upper ? -y[p] * v : y[p] * v;
  }
  x[c] = s;
}
// rows ascending, distinct, inside [0, n): err = -1 otherwise
__global__ void check_rows(const int64_t* __restrict__ rows, int64_t m, int64_t n, int* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rows[i];
    if (!(r >= 0 && r < n && (i == 0 || rows[i - 1] < r))) atomicCAS(err, 0, -1);
  }
}
__global__ void to_df_vec(const double* __restrict__ x, float2* __restrict__ xd, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const df v = to_df(x[i]);
    xd[i] = make_float2(v.hi, v.lo);
  }
}
__global__ void from_df_vec(const float2* __restrict__ g, double sign, double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = sign * ((double)g[i].x + (double)g[i].y);
}
// rows outside [0, n) (reported by the setup kernel) read nothing
__global__ void gather_rows(const double* __restrict__ fwd, const int64_t* __restrict__ rows, double* __restrict__ y,
                            int64_t m, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = rows[i];
    y[i] = (r >= 0 && r < n) ? fwd[r] : NAN;
  }
}
__global__ void sub_vec(double* __restrict__ r, const double* __restrict__ b, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    r[i] -= b[i];
}
// kkt_rel = ||x - S_tau(x - g)|| / (1 + ||x||): one block, fixed order
__global__ void kkt_reduce(const double* __restrict__ x, const double* __restrict__ g, double tau, int64_t n,
                           double* out) {
  __shared__ double red[2][kT / 32];
  double a = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kT) {
    const double xi = x[i], y = xi - g[i];
    const double st = copysign(fmax(fabs(y) - tau, 0.0), y);
    a += (xi - st) * (xi - st);
    c += xi * xi;
  }
  a = warp_sum(a);
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kT / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    *out = sqrt(s0) / (1.0 + sqrt(s1));
  }
}

}  // namespace ap

// ------------------------------------------------------------------ host side
namespace {
struct Carve {
  char* base;
  size_t o = 0;
  void* take(size_t bytes) {
    void* p = base + o;
    o += (bytes + 255) & ~(size_t)255;
    return p;
  }
};
int cu_fail(cudaError_t e, std::string* msg, const char* where) {
  *msg = std::string(where) + ": " + cudaGetErrorString(e);
  return MFIPM_CUDA;
}
unsigned grid_for(int64_t items, int per_block = ap::kT) {
  const int64_t g = (items + per_block - 1) / per_block;
  return (unsigned)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}
}  // namespace

// Bytes of workspace apply_operator uses for op (never more than the solve's workspace for it).
size_t apply_workspace_bytes(const mfipm_operator& op) {
  Carve c{nullptr};
  const int64_t m = op.m, n = op.n;
  c.take(256);                                  // error word, kkt result
  c.take((size_t)8 * n);                        // g (float64)
  c.take((size_t)8 * (m > n ? m : n));          // A x (float64)
  if (op.kind == MFIPM_OP_PARTIAL_DCT && n >= kLdMinN && (n & (n - 1)) == 0) {
    const LdShape s = ld_shape(n);
    const size_t tw = (size_t)2 << (s.logN + 2);
    c.take(sizeof(ProbDesc));
    c.take(tw * 8);
    c.take(tw * 16);
    c.take((size_t)n);                          // mask
    c.take((size_t)8 * n);                      // b_u
    c.take((size_t)8 * n);                      // b_u double-float
    c.take(ld_mask_code_bytes(n, 1));
    c.take((size_t)8 * n);                      // x double-float
    c.take((size_t)8 * n);                      // g double-float / forward coefficients
    c.take((size_t)8 * n);                      // L-point intermediate
    c.take((size_t)(1 << (s.logN1 - 1)) * 8 * 8);  // masked energy partials
  }
  return c.o;
}

// what: 0 = A x, 1 = A^T y, 2 = kkt_rel of x (b, tau).  in, b, out: DEVICE; kkt: HOST.
int apply_operator(int what, const mfipm_operator& op, const double* in, const double* b, double tau, double* out,
                   double* kkt, void* workspace, size_t ws_bytes, cudaStream_t st, std::string* msg) {
  const int64_t m = op.m, n = op.n;
  if (ws_bytes < apply_workspace_bytes(op)) {
    *msg = "workspace too small for the operator product";
    return MFIPM_INVALID_ARG;
  }
  Carve c{static_cast<char*>(workspace)};
  int* err = static_cast<int*>(c.take(256));
  double* kdev = reinterpret_cast<double*>(reinterpret_cast<char*>(err) + 64);
  double* gbuf = static_cast<double*>(c.take((size_t)8 * n));
  double* ybuf = static_cast<double*>(c.take((size_t)8 * (m > n ? m : n)));
  cudaError_t e;
  if ((e = cudaMemsetAsync(err, 0, 4, st))) return cu_fail(e, msg, "clear error word");
  const bool dct = op.kind == MFIPM_OP_PARTIAL_DCT, haar = op.kind == MFIPM_OP_PARTIAL_HAAR;
  if (dct && n >= kLdMinN && (n & (n - 1)) == 0) {  // powers of two: the multi-pass chain
    const LdShape s = ld_shape(n);
    const int log2_tw = s.logN + 2;
    const size_t tw = (size_t)2 << log2_tw;
    ProbDesc* desc = static_cast<ProbDesc*>(c.take(sizeof(ProbDesc)));
    float2* tw32 = static_cast<float2*>(c.take(tw * 8));
    float4* twdf = static_cast<float4*>(c.take(tw * 16));
    uint8_t* mask = static_cast<uint8_t*>(c.take((size_t)n));
    double* bsu = static_cast<double*>(c.take((size_t)8 * n));
    float2* bsu_df = static_cast<float2*>(c.take((size_t)8 * n));
    uint8_t* mcode = static_cast<uint8_t*>(c.take(ld_mask_code_bytes(n, 1)));
    float2* xin = static_cast<float2*>(c.take((size_t)8 * n));
    float2* gout = static_cast<float2*>(c.take((size_t)8 * n));
    void* inter = c.take((size_t)8 * n);
    double* part2 = static_cast<double*>(c.take((size_t)(1 << (s.logN1 - 1)) * 8 * 8));
    ProbDesc pd;
    memset(&pd, 0, sizeof(pd));
    pd.n = n;
    pd.m = m;
    pd.kind = MFIPM_OP_PARTIAL_DCT;
    pd.log2n = s.logN;
    pd.rows = op.rows;
    pd.b = what == 0 ? nullptr : (what == 1 ? in : b);  // A^T y: b_u from y
    pd.mask = mask;
    pd.bsu = bsu;
    pd.bsu_df = bsu_df;
    if ((e = cudaMemcpyAsync(desc, &pd, sizeof(pd), cudaMemcpyHostToDevice, st)) ||
        (e = launch_twiddles(nullptr, tw32, twdf, log2_tw, st)) || (e = launch_dct_setup(desc, 1, n, err, st)))
      return cu_fail(e, msg, "setup kernels");
    LdArgs a{};
    a.logN = s.logN;
    a.logL = s.logL;
    a.logN1 = s.logN1;
    a.logN2 = s.logN2;
    a.log2_tw = log2_tw;
    a.gate = GATE_ALL;
    a.inter = inter;
    a.mask = mask;
    a.bsu = bsu;
    a.bsu_df = bsu_df;
    a.mcode = mcode;
    a.part2 = part2;
    a.nb2 = 1 << (s.logN1 - 1);
    a.kpart = 8;
    a.tw32 = tw32;
    a.twdf = twdf;
    a.din = xin;
    a.dout = gout;
    const unsigned gn = grid_for(n);
    if (what == 0) {
      ap::to_df_vec<<<gn, ap::kT, 0, st>>>(in, xin, n);
      a.fwd = gbuf;
      if ((e = ld_forward(a, 1, st))) return cu_fail(e, msg, "forward transform");
      ap::gather_rows<<<grid_for(m), ap::kT, 0, st>>>(gbuf, op.rows, out, m, n);
    } else {
      if (what == 1) {
        if ((e = cudaMemsetAsync(xin, 0, (size_t)8 * n, st))) return cu_fail(e, msg, "clear x");
      } else {
        ap::to_df_vec<<<gn, ap::kT, 0, st>>>(in, xin, n);
      }
      if ((e = ld_mask_codes(a, 1, st)) || (e = ld_resid(a, 1, st))) return cu_fail(e, msg, "residual chain");
      if (what == 1) {
        ap::from_df_vec<<<gn, ap::kT, 0, st>>>(gout, -1.0, out, n);
      } else {
        ap::from_df_vec<<<gn, ap::kT, 0, st>>>(gout, 1.0, gbuf, n);
        ap::kkt_reduce<<<1, ap::kT, 0, st>>>(in, gbuf, tau, n, kdev);
      }
    }
  } else {
    auto Ax = [&](const double* x, double* y) {
      if (dct) {
        ap::dct_rows_direct<<<grid_for(32 * m), ap::kT, 0, st>>>(x, op.rows, y, m, n);
      } else if (haar) {
        ap::haar_rows_direct<<<grid_for(32 * m), ap::kT, 0, st>>>(x, op.rows, y, m, n);
      } else {
        ap::gemv_rows<<<grid_for(32 * m), ap::kT, 0, st>>>(op.A, op.a_dtype, op.a_scale, op.lda, x, y, m, n);
      }
    };
    auto Aty = [&](const double* y, double* x) {
      if (dct) {
        ap::dct_rows_t_direct<<<grid_for(n), ap::kT, 0, st>>>(y, op.rows, x, m, n);
      } else if (haar) {
        ap::haar_rows_t_direct<<<grid_for(n), ap::kT, 0, st>>>(y, op.rows, x, m, n);
      } else {
        ap::gemv_cols<<<grid_for(n), ap::kT, 0, st>>>(op.A, op.a_dtype, op.a_scale, op.lda, y, x, m, n);
      }
    };
    if ((dct || haar) && m > 0) ap::check_rows<<<grid_for(m), ap::kT, 0, st>>>(op.rows, m, n, err);
    if (what == 0) {
      Ax(in, out);
    } else if (what == 1) {
      Aty(in, out);
    } else {
      Ax(in, ybuf);
      ap::sub_vec<<<grid_for(m), ap::kT, 0, st>>>(ybuf, b, m);
      Aty(ybuf, gbuf);
      ap::kkt_reduce<<<1, ap::kT, 0, st>>>(in, gbuf, tau, n, kdev);
    }
  }
  if ((e = cudaGetLastError())) return cu_fail(e, msg, "operator kernels");
  int herr = 0;
  if ((e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st))) return cu_fail(e, msg, "read error word");
  if (what == 2 && (e = cudaMemcpyAsync(kkt, kdev, 8, cudaMemcpyDeviceToHost, st))) return cu_fail(e, msg, "read kkt");
  if ((e = cudaStreamSynchronize(st))) return cu_fail(e, msg, "operator product");
  if (herr == -1) {
    *msg = "rows must be distinct, ascending and inside [0, n)";
    return MFIPM_INVALID_ARG;
  }
  if (herr == -2) {
    *msg = "b or y contains a non-finite value";
    return MFIPM_NUMERIC;
  }
  return MFIPM_OK;
}

}  // namespace mfipm
