// Partial-DCT operator for signals too long for one cluster's shared memory (n above
// the persistent kernel's limit): the same chain as the cluster path of solver_impl.cuh
//     A^T A w = D^-1 M D w,   A^T (A x - b) = D^-1 M (D x - b_u),   D x (forward only),
// (A = rows of the orthonormal DCT-II, Sec. 2, Eq. eq:orthonormality; D the unnormalised
// DCT-II evaluated by Makhoul's even/odd reordering and a complex FFT of length L = n/2),
// with the FFT split four-step style over global memory, L = N1 x N2:
//   pass A  per column t2: h[N2 t1 + t2] (packed from w on the fly), N1-point FFT over
//           t1, times exp(-2 pi i t2 k1 / L), stored as Y[k1][t2];
//   pass B  per row pair (k1, N1 - k1): N2-point FFTs over t2, the real-DCT untangling,
//           row mask (minus b_u) and its exact inverse (dct_pointwise), inverse FFTs;
//           frequency k = k1 + N1 k2 pairs with L - k = (N1 - k1) + N1 (N2 - 1 - k2), so
//           a row pair holds every pair of the untangling;
//   pass C  per column: conjugate twiddles, inverse N1-point FFT, unpacked back to n reals.
// Pass A's column group {t2} is closed under t2 -> N2 - 1 - t2 and the rows t1 < N1/2
// pair with N1 - 1 - t1, so each CTA reads and writes whole aligned runs of w: packing
// index t and L - 1 - t consume w[4t .. 4t+3] together.  Each pass reads and writes the
// L-point intermediate once: three passes per operator product instead of the single
// on-chip chain of the cluster path.  float2 carries the PCG products; double-float
// carries the float64-grade residual and the forward transform.
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "device_common.cuh"
#include "internal.h"
#include "large_dct.h"
#include "lockstep.h"
#include "solver_impl.cuh"

namespace mfipm {
namespace ld {

// columns per pass A / pass C block (half of them and their mirrors): 16 for float32,
// 8 for double-float (keeps three blocks' shared memory on an SM)
template <class C> struct ColsOf { static constexpr int v = 16; };
template <> struct ColsOf<dfc> { static constexpr int v = 8; };
constexpr int kThr = 512;     // threads per pass A / pass C block
constexpr int kThrB = 256;    // threads per pass B block

__device__ __forceinline__ bool gated_out(const LdArgs& a, int j) {
  if (a.gate == GATE_ACTIVE) return !a.col[j].active;
  if (a.gate == GATE_LIVE) return a.col[j].done != 0;
  return false;
}

// radix-4 DIF FFT (natural in, bit-reversed out) of ncols columns of M = 2^logM points,
// column c at buf + c * stride; forward sign.
template <class C>
__device__ void cols_fft_dif(C* buf, int logM, int ncols, int stride, const Twiddle<C>& tw) {
  const int M = 1 << logM;
  int logB = logM;
  for (; logB >= 2; logB -= 2) {
    const int logS = logB - 2, S = 1 << logS;
    for (int g = threadIdx.x; g < ncols * (M >> 2); g += blockDim.x) {
      const int col = g >> (logM - 2), gi = g & ((M >> 2) - 1);
      const int blk = gi >> logS, t = gi & (S - 1);
      C* p = buf + col * stride + (blk << logB) + t;
      C a0 = p[0], a1 = p[S], a2 = p[2 * S], a3 = p[3 * S];
      C w1 = tw.root(t, logB), w2 = tw.root(2 * t, logB), w3 = tw.root(3 * t, logB);
      C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
      p[0] = cadd(s02, s13);
      p[S] = cmul(csub(s02, s13), w2);
      p[2 * S] = cmul(cadd(d02, cmul_mi(d13)), w1);
      p[3 * S] = cmul(cadd(d02, cmul_i(d13)), w3);
    }
    __syncthreads();
  }
  if (logB == 1) {
    for (int g = threadIdx.x; g < ncols * (M >> 1); g += blockDim.x) {
      const int col = g >> (logM - 1), gi = g & ((M >> 1) - 1);
      C* p = buf + col * stride + 2 * gi;
      const C a0 = p[0], a1 = p[1];
      p[0] = cadd(a0, a1);
      p[1] = csub(a0, a1);
    }
    __syncthreads();
  }
}

// unnormalised inverse of cols_fft_dif: bit-reversed in, natural out, + sign
template <class C>
__device__ void cols_fft_dit_inv(C* buf, int logM, int ncols, int stride, const Twiddle<C>& tw) {
  const int M = 1 << logM;
  int logB = 2;
  if (logM & 1) {
    for (int g = threadIdx.x; g < ncols * (M >> 1); g += blockDim.x) {
      const int col = g >> (logM - 1), gi = g & ((M >> 1) - 1);
      C* p = buf + col * stride + 2 * gi;
      const C a0 = p[0], a1 = p[1];
      p[0] = cadd(a0, a1);
      p[1] = csub(a0, a1);
    }
    __syncthreads();
    logB = 3;
  }
  for (; logB <= logM; logB += 2) {
    const int logS = logB - 2, S = 1 << logS;
    for (int g = threadIdx.x; g < ncols * (M >> 2); g += blockDim.x) {
      const int col = g >> (logM - 2), gi = g & ((M >> 2) - 1);
      const int blk = gi >> logS, t = gi & (S - 1);
      C* p = buf + col * stride + (blk << logB) + t;
      C o0 = p[0];
      C b1 = cmulc(p[S], tw.root(2 * t, logB));
      C b2 = cmulc(p[2 * S], tw.root(t, logB));
      C b3 = cmulc(p[3 * S], tw.root(3 * t, logB));
      C Ss = cadd(o0, b1), D = csub(o0, b1), E = cadd(b2, b3), F = csub(b3, b2);
      p[0] = cadd(Ss, E);
      p[S] = cadd(D, cmul_mi(F));
      p[2 * S] = csub(Ss, E);
      p[3 * S] = cadd(D, cmul_i(F));
    }
    __syncthreads();
  }
}

template <class C> struct Io;
// PCG products: w = p_u - p_v from the (u, v) pairs; result y as float32
template <> struct Io<float2> {
  using R = float;
  static __device__ __forceinline__ float load(const LdArgs& a, int64_t gi) {
    const float2 p = a.pin[gi];
    return p.x - p.y;
  }
  static __device__ __forceinline__ void store4(const LdArgs& a, int64_t gi, float w0, float w1, float w2, float w3) {
    *reinterpret_cast<float4*>(a.yout + gi) = make_float4(w0, w1, w2, w3);
  }
  static __device__ __forceinline__ Twiddle<float2> tw(const LdArgs& a) { return Twiddle<float2>{a.tw32, a.log2_tw}; }
  static __device__ __forceinline__ float2* inter(const LdArgs& a) { return reinterpret_cast<float2*>(a.inter); }
};
// double-float vectors
template <> struct Io<dfc> {
  using R = df;
  static __device__ __forceinline__ df load(const LdArgs& a, int64_t gi) {
    const float2 v = a.din[gi];
    return df(v.x, v.y);
  }
  static __device__ __forceinline__ void store4(const LdArgs& a, int64_t gi, df w0, df w1, df w2, df w3) {
    float4* o = reinterpret_cast<float4*>(a.dout + gi);
    o[0] = make_float4(w0.hi, w0.lo, w1.hi, w1.lo);
    o[1] = make_float4(w2.hi, w2.lo, w3.hi, w3.lo);
  }
  static __device__ __forceinline__ Twiddle<dfc> tw(const LdArgs& a) { return Twiddle<dfc>{a.twdf, a.log2_tw}; }
  static __device__ __forceinline__ dfc* inter(const LdArgs& a) { return reinterpret_cast<dfc*>(a.inter); }
};

// the outer residual of the large-gap iterations (reading R17) through the float32 chain:
// x from its double-float pairs rounded to float32, A^T (A x - b) stored as double-float pairs
struct IoR32 {
  using R = float;
  static __device__ __forceinline__ float load(const LdArgs& a, int64_t gi) {
    const float2 v = a.din[gi];
    return v.x + v.y;
  }
  static __device__ __forceinline__ void store4(const LdArgs& a, int64_t gi, float w0, float w1, float w2, float w3) {
    float4* o = reinterpret_cast<float4*>(a.dout + gi);
    o[0] = make_float4(w0, 0.f, w1, 0.f);
    o[1] = make_float4(w2, 0.f, w3, 0.f);
  }
  static __device__ __forceinline__ Twiddle<float2> tw(const LdArgs& a) { return Twiddle<float2>{a.tw32, a.log2_tw}; }
  static __device__ __forceinline__ float2* inter(const LdArgs& a) { return reinterpret_cast<float2*>(a.inter); }
};

// column t2 of slot ci of block cb (K columns: h = K/2 slots h cb + ci, then their mirrors
// N2 - 2h - h cb + ci; slot ci and slot K - 1 - ci hold mirror columns t2 and N2 - 1 - t2)
template <int K>
__device__ __forceinline__ int col_of(int ci, int cb, int N2) {
  constexpr int h = K / 2;
  return ci < h ? h * cb + ci : N2 - 2 * h - h * cb + ci;
}

template <class C, class IO = Io<C>>
__global__ void __launch_bounds__(kThr) pass_a(LdArgs a) {
  constexpr int kCols = ColsOf<C>::v, kLog = kCols == 16 ? 4 : 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = blockIdx.y, cb = blockIdx.x;
  if (gated_out(a, j)) return;
  const int N1 = 1 << a.logN1, N2 = 1 << a.logN2, stride = N1 + 1;
  const int64_t n = (int64_t)1 << a.logN, L = n >> 1, base = (int64_t)j * n;
  // pack: t = N2 t1 + t2 (t1 < N1/2) takes w[4t], w[4t+2]; its mirror L-1-t (row N1-1-t1,
  // slot kCols-1-ci) takes w[4t+3], w[4t+1]
#pragma unroll 4
  for (int e = threadIdx.x; e < kCols * (N1 >> 1); e += blockDim.x) {
    const int ci = e & (kCols - 1), t1 = e >> kLog;
    const int64_t t = (int64_t)t1 * N2 + col_of<kCols>(ci, cb, N2);
    const int64_t gi = base + 4 * t;
    const auto w0 = IO::load(a, gi), w1 = IO::load(a, gi + 1), w2 = IO::load(a, gi + 2), w3 = IO::load(a, gi + 3);
    buf[ci * stride + t1] = mk(w0, w2);
    buf[(kCols - 1 - ci) * stride + (N1 - 1 - t1)] = mk(w3, w1);
  }
  __syncthreads();
  const Twiddle<C> tw = IO::tw(a);
  cols_fft_dif<C>(buf, a.logN1, kCols, stride, tw);
  C* Y = IO::inter(a) + (int64_t)j * L;
#pragma unroll 4
  for (int e = threadIdx.x; e < kCols * N1; e += blockDim.x) {
    const int ci = e & (kCols - 1), k1 = e >> kLog, t2 = col_of<kCols>(ci, cb, N2);
    const C v = buf[ci * stride + bitrev(k1, a.logN1)];
    Y[(int64_t)k1 * N2 + t2] = cmul(v, tw.root((int64_t)t2 * k1, a.logL));
  }
}

// Work item e of row-pair block rb in pass B: frequencies kA = rowA + N1 k2A and its partner
// kB = L - kA = rowB + N1 k2B, their buffer positions (bit-reversed order, row B at +stride)
// and whether kB is a second frequency (false when kA pairs with itself: k = 0 and L/2).
// Row pair (rb, N1 - rb): N2 items.  rb = 0 holds rows 0 and N1/2: N2/2 + 1 items pair
// k2 <-> N2 - k2 in row 0, then N2/2 items pair k2 <-> N2 - 1 - k2 in row N1/2.
struct PairItem {
  int rowA, k2A, rowB, k2B, pA, pB;
  bool two;
};
__device__ __forceinline__ PairItem pair_item(int rb, int e, int logN1, int logN2) {
  const int N1 = 1 << logN1, N2 = 1 << logN2, stride = N2 + 1;
  PairItem it;
  if (rb != 0) {
    it.rowA = rb;
    it.k2A = e;
    it.rowB = N1 - rb;
    it.k2B = N2 - 1 - e;
    it.pA = bitrev(it.k2A, logN2);
    it.pB = stride + bitrev(it.k2B, logN2);
    it.two = true;
  } else if (e <= (N2 >> 1)) {
    it.rowA = it.rowB = 0;
    it.k2A = e;
    it.k2B = (N2 - e) & (N2 - 1);
    it.pA = bitrev(it.k2A, logN2);
    it.pB = bitrev(it.k2B, logN2);
    it.two = (e != 0 && e != (N2 >> 1));
  } else {
    it.rowA = it.rowB = N1 >> 1;
    it.k2A = e - (N2 >> 1) - 1;
    it.k2B = N2 - 1 - it.k2A;
    it.pA = stride + bitrev(it.k2A, logN2);
    it.pB = stride + bitrev(it.k2B, logN2);
    it.two = true;
  }
  return it;
}
__device__ __forceinline__ int items_of(int rb, int logN2) { return (1 << logN2) + (rb == 0 ? 1 : 0); }

// bits 0..3 of the pointwise step's row mask for frequency k (rows k, n-k, L-k, L+k)
__device__ __forceinline__ unsigned mask_bits(const uint8_t* mask, int64_t k, int64_t n) {
  const int64_t L = n >> 1;
  return (mask[k] ? 1u : 0u) | ((k > 0 && mask[n - k]) ? 2u : 0u) | (mask[L - k] ? 4u : 0u) | (mask[L + k] ? 8u : 0u);
}

// The mask bits of every pass-B work item, once per solve: code[j][rb][e] = bits(kA) | bits(kB) << 4.
__global__ void mask_codes(LdArgs a) {
  const int j = blockIdx.y, rb = blockIdx.x;
  const int N1 = 1 << a.logN1, N2 = 1 << a.logN2;
  const int64_t n = (int64_t)1 << a.logN;
  const uint8_t* mask = a.mask + (int64_t)j * n;
  uint8_t* code = a.mcode + ((int64_t)j * (N1 >> 1) + rb) * (N2 + 1);
  for (int e = threadIdx.x; e < items_of(rb, a.logN2); e += blockDim.x) {
    const PairItem it = pair_item(rb, e, a.logN1, a.logN2);
    const int64_t kA = it.rowA + (int64_t)N1 * it.k2A, kB = it.rowB + (int64_t)N1 * it.k2B;
    code[e] = (uint8_t)(mask_bits(mask, kA, n) | (it.two ? mask_bits(mask, kB, n) << 4 : 0u));
  }
}

// exp(-2 pi i (row + N1 k2) / 2^l).  float32: as exp(-2 pi i row / 2^l) exp(-2 pi i k2 / 2^(l -
// logN1)), so consecutive k2 read consecutive table entries; double-float: one table entry
// (a double-float complex product costs more than the scattered load).
template <class C>
__device__ __forceinline__ C tw_rowcol(const Twiddle<C>& tw, int row, int k2, int l, int logN1) {
  if constexpr (std::is_same<C, dfc>::value) {
    return tw.root(row + ((int64_t)k2 << logN1), l);
  } else {
    const C f = tw.root(k2, l - logN1);
    return row ? cmul(tw.root(row, l), f) : f;
  }
}

// MODE_NORMAL / MODE_RESID: rows through the pointwise chain and back; MODE_FORWARD:
// alpha_j X_j of the forward transform into fwd (float64, natural order).
template <class C, int MODE>
__global__ void __launch_bounds__(kThrB) pass_b(LdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[kThrB / 32];
  const int j = blockIdx.y, rb = blockIdx.x;
  if (gated_out(a, j)) return;
  using IO = Io<C>;
  using R = typename IO::R;
  const int N1 = 1 << a.logN1, N2 = 1 << a.logN2, stride = N2 + 1;
  const int64_t n = (int64_t)1 << a.logN, L = n >> 1;
  const int rA = rb, rB = rb == 0 ? (N1 >> 1) : N1 - rb;
  C* Y = IO::inter(a) + (int64_t)j * L;
#pragma unroll 4
  for (int e = threadIdx.x; e < 2 * N2; e += blockDim.x) {
    const int row = e >= N2, t2 = e & (N2 - 1);
    buf[row * stride + t2] = Y[(int64_t)(row ? rB : rA) * N2 + t2];
  }
  __syncthreads();
  const Twiddle<C> tw = IO::tw(a);
  cols_fft_dif<C>(buf, a.logN2, 2, stride, tw);
  DctGeom geo;
  geo.logN = a.logN;
  geo.logL = a.logN - 1;
  geo.logM = a.logN2;
  geo.rank = 0;
  geo.N = n;
  geo.mask = a.mask + (int64_t)j * n;
  geo.bsu = a.bsu + (int64_t)j * n;
  geo.bsu_df = a.bsu_df + (int64_t)j * n;
  double* fwd = MODE == MODE_FORWARD ? a.fwd + (int64_t)j * n : nullptr;
  const PwConst<R> pc(geo);
  R acc = pc.zero;
  // one work item per pair (k, L - k); the pair's two new values overwrite the old ones
  const uint8_t* code = a.mcode + ((int64_t)j * (N1 >> 1) + rb) * (N2 + 1);
  for (int e = threadIdx.x; e < items_of(rb, a.logN2); e += blockDim.x) {
    const PairItem it = pair_item(rb, e, a.logN1, a.logN2);
    const int64_t kA = it.rowA + (int64_t)N1 * it.k2A, kB = it.rowB + (int64_t)N1 * it.k2B;
    const unsigned mb = MODE == MODE_FORWARD ? 0u : code[e];
    const C zA = buf[it.pA], zB = buf[it.pB];
    const C nA = dct_pointwise_w<C, MODE>(kA, zA, zB, tw_rowcol(tw, it.rowA, it.k2A, a.logN, a.logN1),
                                          tw_rowcol(tw, it.rowA, it.k2A, a.logN + 2, a.logN1), mb & 15u, geo, pc,
                                          true, acc, fwd);
    if (it.two) {
      const C nB = dct_pointwise_w<C, MODE>(kB, zB, zA, tw_rowcol(tw, it.rowB, it.k2B, a.logN, a.logN1),
                                            tw_rowcol(tw, it.rowB, it.k2B, a.logN + 2, a.logN1), mb >> 4, geo, pc,
                                            true, acc, fwd);
      if (MODE != MODE_FORWARD) buf[it.pB] = nB;
    }
    if (MODE != MODE_FORWARD) buf[it.pA] = nA;
  }
  if (MODE == MODE_FORWARD) return;
  // block total of the masked energy (||A w||^2 or ||A x - b||^2): warp sums in the
  // accumulator's own type (float32 or double-float, no float64 instruction per thread)
  R wsum = acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum = wsum + shfl_xor(wsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = to_double(wsum);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    a.part2[((int64_t)j * a.nb2 + rb) * a.kpart] = t;
  }
  cols_fft_dit_inv<C>(buf, a.logN2, 2, stride, tw);
  for (int e = threadIdx.x; e < 2 * N2; e += blockDim.x) {
    const int row = e >= N2, t2 = e & (N2 - 1);
    Y[(int64_t)(row ? rB : rA) * N2 + t2] = buf[row * stride + t2];
  }
}

template <class C, class IO = Io<C>>
__global__ void __launch_bounds__(kThr) pass_c(LdArgs a) {
  constexpr int kCols = ColsOf<C>::v, kLog = kCols == 16 ? 4 : 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int j = blockIdx.y, cb = blockIdx.x;
  if (gated_out(a, j)) return;
  const int N1 = 1 << a.logN1, N2 = 1 << a.logN2, stride = N1 + 1;
  const int64_t n = (int64_t)1 << a.logN, L = n >> 1, base = (int64_t)j * n;
  const Twiddle<C> tw = IO::tw(a);
  const C* Y = IO::inter(a) + (int64_t)j * L;
#pragma unroll 4
  for (int e = threadIdx.x; e < kCols * N1; e += blockDim.x) {
    const int ci = e & (kCols - 1), k1 = e >> kLog, t2 = col_of<kCols>(ci, cb, N2);
    const C v = Y[(int64_t)k1 * N2 + t2];
    buf[ci * stride + bitrev(k1, a.logN1)] = cmulc(v, tw.root((int64_t)t2 * k1, a.logL));
  }
  __syncthreads();
  cols_fft_dit_inv<C>(buf, a.logN1, kCols, stride, tw);
  for (int e = threadIdx.x; e < kCols * (N1 >> 1); e += blockDim.x) {
    const int ci = e & (kCols - 1), t1 = e >> kLog;
    const int64_t t = (int64_t)t1 * N2 + col_of<kCols>(ci, cb, N2);
    const C h = buf[ci * stride + t1], hm = buf[(kCols - 1 - ci) * stride + (N1 - 1 - t1)];
    IO::store4(a, base + 4 * t, h.x, hm.y, h.y, hm.x);
  }
}

}  // namespace ld

// ------------------------------------------------------------------ host side
LdShape ld_shape(int64_t n) {
  LdShape s{};
  int logN = 0;
  while (((int64_t)1 << logN) < n) ++logN;
  s.logN = logN;
  s.logL = logN - 1;
  s.logN2 = (s.logL + 1) / 2;
  s.logN1 = s.logL - s.logN2;
  return s;
}
bool ld_supported(int64_t n) { return n >= kLdMinN && n <= kLdMaxN && (n & (n - 1)) == 0; }

template <class C> static size_t smem_cols(int logN1) {
  return (size_t)ld::ColsOf<C>::v * (((size_t)1 << logN1) + 1) * sizeof(C);
}
static size_t smem_rows(int logN2, size_t elem) { return (size_t)2 * (((size_t)1 << logN2) + 1) * elem; }

// shared memory size and the largest carveout, so that several blocks share an SM
static cudaError_t prep_kernel(void (*k)(LdArgs), size_t sm) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}
template <class C>
static cudaError_t launch_cols(void (*k)(LdArgs), const LdArgs& a, int R, cudaStream_t st) {
  const size_t sm = smem_cols<C>(a.logN1);
  cudaError_t e = prep_kernel(k, sm);
  if (e != cudaSuccess) return e;
  k<<<dim3((1u << a.logN2) / ld::ColsOf<C>::v, R), ld::kThr, sm, st>>>(a);
  return cudaGetLastError();
}
template <class C>
static cudaError_t launch_rows(void (*k)(LdArgs), const LdArgs& a, int R, cudaStream_t st) {
  const size_t sm = smem_rows(a.logN2, sizeof(C));
  cudaError_t e = prep_kernel(k, sm);
  if (e != cudaSuccess) return e;
  k<<<dim3((1u << a.logN1) / 2, R), ld::kThrB, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t ld_mask_codes(const LdArgs& a, int R, cudaStream_t st) {
  ld::mask_codes<<<dim3((1u << a.logN1) / 2, R), 256, 0, st>>>(a);
  return cudaGetLastError();
}
size_t ld_mask_code_bytes(int64_t n, int R) {
  const LdShape s = ld_shape(n);
  return (size_t)R * ((size_t)1 << (s.logN1 - 1)) * (((size_t)1 << s.logN2) + 1);
}

// y = A^T A w for w = p_u - p_v (float32)
cudaError_t ld_normal(const LdArgs& a, int R, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cols<float2>(ld::pass_a<float2>, a, R, st))) return e;
  if ((e = launch_rows<float2>(ld::pass_b<float2, MODE_NORMAL>, a, R, st))) return e;
  return launch_cols<float2>(ld::pass_c<float2>, a, R, st);
}
// g = A^T (A x - b) (float64 in and out, double-float arithmetic)
cudaError_t ld_resid(const LdArgs& a, int R, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cols<dfc>(ld::pass_a<dfc>, a, R, st))) return e;
  if ((e = launch_rows<dfc>(ld::pass_b<dfc, MODE_RESID>, a, R, st))) return e;
  return launch_cols<dfc>(ld::pass_c<dfc>, a, R, st);
}
// the same residual through the float32 chain (the outer loop's large-gap iterations)
cudaError_t ld_resid_f32(const LdArgs& a, int R, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cols<float2>(ld::pass_a<float2, ld::IoR32>, a, R, st))) return e;
  if ((e = launch_rows<float2>(ld::pass_b<float2, MODE_RESID>, a, R, st))) return e;
  return launch_cols<float2>(ld::pass_c<float2, ld::IoR32>, a, R, st);
}
// fwd = C x, the full orthonormal DCT-II (float64 in and out)
cudaError_t ld_forward(const LdArgs& a, int R, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cols<dfc>(ld::pass_a<dfc>, a, R, st))) return e;
  return launch_rows<dfc>(ld::pass_b<dfc, MODE_FORWARD>, a, R, st);
}

}  // namespace mfipm
