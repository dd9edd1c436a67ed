#pragma once
// Device-resident matrix-free primal-dual IPM (arXiv:1208.5435, Sec. 5.1 Algorithm)
// with PCG Newton solves (Sec. 4) for  min tau||x||_1 + 1/2||Ax - b||^2.
//
// Execution model: one thread-block cluster of G CTAs solves one problem from start to
// finish inside a single kernel launch; clusters take problems from a device work
// queue (persistent launch).  CTA rank r of a cluster owns a contiguous chunk of the
// 2n-vectors' indices; per-index work (PCG updates, preconditioner, IPM residuals,
// step lengths) is local, and the only cross-CTA traffic is
//   * scalar reductions through distributed shared memory (cluster barrier + DSMEM reads),
//   * the operator: partial DCT = a distributed FFT whose single exchange step reads and
//     writes the other CTAs' shared-memory buffers; dense A = an all-reduce of A w.
//
// Partial DCT operator, A = R C with C the orthonormal DCT-II (Sec. 2, Eq.
// eq:orthonormality).  With the unnormalised DCT-II D (C = diag(alpha) D),
//     A^T A w = D^-1 M D w,   A^T (A x - b) = D^-1 M (D x - b_u),
// where M masks the sampled rows and b_u holds b_i / alpha_{row_i} at the sampled rows.
// D of length N is evaluated through a complex FFT of length L = N/2 (the even/odd
// reordering of Makhoul and the half-length real-FFT packing): v_j = x_{2j},
// v_{N-1-j} = x_{2j+1}; h_j = v_{2j} + i v_{2j+1}.  The FFT is split four-step
// style over the cluster: L = M G, CTA g holds h_{g + G n2} (n2 < M) and runs a local
// M-point FFT; a "slot step" then gathers, for each output column k2, the G values
// Y_g[k2] from all CTAs, applies the four-step twiddles and a G-point DFT, performs the
// real-DCT untangling, the row mask (and the subtraction of b), and the exact inverse of
// all of it, and writes the results back.  k2 and M-k2 are handled by lanes l and l^16
// of one warp, so the pairing H[k] <-> H[L-k] of the real-FFT untangling is a shuffle.
// Because every per-index operation of the IPM and the PCG is elementwise, all
// n-vectors are stored directly in this FFT order ("storage order"): no gather or
// scatter happens inside the iteration.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "device_common.cuh"
#include "internal.h"

namespace mfipm {

// ------------------------------------------------------------------ small helpers
// Reciprocal by Newton-Raphson iteration r <- r + r (1 - z r) from a float32 seed
// (two steps: the relative error squares each step, 1e-7 -> 1e-14 -> rounding).
__device__ __forceinline__ double rcp64(double z) {
  const float zf = (float)z;
  if (!(fabsf(zf) > 1e-36f && fabsf(zf) < 1e36f)) return 1.0 / z;
  double r = (double)__frcp_rn(zf);
  double e = fma(-z, r, 1.0);
  r = fma(r, e, r);
  e = fma(-z, r, 1.0);
  return fma(r, e, r);
}

__device__ __forceinline__ float to_float(df v) { return __fadd_rn(v.hi, v.lo); }
__device__ __forceinline__ float to_float(double v) { return (float)v; }
template <class T> __device__ __forceinline__ T from_float(float f);
template <> __device__ __forceinline__ df from_float<df>(float f) { return df(f, 0.f); }
template <> __device__ __forceinline__ double from_float<double>(float f) { return (double)f; }

template <class PS> struct V2;
template <> struct V2<float> { using T = float2; };
template <> struct V2<double> { using T = double2; };

// P^-1 r for one index: P block [[du + rho, -rho], [-rho, dv + rho]]  (Eq. eq:ne2_P)
template <class PS>
__device__ __forceinline__ typename V2<PS>::T precond(typename V2<PS>::T d, typename V2<PS>::T r, PS rho) {
  const PS a = d.x + rho, c = d.y + rho;
  const PS det = d.x * d.y + rho * (d.x + d.y);
  const PS inv = (PS)1 / det;
  typename V2<PS>::T z;
  z.x = (c * r.x + rho * r.y) * inv;
  z.y = (rho * r.x + a * r.y) * inv;
  return z;
}

enum { MODE_NORMAL = 0, MODE_RESID = 1, MODE_FORWARD = 2 };

// ------------------------------------------------------------------ partial DCT op
struct DctGeom {
  int logN, logL, logM, rank;
  int64_t N;
  const uint8_t* mask;
  const double* bsu;      // b scattered to its rows / DCT scale (float64)
  const float2* bsu_df;   // the same as double-float (hi, lo)
  // per frequency k < L (persistent kernel; null elsewhere): mask bits of rows k, N-k, L-k,
  // L+k and their four b_u values as one 32-byte record in the residual's arithmetic
  const uint8_t* mcode = nullptr;
  const void* bpk = nullptr;
  bool bpk_f64 = false;   // records hold float64 values (else double-float hi[4], lo[4])
};

// The four b_u values of frequency k from its packed record (loaded only when a row is sampled).
template <class R> struct B4 { R b1, b2, b3, b4; };
__device__ __forceinline__ B4<float> load_b4(const DctGeom& g, int64_t k, float) {
  if (g.bpk_f64) {
    const double2* r = static_cast<const double2*>(g.bpk) + 2 * k;
    const double2 u = __ldg(r), v = __ldg(r + 1);
    return B4<float>{(float)u.x, (float)u.y, (float)v.x, (float)v.y};
  }
  const float4 h = __ldg(static_cast<const float4*>(g.bpk) + 2 * k);
  return B4<float>{h.x, h.y, h.z, h.w};
}
__device__ __forceinline__ B4<double> load_b4(const DctGeom& g, int64_t k, double) {
  const double2* r = static_cast<const double2*>(g.bpk) + 2 * k;
  const double2 u = __ldg(r), v = __ldg(r + 1);
  return B4<double>{u.x, u.y, v.x, v.y};
}
__device__ __forceinline__ B4<df> load_b4(const DctGeom& g, int64_t k, df) {
  const float4* r = static_cast<const float4*>(g.bpk) + 2 * k;
  const float4 h = __ldg(r), l = __ldg(r + 1);
  return B4<df>{df(h.x, l.x), df(h.y, l.y), df(h.z, l.z), df(h.w, l.w)};
}

// Constants of the pointwise step in the chain's arithmetic, built once per exchange step.
template <class R> __device__ __forceinline__ R cst(double v);
template <> __device__ __forceinline__ float cst<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ double cst<double>(double v) { return v; }
template <> __device__ __forceinline__ df cst<df>(double v) { return to_df(v); }
// 2^e built from its exponent bits (|e| small), and 1/sqrt(2): exact or correctly rounded
// constants without float64 arithmetic (a float64 division costs more here than the
// float32 work of a pointwise block: the float64 pipe runs at a small fraction of FP32)
template <class R> __device__ __forceinline__ R pow2(int e);
template <> __device__ __forceinline__ float pow2<float>(int e) { return __int_as_float((127 + e) << 23); }
template <> __device__ __forceinline__ double pow2<double>(int e) {
  return __longlong_as_double((long long)(1023 + e) << 52);
}
template <> __device__ __forceinline__ df pow2<df>(int e) { return df(pow2<float>(e), 0.f); }
template <class R> __device__ __forceinline__ R rsqrt2();
template <> __device__ __forceinline__ float rsqrt2<float>() { return 0x1.6a09e6p-1f; }
template <> __device__ __forceinline__ double rsqrt2<double>() { return 0.70710678118654752440; }
template <> __device__ __forceinline__ df rsqrt2<df>() { return df(0x1.6a09e6p-1f, 0x1.9fcef4p-27f); }

// N = 2^logN and L = N/2 are powers of two, so 1/L, 1/N and 2/N are exact
template <class R> struct PwConst {
  R half, invL, a2_0, a2_j, rs2, zero;
  __device__ explicit PwConst(const DctGeom& geo)
      : half(pow2<R>(-1)),
        invL(pow2<R>(-geo.logL)),
        a2_0(pow2<R>(-geo.logN)),
        a2_j(pow2<R>(1 - geo.logN)),
        rs2(rsqrt2<R>()),
        zero() {}
  // any even N (the mixed-radix chain): 1/L = 2/N, 1/N and 2/N, computed once per problem in
  // float64 and rounded to the chain's arithmetic
  __device__ PwConst(double inv_n)
      : half(pow2<R>(-1)), invL(cst<R>(2.0 * inv_n)), a2_0(cst<R>(inv_n)), a2_j(cst<R>(2.0 * inv_n)),
        rs2(rsqrt2<R>()), zero() {}
};
__device__ __forceinline__ float load_bsu(const DctGeom& g, int64_t i, float) { return g.bsu_df[i].x; }
__device__ __forceinline__ double load_bsu(const DctGeom& g, int64_t i, double) { return g.bsu[i]; }
__device__ __forceinline__ df load_bsu(const DctGeom& g, int64_t i, df) {
  const float2 v = g.bsu_df[i];
  return df(v.x, v.y);
}

// Real-DCT untangling, row mask (minus b_u) and its exact inverse for one frequency k of
// the length-L FFT, given a = H[k] and b = H[L-k].  Returns the value H'[k] that the
// inverse chain needs; accumulates this index's share of the masked energy into acc and,
// in MODE_FORWARD, writes alpha_j X_j instead.  Each DCT coefficient j is counted by
// exactly one k: j in {k, N-k (k>0)} and, for k = 0, also j = L.
// With the twiddles wN = exp(-2 pi i k / N), eps = exp(-i pi k / (2N)) and the row-mask bits
// mb (bit 0..3: rows k, N-k (k > 0), L-k, L+k sampled; unused in MODE_FORWARD) supplied by the
// caller.
template <class C, int MODE, class R = decltype(C().x)>
__device__ __forceinline__ C dct_pointwise_w(int64_t k, C a, C b, C wN, C eps, unsigned mb, const DctGeom& geo,
                                             const PwConst<R>& pc, bool valid, R& acc, double* fwd_out) {
  const int64_t N = geo.N, L = N >> 1;
  const C c45 = mk(pc.rs2, -pc.rs2);  // exp(-i pi/4)
  const C E = cscale(cadd(a, cconj(b)), pc.half);
  const C O = cscale(cmul_mi(csub(a, cconj(b))), pc.half);
  const C wO = cmul(wN, O);
  const C Wk = cmul(eps, cadd(E, wO));                   // eps^k V[k]
  const C Wlk = cmul(c45, cconj(cmul(eps, csub(E, wO))));  // eps^(L-k) V[L-k]
  const int64_t i1 = k, i2 = N - k, i3 = L - k, i4 = L + k;
  R X1 = Wk.x, X2 = -Wk.y, X3 = Wlk.x, X4 = -Wlk.y;
  if constexpr (MODE == MODE_FORWARD) {
    if (valid) {
      const double sj = sqrt(2.0 / (double)N);
      fwd_out[i1] = (i1 == 0 ? sqrt(1.0 / (double)N) : sj) * to_double(X1);
      if (k > 0) fwd_out[i2] = sj * to_double(X2);
      if (k == 0) fwd_out[i3] = sj * to_double(X3);
    }
    return a;
  } else {
    const bool m1 = mb & 1u, m2 = mb & 2u, m3 = mb & 4u, m4 = mb & 8u;
    if constexpr (MODE == MODE_RESID) {
      if (geo.bpk) {
        if (mb) {
          const B4<R> bq = load_b4(geo, k, R());
          X1 = m1 ? X1 - bq.b1 : pc.zero;
          X2 = m2 ? X2 - bq.b2 : pc.zero;
          X3 = m3 ? X3 - bq.b3 : pc.zero;
          X4 = m4 ? X4 - bq.b4 : pc.zero;
        } else {
          X1 = X2 = X3 = X4 = pc.zero;
        }
      } else {
        X1 = m1 ? X1 - load_bsu(geo, i1, R()) : pc.zero;
        X2 = m2 ? X2 - load_bsu(geo, i2, R()) : pc.zero;
        X3 = m3 ? X3 - load_bsu(geo, i3, R()) : pc.zero;
        X4 = m4 ? X4 - load_bsu(geo, i4, R()) : pc.zero;
      }
    } else {
      X1 = m1 ? X1 : pc.zero;
      X2 = m2 ? X2 : pc.zero;
      X3 = m3 ? X3 : pc.zero;
      X4 = m4 ? X4 : pc.zero;
    }
    if (valid) {
      R t = (i1 == 0 ? pc.a2_0 : pc.a2_j) * X1 * X1;
      if (k > 0) t += pc.a2_j * X2 * X2;
      if (k == 0) t += pc.a2_j * X3 * X3;
      acc += t;
    }
    const C Vk = cmulc(mk(X1, -X2), eps);                     // conj(eps^k) W'[k]
    const C Vlk = cmul(cconj(c45), cmul(eps, mk(X3, -X4)));    // conj(eps^(L-k)) W'[L-k]
    const C cVlk = cconj(Vlk);
    const C Ep = cscale(cadd(Vk, cVlk), pc.half);
    const C Op = cscale(cmulc(csub(Vk, cVlk), wN), pc.half);
    return cscale(cadd(Ep, cmul_i(Op)), pc.invL);
  }
}

// The exchange step of the distributed DCT chain (see the file comment).  Returns this
// CTA's share of sum_j alpha_j^2 X'_j^2 (||A w||^2 or ||A x - b||^2).  MODE_FORWARD
// writes alpha_j X_j (the full orthonormal DCT-II) to fwd_out[j] and stops there.
template <int G, class C, int MODE>
__device__ __noinline__ double dct_slot_step(C* buf, const DctGeom& geo, const Twiddle<C>& tw, double* fwd_out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = 1 << geo.logM;
  const int spc = (M >> 1) / G;  // slots per CTA (>= 1 by the host's choice of G)
  constexpr int kLogG = G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : 4;
  using R = decltype(C().x);
  const PwConst<R> pc(geo);
  R acc = pc.zero;
  cg::cluster_group cl = cg::this_cluster();
  for (int base = warp * 16; base < spc; base += kWarps * 16) {
    const int sl = base + (lane & 15);
    const bool valid = sl < spc;
    const int s = geo.rank * spc + (valid ? sl : 0);
    // lanes l and l^16 hold columns k2 and M - k2 (slot 0: columns 0 and M/2, each
    // paired with itself)
    const int k2 = (lane < 16) ? s : (s == 0 ? (M >> 1) : M - s);
    const bool self0 = (k2 == 0), selfh = (k2 == (M >> 1));
    const int pos = swz(bitrev(k2, geo.logM), geo.logM);
    // twiddles of frequency k = k2 + M k1 as products of this lane's k2 part and a root of
    // order 2G (resp. 8G) shared by all lanes: w_N^k = w_N^k2 exp(-i pi k1 / G) and
    // eps^k = eps^k2 exp(-i pi k1 / (4G)) (N = 2 M G)
    // every global load of the slot (twiddles of this column, the G four-step twiddles kept
    // for the scatter, the G mask codes) is issued before the exchange's shared-memory reads
    const C wk2 = tw.root(k2, geo.logN), ek2 = tw.root(k2, geo.logN + 2);
    C t4[G];
    unsigned mcs[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      t4[g] = g == 0 ? wk2 : tw.root((int64_t)g * k2, geo.logL);
      mcs[g] = 0;
      if constexpr (MODE != MODE_FORWARD) {
        const int64_t k = (int64_t)k2 + (int64_t)M * g;
        if (geo.mcode) {
          mcs[g] = __ldg(&geo.mcode[k]);
        } else {
          const int64_t L = (int64_t)1 << geo.logL, N = geo.N;
          mcs[g] = (geo.mask[k] ? 1u : 0u) | ((k > 0 && geo.mask[N - k]) ? 2u : 0u) | (geo.mask[L - k] ? 4u : 0u) |
                   (geo.mask[L + k] ? 8u : 0u);
        }
      }
    }
    auto pw = [&](int k1, C a, C b, R& accr) -> C {
      const int64_t k = (int64_t)k2 + (int64_t)M * k1;
      C wN = wk2, eps = ek2;
      if (k1 != 0) {
        wN = cmul(wk2, tw.root(k1, kLogG + 1));
        eps = cmul(ek2, tw.root(k1, kLogG + 3));
      }
      return dct_pointwise_w<C, MODE, R>(k, a, b, wN, eps, mcs[k1], geo, pc, valid, accr, fwd_out);
    };
    C Z[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      C y;
      if constexpr (G == 1) {
        y = buf[pos];
      } else {
        y = cl.map_shared_rank(buf, g)[pos];
      }
      Z[g] = (g == 0) ? y : cmul(y, t4[g]);
    }
    small_dft<G>(Z, false, tw);  // Z[k1] = H[k2 + M k1]
    // column 0: H[M k1] pairs with H[M ((G - k1) mod G)] of the same column
    if (self0) {
      C T[G];
#pragma unroll
      for (int k1 = 0; k1 < G; ++k1) T[k1] = Z[k1];
#pragma unroll
      for (int k1 = 0; k1 < G; ++k1) Z[k1] = pw(k1, T[k1], T[(G - k1) % G], acc);
    }
    // other columns: H[k2 + M k1] pairs with H[(M - k2) + M (G-1-k1)], held by lane^16
    // (column M/2 pairs with itself the same way); update k1 and G-1-k1 together so
    // that no value is overwritten before the partner has read it
#pragma unroll
    for (int j = 0; j < (G + 1) / 2; ++j) {
      const int kA = j, kB = G - 1 - j;
      C bA, bB;
      bA.x = shfl_xor(Z[kB].x, 16);
      bA.y = shfl_xor(Z[kB].y, 16);
      bB.x = shfl_xor(Z[kA].x, 16);
      bB.y = shfl_xor(Z[kA].y, 16);
      if (selfh) {
        bA = Z[kB];
        bB = Z[kA];
      }
      if (!self0) {
        const C nA = pw(kA, Z[kA], bA, acc);
        if (kB != kA) {
          const C nB = pw(kB, Z[kB], bB, acc);
          Z[kB] = nB;
        }
        Z[kA] = nA;
      }
    }
    if constexpr (MODE != MODE_FORWARD) {
      small_dft<G>(Z, true, tw);
      if (valid) {
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const C y = (g == 0) ? Z[g] : cmulc(Z[g], t4[g]);
          if constexpr (G == 1) {
            buf[pos] = y;
          } else {
            cl.map_shared_rank(buf, g)[pos] = y;
          }
        }
      }
    }
  }
  return to_double(acc);
}

// buf (this CTA's chunk, storage order, as complex pairs) := D^-1 M (D buf - b_u) or
// D^-1 M D buf.  Returns this CTA's share of the masked coefficient energy.
template <int G, class C, int MODE>
__device__ double dct_chain(C* buf, const DctGeom& geo, const Twiddle<C>& tw, double* fwd_out = nullptr) {
  using R = decltype(C().x);
  fft_dif<C, R>(buf, geo.logM, tw);
  cluster_barrier<G>();
  const double acc = dct_slot_step<G, C, MODE>(buf, geo, tw, fwd_out);
  cluster_barrier<G>();
  if constexpr (MODE != MODE_FORWARD) fft_dit_inv<C, R>(buf, geo.logM, tw);
  return acc;
}

// natural index of storage position q (global over the cluster): CTA g = q / 2M holds the
// real q % 2M in shared-memory slot q' = (q % 2M) >> 1 as part q & 1, and slot q' holds complex
// element n2 = swz(q') of its M-point FFT input
__device__ __forceinline__ int64_t dct_natural_index(int64_t q, int logM, int G) {
  const int64_t M = (int64_t)1 << logM;
  const int64_t g = q / (2 * M), n2 = swz((int)((q % (2 * M)) >> 1), logM), part = q & 1;
  const int64_t j = g + (int64_t)G * n2;
  const int64_t N = 2 * M * G;
  const int64_t i = 2 * j + part;
  return i < N / 2 ? 2 * i : 2 * N - 1 - 2 * i;
}

template <int G> struct DctOp {
  DctGeom geo;
  double2* buf64;
  float2* buf32;
  Twiddle<double2> tw64;
  Twiddle<float2> tw32;
  Twiddle<dfc> twdf;
  int64_t chunk, gbase;
  double rho;
  int rank;

  __device__ void init(const ProbDesc& pd, const KernelArgs& a, unsigned char* smem, int rank_) {
    rank = rank_;
    geo.N = pd.n;
    geo.logN = pd.log2n;
    geo.logL = pd.log2n - 1;
    geo.logM = geo.logL - (G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : 4);
    geo.rank = rank_;
    geo.mask = pd.mask;
    geo.bsu = pd.bsu;
    geo.bsu_df = pd.bsu_df;
    geo.mcode = pd.mcode;
    geo.bpk = pd.bpk;
    geo.bpk_f64 = a.prm.resid_fp64 != 0;
    const int64_t M = (int64_t)1 << geo.logM;
    buf64 = reinterpret_cast<double2*>(smem);
    buf32 = reinterpret_cast<float2*>(smem + (size_t)16 * M);
    tw64 = Twiddle<double2>{a.tw64, a.log2_tw};
    tw32 = Twiddle<float2>{a.tw32, a.log2_tw};
    twdf = Twiddle<dfc>{a.twdf, a.log2_tw};
    chunk = 2 * M;
    gbase = (int64_t)rank_ * chunk;
    rho = (double)pd.m / (double)pd.n;  // A A^T = I: rho = m/n (Eq. eq:ne2_P)
  }
  __device__ __forceinline__ bool valid(int64_t) const { return true; }
  // residual buffer: this CTA's chunk of x (in) / A^T(Ax - b) (out), one value per storage
  // position, as float64 or as double-float (both 16 bytes per complex pair)
  template <class T> __device__ __forceinline__ T* rbuf() const { return reinterpret_cast<T*>(buf64); }
  // PCG operator buffer: float32 values in their own buffer; float64 values (the float64 PCG)
  // share the residual buffer, whose content every PCG initialisation consumes element by
  // element before writing the operator input in its place (same index, same thread)
  template <class PS> __device__ __forceinline__ PS* wbuf() const {
    if constexpr (sizeof(PS) == 8) {
      return reinterpret_cast<PS*>(buf64);
    } else {
      return reinterpret_cast<PS*>(buf32);
    }
  }
  // rbuf := A^T (A rbuf - b); returns this CTA's share of ||A x - b||^2
  template <class T> __device__ double resid_t() {
    if constexpr (std::is_same<T, df>::value) {
      return dct_chain<G, dfc, MODE_RESID>(reinterpret_cast<dfc*>(buf64), geo, twdf);
    } else {
      return dct_chain<G, double2, MODE_RESID>(buf64, geo, tw64);
    }
  }
  template <class PS> __device__ double normal(PS*) {
    if constexpr (sizeof(PS) == 8) {
      return dct_chain<G, double2, MODE_NORMAL>(buf64, geo, tw64);
    } else {
      return dct_chain<G, float2, MODE_NORMAL>(buf32, geo, tw32);
    }
  }
  // The same residual through the float32 chain on the operator buffer (the outer loop's
  // large-gap iterations): rbuf holds x on entry and A^T(Ax - b) on exit.
  static constexpr bool kLowpResid = true;
  template <class T> __device__ double resid_lowp() {
    T* rb = rbuf<T>();
    float* wb = wbuf<float>();
    for (int64_t q = threadIdx.x; q < chunk; q += kThreads) wb[q] = to_float(rb[q]);
    __syncthreads();
    const double acc = dct_chain<G, float2, MODE_RESID>(buf32, geo, tw32);
    for (int64_t q = threadIdx.x; q < chunk; q += kThreads) rb[q] = from_float<T>(wb[q]);
    __syncthreads();
    return acc;
  }
  // grad_b = A w for w in rbuf<double>() (float64 chain): all n DCT coefficients go to
  // pd.scratch, then the sampled rows are gathered.  Overwrites rbuf.
  __device__ void apply_A_out(const ProbDesc& pd) {
    dct_chain<G, double2, MODE_FORWARD>(buf64, geo, tw64, pd.scratch);
    __threadfence();
    cluster_barrier<G>();
    if (pd.grad_b)
      for (int64_t i = (int64_t)rank * kThreads + threadIdx.x; i < pd.m; i += (int64_t)G * kThreads)
        pd.grad_b[i] = pd.scratch[pd.rows[i]];
  }
  __device__ void grad_A_out(const ProbDesc&, const void*) {}
  __device__ int64_t natural(int64_t q) const { return dct_natural_index(gbase + q, geo.logM, G); }
  template <int GG> __device__ void setup(RedSmem&, int&) {}
};

// ------------------------------------------------------------------ dense op
// CTA rank r owns columns [r*chunk, (r+1)*chunk) of A (row-major m x n, float64).
// A w is summed over the cluster through DSMEM (an all-reduce of m values).
template <int G> struct DenseOp {
  const double* A;
  double a_scale;
  int64_t lda, m, n, chunk, gbase;
  double* buf64;
  void* bufP;
  double* tpart;  // m: this CTA's partial A w
  double* tfull;  // m: reduced A w (identical in every CTA)
  double* aw;     // m: A w kept by the backward
  const double* b;
  double rho;
  int rank;

  __device__ void init(const ProbDesc& pd, const KernelArgs&, unsigned char* smem, int rank_) {
    rank = rank_;
    A = static_cast<const double*>(pd.A);
    a_scale = pd.a_scale;
    lda = pd.lda;
    m = pd.m;
    n = pd.n;
    chunk = (n + G - 1) / G;
    gbase = (int64_t)rank * chunk;
    const size_t c8 = ((size_t)chunk * 8 + 255) & ~(size_t)255;
    buf64 = reinterpret_cast<double*>(smem);
    bufP = smem + c8;
    tpart = reinterpret_cast<double*>(smem + 2 * c8);
    tfull = tpart + ((m + 31) & ~31);
    aw = tfull + ((m + 31) & ~31);
    b = pd.b;
  }
  __device__ __forceinline__ bool valid(int64_t q) const { return gbase + q < n; }
  template <class T> __device__ __forceinline__ T* rbuf() const {
    static_assert(std::is_same<T, double>::value, "dense operators keep a float64 iterate");
    return reinterpret_cast<T*>(buf64);
  }
  template <class PS> __device__ __forceinline__ PS* wbuf() const { return reinterpret_cast<PS*>(bufP); }
  __device__ __forceinline__ int64_t natural(int64_t q) const { return gbase + q; }

  template <class PS, int MODE> __device__ double chain(PS* v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cols = min(chunk, n - gbase);
    // t_part = A[:, own] v
    for (int64_t i = warp; i < m; i += kWarps) {
      const double* Ai = A + i * lda + gbase;
      double s = 0.0;
      for (int64_t j = lane; j < cols; j += 32) s += __ldg(&Ai[j]) * (double)v[j];
      s = warp_sum(s);
      if (lane == 0) tpart[i] = s * a_scale;
    }
    cluster_barrier<G>();
    double acc = 0.0;
    cg::cluster_group cl = cg::this_cluster();
    for (int64_t i = threadIdx.x; i < m; i += kThreads) {
      double t = 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        if constexpr (G == 1) t += tpart[i]; else t += cl.map_shared_rank(tpart, g)[i];
      }
      if (MODE == MODE_RESID) t -= b[i];
      tfull[i] = t;
      if (rank == 0) acc += t * t;
    }
    __syncthreads();
    if constexpr (MODE == MODE_FORWARD) return acc;
    // v = A[:, own]^T t
    for (int64_t j = threadIdx.x; j < cols; j += kThreads) {
      const double* Aj = A + gbase + j;
      double s0 = 0.0, s1 = 0.0;
      int64_t i = 0;
      for (; i + 1 < m; i += 2) {
        s0 += __ldg(&Aj[i * lda]) * tfull[i];
        s1 += __ldg(&Aj[(i + 1) * lda]) * tfull[i + 1];
      }
      if (i < m) s0 += __ldg(&Aj[i * lda]) * tfull[i];
      v[j] = (PS)((s0 + s1) * a_scale);
    }
    __syncthreads();
    return acc;
  }
  template <class T> __device__ double resid_t() { return chain<double, MODE_RESID>(buf64); }
  static constexpr bool kLowpResid = false;
  template <class T> __device__ double resid_lowp() { return resid_t<T>(); }
  // grad_b = A w for w in rbuf<double>(); keeps A w in aw for grad_A_out
  __device__ void apply_A_out(const ProbDesc& pd) {
    chain<double, MODE_FORWARD>(buf64);
    for (int64_t i = threadIdx.x; i < m; i += kThreads) {
      aw[i] = tfull[i];
      if (pd.grad_b && rank == 0) pd.grad_b[i] = tfull[i];
    }
    __syncthreads();
  }
  // dL/dA = r w^T - (A w) x^T with r = b - A x, for this CTA's columns; w from the PCG pairs
  template <class P2> __device__ void grad_A_out(const ProbDesc& pd, const P2* Y) {
    const int64_t cols = min(chunk, n - gbase);
    for (int64_t q = threadIdx.x; q < chunk; q += kThreads) buf64[q] = (q < cols) ? pd.x_in[gbase + q] : 0.0;
    __syncthreads();
    chain<double, MODE_RESID>(buf64);  // tfull = A x - b
    for (int64_t idx = threadIdx.x; idx < m * cols; idx += kThreads) {
      const int64_t i = idx / cols, j = idx % cols;
      const P2 y = Y[gbase + j];
      const double wj = (double)y.x - (double)y.y;
      pd.grad_A[i * n + gbase + j] = -tfull[i] * wj - aw[i] * pd.x_in[gbase + j];
    }
  }
  template <class PS> __device__ double normal(PS* v) { return chain<PS, MODE_NORMAL>(v); }

  // rho = ||A||_F^2 / n: the Frobenius-closest multiple of I to A^T A (equals m/n when
  // A A^T = I, Eq. eq:ne2_P)
  template <int GG> __device__ void setup(RedSmem& rs, int& par) {
    const int64_t cols = min(chunk, n - gbase);
    double s = 0.0;
    for (int64_t idx = threadIdx.x; idx < m * cols; idx += kThreads) {
      const int64_t i = idx / cols, j = idx % cols;
      const double a = __ldg(&A[i * lda + gbase + j]) * a_scale;
      s += a * a;
    }
    double v[1] = {s};
    cluster_reduce<GG, 1>(rs, par, v, [&](const double (&t)[1]) { rs.sd[0] = t[0] / (double)n; });
    rho = rs.sd[0];
  }
};

// ------------------------------------------------------------------ the IPM driver
// Precision split of the per-index work.  Kept in float64: the iterate (z, s) and its
// update, x = u - v, the residual A^T(Ax - b) and the dual-residual terms tau +/- g built
// from it, and the scalar reductions across the cluster.  Computed in the PCG precision H
// (float32 for the partial DCT): quantities that only steer the iteration or feed the
// float32 PCG -- Theta^-1 = s/z, sigma*mu/z, the direction components and the
// step-to-boundary ratios.  Both uses of a direction (ratio test and update) evaluate it
// through the same function from the same inputs, so the fraction-to-boundary rule keeps
// z, s > 0.
template <class H> struct ScH {
  H smu, ap1, ad1, s3mut;
  bool corr;
  bool mcc;  // multiple centrality correctors: the second vector holds the summed targets t
};

__device__ __forceinline__ float rcpH(float z) { return __frcp_rn(z); }
__device__ __forceinline__ double rcpH(double z) { return rcp64(z); }

template <class H> struct Dir {
  H dz, ds;
};
// dz and ds of one index (Eq. redNewtonB):
//   predictor ds1 = Z^-1 f_s - Theta^-1 dz1 = sigma mu / z - s - (s / z) dz1
//   corrector ds2 = Z^-1 f_s~ - Theta^-1 dz2, f_s~ = sigma3 mu~ - z~ s~ at the trial point
//             z~ = z + alpha_p1 dz1, s~ = s + alpha_d1 ds1 (reading: Theta and Z of the current
//             point); the combined direction is (dz1 + dz2, ds1 + ds2)
template <class H>
__device__ __forceinline__ Dir<H> direction(H z, H s, H dz1, H dz2, const ScH<H>& c) {
  const H rz = rcpH(z);
  const H d = s * rz;
  // with centrality correctors (reading R19) dz1 is the summed direction and dz2 the summed
  // targets T: ds = Z^-1 (f_s + T) - Theta^-1 dz (Eq. redNewtonB, right-hand side f_s + T)
  const H ds1 = ((c.mcc ? c.smu + dz2 : c.smu) * rz - s) - d * dz1;
  Dir<H> r{dz1, ds1};
  if (c.corr) {
    const H zt = z + c.ap1 * dz1;
    const H st = s + c.ad1 * ds1;
    const H ds2 = (c.s3mut - zt * st) * rz - d * dz2;
    r.dz = dz1 + dz2;
    r.ds = ds1 + ds2;
  }
  return r;
}

// ------------------------------------------------------------------ iterate storage
// The iterate z = [u; v], s = [s_u; s_v] is kept per index as {u, v, s_u, s_v} (32 bytes)
// either in float64 (StateF64) or in double-float (StateDF: two float32 words per value,
// about 48 significant bits, all arithmetic on the float32 pipes).  Both policies expose
// the same operations on their component type T.
struct StateF64 {
  using T = double;
  struct Q { double u, v, su, sv; };
  __device__ static __forceinline__ Q load(const void* zs, int64_t gi) {
    const double2* p = static_cast<const double2*>(zs) + 2 * gi;
    const double2 z = p[0], s = p[1];
    return Q{z.x, z.y, s.x, s.y};
  }
  __device__ static __forceinline__ void store(void* zs, int64_t gi, const Q& q) {
    double2* p = static_cast<double2*>(zs) + 2 * gi;
    p[0] = make_double2(q.u, q.v);
    p[1] = make_double2(q.su, q.sv);
  }
  __device__ static __forceinline__ float hf(double a) { return (float)a; }
  __device__ static __forceinline__ double axpy(double z, double a, float d) { return fma(a, (double)d, z); }
  __device__ static __forceinline__ double sub(double a, double b) { return a - b; }
  __device__ static __forceinline__ double add(double a, double b) { return a + b; }
  __device__ static __forceinline__ bool positive(double a) { return a > 0.0; }
  __device__ static __forceinline__ double scale(double a, double k) { return a * k; }
  __device__ static __forceinline__ double from_d(double a) { return a; }
  __device__ static __forceinline__ double to_d(double a) { return a; }
};
struct StateDF {
  using T = df;
  struct Q { df u, v, su, sv; };
  __device__ static __forceinline__ Q load(const void* zs, int64_t gi) {
    const float4* p = static_cast<const float4*>(zs) + 2 * gi;
    const float4 z = p[0], s = p[1];
    return Q{df(z.x, z.y), df(z.z, z.w), df(s.x, s.y), df(s.z, s.w)};
  }
  __device__ static __forceinline__ void store(void* zs, int64_t gi, const Q& q) {
    float4* p = static_cast<float4*>(zs) + 2 * gi;
    p[0] = make_float4(q.u.hi, q.u.lo, q.v.hi, q.v.lo);
    p[1] = make_float4(q.su.hi, q.su.lo, q.sv.hi, q.sv.lo);
  }
  __device__ static __forceinline__ float hf(df a) { return a.hi; }
  __device__ static __forceinline__ df axpy(df z, df a, float d) { return z + a * df(d); }
  __device__ static __forceinline__ df sub(df a, df b) { return a - b; }
  __device__ static __forceinline__ df add(df a, df b) { return a + b; }
  __device__ static __forceinline__ bool positive(df a) { return a.hi > 0.f; }
  __device__ static __forceinline__ df scale(df a, df k) { return a * k; }
  __device__ static __forceinline__ df from_d(double a) { return to_df(a); }
  __device__ static __forceinline__ double to_d(df a) { return to_double(a); }
};

// Scalars of one solve, written by thread 0 inside cluster_reduce and read by every
// thread after its closing barrier (identical in all CTAs of the cluster).
template <class H, class T> struct IpmShared {
  double mu, sigma, alpha_p, alpha_d, mu_t, alpha_p1, alpha_d1, prev_ap, prev_ad;
  double rel_gap, P_obj, cn, rz0, rz;
  T apT, adT, ap1T, ad1T, tauT, keepT;  // step lengths etc. in the iterate's arithmetic
  H smu, ap1, ad1, s3mut, apH, adH, alpha, beta;
  int corr, corr_next, stop, pcg_stop, pcg_brk, correctors;
  int lowp, redo;  // outer residual in float32 (large gap); recompute it in full precision
  int mcc_on, mcc_acc;  // centrality correctors enabled; the last one was accepted
};

template <class H, class T>
__device__ __forceinline__ ScH<H> steering(const IpmShared<H, T>& sh, bool corr) {
  ScH<H> c;
  c.smu = sh.smu;
  c.ap1 = sh.ap1;
  c.ad1 = sh.ad1;
  c.s3mut = sh.s3mut;
  c.corr = corr;
  c.mcc = sh.mcc_on != 0;
  return c;
}

// Correction of one complementarity product v = z~ s~ toward [beta_min mu_t, beta_max mu_t]
// (multiple centrality correctors, reading R19).
template <class H> __device__ __forceinline__ H centrality_t(H v, H lo, H hi) {
  if (v < lo) return lo - v;
  if (v > hi) return fmax(hi - v, -hi);
  return (H)0;
}

// PCG on (Theta^-1 + F F^T) y = rhs (Sec. 4, preconditioner of Eq. eq:ne2_P).  On entry
// r = rhs and p = P^-1 r are stored, the operator input w = p_u - p_v is in the shared buffer,
// and rz_part, pdp_part are this thread's shares of r.P^-1 r and p.(Theta^-1 p).  Stops when
// sqrt(r.P^-1 r) <= tol * its initial value (reading R9) or after max_iter iterations; y = 0
// for a zero right-hand side.  Returns the iteration count; adds 2 per iteration to nmat.
template <int G, class Op, class PS, class SH>
__device__ int pcg_solve(Op& op, RedSmem& rs, SH& sh, int& par, typename V2<PS>::T* __restrict__ Xo,
                         typename V2<PS>::T* __restrict__ Rv, typename V2<PS>::T* __restrict__ Pv,
                         const typename V2<PS>::T* __restrict__ Dv, PS* __restrict__ w, PS rho, double tol,
                         int max_iter, PS rz_part, PS pdp_part, int64_t& nmat) {
  using P2 = typename V2<PS>::T;
  const int tid = threadIdx.x;
  const int64_t chunk = op.chunk, gb = op.gbase;
  int k = 0;
  PS pdp_acc = pdp_part;
  for (;;) {
    const double aw2 = op.normal(w);
    nmat += 2;
    {
      PS v[2] = {pdp_acc + (PS)aw2, k == 0 ? rz_part : (PS)0};
      cluster_reduce<G, 2>(rs, par, v, [&](const double (&t)[2]) {
        if (k == 0) {
          sh.rz0 = sh.rz = t[1];
          sh.pcg_stop = !(t[1] > 0.0) || !isfinite(t[1]);
        }
        // breakdown guard: a direction with p^T H p not positive and finite (rounding when
        // Theta^-1 spans many orders of magnitude) ends the solve with the last iterate
        const double a_ = sh.rz / t[0];
        sh.pcg_brk = !(t[0] > 0.0) || !isfinite(t[0]) || !isfinite(a_) || !isfinite((double)(PS)a_);
        sh.alpha = (PS)a_;
      });
    }
    if (sh.pcg_brk && !sh.pcg_stop && k > 0) break;  // keep the iterate of the last step
    if (sh.pcg_stop || sh.pcg_brk) {  // zero right-hand side (or breakdown at once): y = 0
      P2 zero;
      zero.x = (PS)0;
      zero.y = (PS)0;
      for (int64_t q = tid; q < chunk; q += kThreads)
        if (op.valid(q)) Xo[gb + q] = zero;
      break;
    }
    const PS alpha = sh.alpha;
    PS rzn_part = 0;
    const bool first = (k == 0);
#pragma unroll 4
    for (int64_t q = tid; q < chunk; q += kThreads) {
      if (!op.valid(q)) continue;
      const int64_t gi = gb + q;
      const P2 p = Pv[gi], d = Dv[gi];
      P2 r = Rv[gi];
      P2 x;
      if (first) { x.x = (PS)0; x.y = (PS)0; } else { x = Xo[gi]; }
      const PS y = w[q];
      const PS qu = d.x * p.x + y, qv = d.y * p.y - y;
      x.x += alpha * p.x;
      x.y += alpha * p.y;
      r.x -= alpha * qu;
      r.y -= alpha * qv;
      const P2 zz = precond<PS>(d, r, rho);
      rzn_part += r.x * zz.x + r.y * zz.y;
      Xo[gi] = x;
      Rv[gi] = r;
    }
    ++k;
    {
      PS v[1] = {rzn_part};
      cluster_reduce<G, 1>(rs, par, v, [&](const double (&t)[1]) {
        const double rzn = t[0];
        sh.pcg_stop = !(rzn > tol * tol * sh.rz0) || k >= max_iter || !isfinite(rzn);
        sh.beta = (PS)(rzn / sh.rz);
        sh.rz = rzn;
      });
    }
    if (sh.pcg_stop) break;
    const PS beta = sh.beta;
    PS pdp = 0;
#pragma unroll 4
    for (int64_t q = tid; q < chunk; q += kThreads) {
      if (!op.valid(q)) { w[q] = (PS)0; continue; }
      const int64_t gi = gb + q;
      const P2 d = Dv[gi], r = Rv[gi];
      P2 p = Pv[gi];
      const P2 zz = precond<PS>(d, r, rho);
      p.x = zz.x + beta * p.x;
      p.y = zz.y + beta * p.y;
      Pv[gi] = p;
      w[q] = p.x - p.y;
      pdp += d.x * p.x * p.x + d.y * p.y * p.y;
    }
    __syncthreads();
    pdp_acc = pdp;
  }
  return k;
}

template <int G, class Op, class PS, class S>
__device__ void solve_one(const ProbDesc& pd, const KernelArgs& a, Op& op, RedSmem& rs,
                          IpmShared<PS, typename S::T>& sh, int& par) {
  using P2 = typename V2<PS>::T;
  using H = PS;
  using T = typename S::T;
  using Q = typename S::Q;
  const SolveParams& prm = a.prm;
  const int tid = threadIdx.x;
  const int64_t n = pd.n;
  const double tau = pd.tau;
  const int64_t chunk = op.chunk, gb = op.gbase;
  void* __restrict__ zs = pd.zs;
  P2* __restrict__ X1 = reinterpret_cast<P2*>(pd.pcg);
  P2* __restrict__ X2 = X1 + n;
  P2* __restrict__ Rv = X2 + n;
  P2* __restrict__ Pv = Rv + n;
  P2* __restrict__ Dv = Pv + n;
  P2* __restrict__ Xc = Dv + n;  // a centrality corrector's direction before it is accepted
  T* __restrict__ gbuf = op.template rbuf<T>();
  PS* __restrict__ w = op.template wbuf<PS>();
  const T zeroT = S::from_d(0.0);
  int64_t nmat = 0;
  int pcg_total = 0, it = 0;

  op.template setup<G>(rs, par);
  const PS rho = (PS)op.rho;

  // ||c||^2 = sum 2 tau^2 + 2 (A^T b)_i^2 with A^T b = -A^T (A 0 - b)  (c: Sec. 3)
  for (int64_t q = tid; q < chunk; q += kThreads) gbuf[q] = zeroT;
  __syncthreads();
  {
    const double bb = op.template resid_t<T>();
    ++nmat;
    double atb2 = 0.0, atbmax = 0.0;
    for (int64_t q = tid; q < chunk; q += kThreads)
      if (op.valid(q)) {
        const double g = S::to_d(gbuf[q]);
        atb2 += g * g;
        atbmax = fmax(atbmax, fabs(g));
      }
    {
      // the float32 residual chain errs by ~1e-6 ||A^T b||_inf; it is used only while that
      // stays three orders below tau, the scale of the dual residual f_z = s - tau -+ g
      double vm[1] = {-atbmax};
      cluster_reduce<G, 1, true>(rs, par, vm, [&](const double (&t)[1]) {
        sh.lowp = Op::kLowpResid && prm.f32_gap > 0.0 && tau >= 1e-3 * (-t[0]);
      });
    }
    double v[2] = {atb2, bb};
    cluster_reduce<G, 2>(rs, par, v, [&](const double (&t)[2]) {
      sh.cn = sqrt(2.0 * (double)n * tau * tau + 2.0 * t[0]);
      sh.alpha_p = sh.alpha_d = 1.0;
      sh.prev_ap = sh.prev_ad = 1.0;
      sh.apH = sh.adH = (H)1;
      sh.apT = sh.adT = S::from_d(1.0);
      sh.tauT = S::from_d(tau);
      sh.keepT = S::from_d(1.0 - prm.eta);
      sh.corr = sh.corr_next = 0;
      sh.correctors = 0;
      sh.stop = 0;
      sh.redo = 0;
      sh.mcc_on = prm.mcc > 0;
      sh.mcc_acc = 0;
      sh.rel_gap = INFINITY;
      sh.P_obj = 0.0;
    });
  }
  const T tauT = sh.tauT, keepT = sh.keepT;

  auto pcg = [&](P2* __restrict__ Xo, PS rz_part, PS pdp_part) {
    pcg_total += pcg_solve<G>(op, rs, sh, par, Xo, Rv, Pv, Dv, w, rho, prm.tol_pcg, prm.max_iter_pcg, rz_part,
                              pdp_part, nmat);
  };

  // PCG initialisation: r = rhs (from rhs_fn(q, gi, state) in precision H), p = P^-1 r,
  // w = p_u - p_v.  Writes Theta^-1 = s/z when write_d.
  auto pcg_init = [&](auto rhs_fn, bool write_d, PS& rz_part, PS& pdp_part) {
    rz_part = 0;
    pdp_part = 0;
#pragma unroll 2
    for (int64_t q = tid; q < chunk; q += kThreads) {
      if (!op.valid(q)) { w[q] = (PS)0; continue; }
      const int64_t gi = gb + q;
      const Q st = S::load(zs, gi);
      P2 d;
      if (write_d) {
        d.x = (H)S::hf(st.su) * rcpH((H)S::hf(st.u));
        d.y = (H)S::hf(st.sv) * rcpH((H)S::hf(st.v));
        Dv[gi] = d;
      } else {
        d = Dv[gi];
      }
      const P2 r = rhs_fn(q, gi, st);
      const P2 p = precond<PS>(d, r, rho);
      Rv[gi] = r;
      Pv[gi] = p;
      w[q] = p.x - p.y;
      rz_part += r.x * p.x + r.y * p.y;
      pdp_part += d.x * p.x * p.x + d.y * p.y * p.y;
    }
    __syncthreads();
  };

  auto load_dir = [&](int64_t gi, const Q& st, const ScH<H>& c, Dir<H>& du, Dir<H>& dv) {
    const P2 x1 = X1[gi];
    P2 x2;
    x2.x = (PS)0;
    x2.y = (PS)0;
    if (c.corr || c.mcc) x2 = X2[gi];
    du = direction<H>((H)S::hf(st.u), (H)S::hf(st.su), x1.x, x2.x, c);
    dv = direction<H>((H)S::hf(st.v), (H)S::hf(st.sv), x1.y, x2.y, c);
  };

  // step lengths alpha = min(1, eta * min_{dv<0} -v/dv) for z and s (reading R4); then the
  // corrector test of the Algorithm (alpha_P or alpha_D <= alpha_tilde)
  auto step_lengths = [&](bool corr) {
    const ScH<H> c = steering(sh, corr);
    H mp = (H)INFINITY, md = (H)INFINITY;
#pragma unroll 2
    for (int64_t q = tid; q < chunk; q += kThreads) {
      if (!op.valid(q)) continue;
      const int64_t gi = gb + q;
      const Q st = S::load(zs, gi);
      Dir<H> du, dv;
      load_dir(gi, st, c, du, dv);
      if (du.dz < (H)0) mp = fmin(mp, (H)S::hf(st.u) * rcpH(-du.dz));
      if (dv.dz < (H)0) mp = fmin(mp, (H)S::hf(st.v) * rcpH(-dv.dz));
      if (du.ds < (H)0) md = fmin(md, (H)S::hf(st.su) * rcpH(-du.ds));
      if (dv.ds < (H)0) md = fmin(md, (H)S::hf(st.sv) * rcpH(-dv.ds));
    }
    H v[2] = {mp, md};
    cluster_reduce<G, 2, true>(rs, par, v, [&](const double (&t)[2]) {
      double ap = fmin(1.0, prm.eta * t[0]);
      double ad = fmin(1.0, prm.eta * t[1]);
      if (prm.equal_steps) ap = ad = fmin(ap, ad);
      sh.alpha_p = ap;
      sh.alpha_d = ad;
      sh.apH = (H)ap;
      sh.adH = (H)ad;
      sh.apT = S::from_d(ap);
      sh.adT = S::from_d(ad);
      sh.corr_next = (corr || sh.mcc_on) ? 0 : (ap <= prm.alpha_tilde || ad <= prm.alpha_tilde);
      if (sh.corr_next) {
        sh.alpha_p1 = ap;
        sh.alpha_d1 = ad;
        sh.ap1 = (H)ap;
        sh.ad1 = (H)ad;
        sh.ap1T = sh.apT;
        sh.ad1T = sh.adT;
        ++sh.correctors;
      }
      sh.corr = corr;
      sh.prev_ap = ap;
      sh.prev_ad = ad;
    });
  };

  for (it = 1;; ++it) {
    // ---- update (previous direction) fused with x = u - v for the residual
    H part[3] = {0, 0, 0};  // z.s, 1^T z, ||x||^2
    {
      const ScH<H> c = steering(sh, sh.corr != 0);
      const T apT = sh.apT, adT = sh.adT;
      const H apH = sh.apH, adH = sh.adH;
#pragma unroll 2
      for (int64_t q = tid; q < chunk; q += kThreads) {
        if (!op.valid(q)) { gbuf[q] = zeroT; continue; }
        const int64_t gi = gb + q;
        Q st;
        H zu, zv, su, sv;
        if (it == 1) {
          const T one = S::from_d(1.0);  // reading R3: z0 = s0 = 1
          st = Q{one, one, one, one};
          zu = zv = su = sv = (H)1;
        } else {
          const Q o = S::load(zs, gi);
          Dir<H> du, dv;
          load_dir(gi, o, c, du, dv);
          st.u = S::axpy(o.u, apT, du.dz);
          st.v = S::axpy(o.v, apT, dv.dz);
          st.su = S::axpy(o.su, adT, du.ds);
          st.sv = S::axpy(o.sv, adT, dv.ds);
          // the step keeps z, s > 0 by construction; guard against a rounding-level crossing
          if (!S::positive(st.u)) st.u = S::scale(o.u, keepT);
          if (!S::positive(st.v)) st.v = S::scale(o.v, keepT);
          if (!S::positive(st.su)) st.su = S::scale(o.su, keepT);
          if (!S::positive(st.sv)) st.sv = S::scale(o.sv, keepT);
          zu = (H)S::hf(o.u) + apH * du.dz;
          zv = (H)S::hf(o.v) + apH * dv.dz;
          su = (H)S::hf(o.su) + adH * du.ds;
          sv = (H)S::hf(o.sv) + adH * dv.ds;
        }
        S::store(zs, gi, st);
        gbuf[q] = S::sub(st.u, st.v);
        const H xh = zu - zv;
        part[0] += zu * su + zv * sv;
        part[1] += zu + zv;
        part[2] += xh * xh;
      }
    }
    __syncthreads();
    // ---- residual g = A^T (A x - b)  (f_z of Eq. fzfs needs F F^T z + c).  While the relative
    // gap exceeds f32_gap the chain runs in float32: the Newton directions of those iterations
    // are inexact to ~tol_pcg anyway, and each iteration recomputes the residual from scratch,
    // so its rounding does not carry over.  At the first iteration whose gap falls to f32_gap,
    // and before any stop, the residual of that iterate is recomputed in the outer loop's
    // precision, which every later iteration keeps.
    for (;;) {
      const double res2 = sh.lowp ? op.template resid_lowp<T>() : op.template resid_t<T>();
      nmat += 2;
      double v[4] = {(double)part[0], (double)part[1], (double)part[2], res2};
      const int itc = it;
      cluster_reduce<G, 4>(rs, par, v, [&](const double (&t)[4]) {
        sh.mu = t[0] / (2.0 * (double)n);
        sh.P_obj = tau * t[1] + 0.5 * t[3];
        sh.rel_gap = t[0] / (1.0 + fabs(sh.P_obj));
        sh.corr = 0;
        if (!isfinite(sh.rel_gap)) sh.stop = MFIPM_NUMERIC;
        else if (sh.rel_gap <= prm.tol) sh.stop = -1;                       // converged (reading R7)
        else if (itc > prm.max_iter) sh.stop = MFIPM_NOT_CONVERGED;
        sh.redo = sh.lowp && (sh.stop != 0 || !(sh.rel_gap > prm.f32_gap));
        if (sh.redo) {
          sh.lowp = 0;
          sh.stop = 0;
        }
        // predictor centering (Algorithm; reading R8)
        sh.sigma = (itc != 1 && (sh.prev_ap <= prm.alpha_bar || sh.prev_ad <= prm.alpha_bar)) ? prm.sigma2 : prm.sigma1;
        sh.smu = (H)(sh.sigma * sh.mu);
      });
      if (!sh.redo) break;
      // x = u - v of the iterate again (the chain replaced it by the residual)
      for (int64_t q = tid; q < chunk; q += kThreads) {
        if (!op.valid(q)) { gbuf[q] = zeroT; continue; }
        const Q st = S::load(zs, gb + q);
        gbuf[q] = S::sub(st.u, st.v);
      }
      __syncthreads();
    }
    if (sh.stop) break;
    // ---- predictor
    PS rzp, pdpp;
    {
      const H smuH = sh.smu;
      // rhs = f_z + Z^-1 f_s = sigma mu / z - (c + F F^T z) = sigma mu / z - [tau + g; tau - g]
      const bool mcc = sh.mcc_on != 0;
      pcg_init([&](int64_t q, int64_t gi, const Q& st) {
                 const T g = gbuf[q];
                 P2 r;
                 r.x = smuH * rcpH((H)S::hf(st.u)) - (H)S::hf(S::add(tauT, g));
                 r.y = smuH * rcpH((H)S::hf(st.v)) - (H)S::hf(S::sub(tauT, g));
                 if (mcc) {  // no centrality targets yet
                   P2 zero;
                   zero.x = (PS)0;
                   zero.y = (PS)0;
                   X2[gi] = zero;
                 }
                 return r;
               }, true, rzp, pdpp);
    }
    pcg(X1, rzp, pdpp);
    step_lengths(false);
    // ---- multiple centrality correctors (reading R19), in place of the single corrector
    for (int kc = 0; sh.mcc_on && kc < prm.mcc; ++kc) {
      if (sh.alpha_p >= 1.0 && sh.alpha_d >= 1.0) break;
      const ScH<H> c = steering(sh, false);
      const H apt = (H)fmin(1.0, sh.alpha_p + prm.mcc_delta), adt = (H)fmin(1.0, sh.alpha_d + prm.mcc_delta);
      const H lo = (H)(prm.mcc_beta_min * sh.sigma * sh.mu), hi = (H)(prm.mcc_beta_max * sh.sigma * sh.mu);
      // targets of this corrector from the current summed direction, at the aspiration steps
      auto targets = [&](int64_t gi, const Q& st, P2& tv) {
        Dir<H> du, dv;
        load_dir(gi, st, c, du, dv);
        const H zu = (H)S::hf(st.u), zv = (H)S::hf(st.v);
        tv.x = centrality_t<H>((zu + apt * du.dz) * ((H)S::hf(st.su) + adt * du.ds), lo, hi);
        tv.y = centrality_t<H>((zv + apt * dv.dz) * ((H)S::hf(st.sv) + adt * dv.ds), lo, hi);
      };
      // (Theta^-1 + F F^T) dz~ = Z^-1 t  (right-hand side (f_z, f_s) = (0, t))
      pcg_init([&](int64_t, int64_t gi, const Q& st) {
                 P2 tv;
                 targets(gi, st, tv);
                 P2 r;
                 r.x = tv.x * rcpH((H)S::hf(st.u));
                 r.y = tv.y * rcpH((H)S::hf(st.v));
                 return r;
               }, false, rzp, pdpp);
      pcg(Xc, rzp, pdpp);
      // step lengths of the sum (dz + dz~, T + t); keep it when the smaller step grows by
      // at least gamma * delta
      {
        H mp = (H)INFINITY, md = (H)INFINITY;
        for (int64_t q = tid; q < chunk; q += kThreads) {
          if (!op.valid(q)) continue;
          const int64_t gi = gb + q;
          const Q st = S::load(zs, gi);
          P2 tv;
          targets(gi, st, tv);
          const P2 x1 = X1[gi], xc = Xc[gi], x2 = X2[gi];
          const Dir<H> du = direction<H>((H)S::hf(st.u), (H)S::hf(st.su), x1.x + xc.x, x2.x + tv.x, c);
          const Dir<H> dv = direction<H>((H)S::hf(st.v), (H)S::hf(st.sv), x1.y + xc.y, x2.y + tv.y, c);
          if (du.dz < (H)0) mp = fmin(mp, (H)S::hf(st.u) * rcpH(-du.dz));
          if (dv.dz < (H)0) mp = fmin(mp, (H)S::hf(st.v) * rcpH(-dv.dz));
          if (du.ds < (H)0) md = fmin(md, (H)S::hf(st.su) * rcpH(-du.ds));
          if (dv.ds < (H)0) md = fmin(md, (H)S::hf(st.sv) * rcpH(-dv.ds));
        }
        H v[2] = {mp, md};
        cluster_reduce<G, 2, true>(rs, par, v, [&](const double (&t)[2]) {
          double ap = fmin(1.0, prm.eta * t[0]);
          double ad = fmin(1.0, prm.eta * t[1]);
          if (prm.equal_steps) ap = ad = fmin(ap, ad);
          sh.mcc_acc = fmin(ap, ad) >= fmin(sh.alpha_p, sh.alpha_d) + prm.mcc_gamma * prm.mcc_delta;
          if (sh.mcc_acc) {
            sh.alpha_p = ap;
            sh.alpha_d = ad;
            sh.apH = (H)ap;
            sh.adH = (H)ad;
            sh.apT = S::from_d(ap);
            sh.adT = S::from_d(ad);
            sh.prev_ap = ap;
            sh.prev_ad = ad;
            ++sh.correctors;
          }
        });
      }
      if (!sh.mcc_acc) break;
      // accept: dz += dz~, T += t (the targets from the direction before the sum)
      for (int64_t q = tid; q < chunk; q += kThreads) {
        if (!op.valid(q)) continue;
        const int64_t gi = gb + q;
        const Q st = S::load(zs, gi);
        P2 tv;
        targets(gi, st, tv);
        P2 x1 = X1[gi], x2 = X2[gi];
        const P2 xc = Xc[gi];
        x1.x += xc.x;
        x1.y += xc.y;
        x2.x += tv.x;
        x2.y += tv.y;
        X1[gi] = x1;
        X2[gi] = x2;
      }
      __syncthreads();
    }
    // ---- corrector (reading R6)
    if (sh.corr_next && !sh.mcc_on) {
      H zts_t = 0;
      {
        const ScH<H> c = steering(sh, false);  // predictor direction only
        const T ap1T = sh.ap1T;
#pragma unroll 2
        for (int64_t q = tid; q < chunk; q += kThreads) {
          if (!op.valid(q)) { gbuf[q] = zeroT; continue; }
          const int64_t gi = gb + q;
          const Q st = S::load(zs, gi);
          Dir<H> du, dv;
          load_dir(gi, st, c, du, dv);
          gbuf[q] = S::sub(S::axpy(st.u, ap1T, du.dz), S::axpy(st.v, ap1T, dv.dz));
          const H zu = (H)S::hf(st.u) + c.ap1 * du.dz, zv = (H)S::hf(st.v) + c.ap1 * dv.dz;
          const H su = (H)S::hf(st.su) + c.ad1 * du.ds, sv = (H)S::hf(st.sv) + c.ad1 * dv.ds;
          zts_t += zu * su + zv * sv;
        }
      }
      __syncthreads();
      if (sh.lowp) op.template resid_lowp<T>();
      else op.template resid_t<T>();
      nmat += 2;
      {
        PS v[1] = {zts_t};
        cluster_reduce<G, 1>(rs, par, v, [&](const double (&t)[1]) {
          sh.mu_t = t[0] / (2.0 * (double)n);
          sh.s3mut = (H)(prm.sigma3 * sh.mu_t);
        });
      }
      {
        const ScH<H> c = steering(sh, false);
        const T ad1T = sh.ad1T;
        // rhs~ = f_z~ + Z^-1 f_s~ with f_z~ = s~ - [tau + g~; tau - g~] (iterate arithmetic),
        // f_s~ = sigma3 mu~ - z~ s~
        pcg_init([&](int64_t q, int64_t gi, const Q& st) {
                   const T g = gbuf[q];
                   Dir<H> du, dv;
                   load_dir(gi, st, c, du, dv);
                   const H zu = (H)S::hf(st.u) + c.ap1 * du.dz, zv = (H)S::hf(st.v) + c.ap1 * dv.dz;
                   const H su = (H)S::hf(st.su) + c.ad1 * du.ds, sv = (H)S::hf(st.sv) + c.ad1 * dv.ds;
                   const T fzu = S::sub(S::axpy(st.su, ad1T, du.ds), S::add(tauT, g));
                   const T fzv = S::sub(S::axpy(st.sv, ad1T, dv.ds), S::sub(tauT, g));
                   P2 r;
                   r.x = (H)S::hf(fzu) + (c.s3mut - zu * su) * rcpH((H)S::hf(st.u));
                   r.y = (H)S::hf(fzv) + (c.s3mut - zv * sv) * rcpH((H)S::hf(st.v));
                   return r;
                 }, false, rzp, pdpp);
      }
      pcg(X2, rzp, pdpp);
      step_lengths(true);
    }
  }

  // ---- exit: certificates and outputs in float64 (gbuf holds A^T(Ax - b) of the final iterate)
  double fin[3] = {0.0, 0.0, 0.0};  // ||f_z||^2, kkt^2, ||x||^2
  for (int64_t q = tid; q < chunk; q += kThreads) {
    if (!op.valid(q)) continue;
    const int64_t gi = gb + q;
    const Q st = S::load(zs, gi);
    const double g = S::to_d(gbuf[q]);
    const double u = S::to_d(st.u), v = S::to_d(st.v), su = S::to_d(st.su), sv = S::to_d(st.sv);
    const double fzu = su - (tau + g), fzv = sv - (tau - g);
    const double x = S::to_d(S::sub(st.u, st.v));
    const double y = x - g;
    const double sth = copysign(fmax(fabs(y) - tau, 0.0), y);
    fin[0] += fzu * fzu + fzv * fzv;
    fin[1] += (x - sth) * (x - sth);
    fin[2] += x * x;
    const int64_t ni = op.natural(q);
    pd.x_out[ni] = x;
    if (pd.zs_out) {
      pd.zs_out[ni] = u;
      pd.zs_out[n + ni] = v;
      pd.zs_out[2 * n + ni] = su;
      pd.zs_out[3 * n + ni] = sv;
    }
  }
  const int its = it;
  cluster_reduce<G, 3>(rs, par, fin, [&](const double (&t)[3]) {
    if (op.rank == 0) {
      mfipm_info info{};
      info.ipm_iters = its - 1;
      info.correctors = sh.correctors;
      info.pcg_iters = pcg_total;
      info.n_mat = nmat;
      info.rel_gap = sh.rel_gap;
      info.dual_res = sqrt(t[0]) / (1.0 + sh.cn);
      info.kkt_rel = sqrt(t[1]) / (1.0 + sqrt(t[2]));
      // converged: the gap test (reading R7) and a KKT residual of x within sqrt(tol); the
      // complementarity gap alone also shrinks on an iterate that has run away (|P| huge)
      info.status = sh.stop != -1 ? sh.stop : (info.kkt_rel <= sqrt(prm.tol) ? MFIPM_OK : MFIPM_NOT_CONVERGED);
      info.primal_obj = sh.P_obj;
      *pd.info = info;
      if (info.status != MFIPM_OK) atomicCAS(a.err, 0, info.status);
    }
  });
}

// Reverse mode (mfipm_backward; the paper has no derivative): differentiating the KKT
// conditions Q z + c - s = 0, Z S e = mu e of Eq. fzfs at fixed mu gives
// (Theta^-1 + F F^T) dz = -dc - dQ z, so for dL/dx = g and J = [I; -I]:
//   y = H^-1 J g (the PCG of the forward, same matrix and preconditioner),
//   w = J^T y,  dL/db = A w,  dL/dtau = -1^T y,  dL/dA = r w^T - (A w) x^T (r = b - A x).
template <int G, class Op, class PS>
__device__ void backward_one(const ProbDesc& pd, const KernelArgs& a, Op& op, RedSmem& rs,
                             IpmShared<PS, double>& sh, int& par) {
  using P2 = typename V2<PS>::T;
  const SolveParams& prm = a.prm;
  const int tid = threadIdx.x;
  const int64_t n = pd.n, chunk = op.chunk, gb = op.gbase;
  P2* __restrict__ Y = reinterpret_cast<P2*>(pd.pcg);
  P2* __restrict__ Rv = Y + 2 * n;
  P2* __restrict__ Pv = Rv + n;
  P2* __restrict__ Dv = Pv + n;
  PS* __restrict__ w = op.template wbuf<PS>();
  double* __restrict__ buf = op.template rbuf<double>();
  int64_t nmat = 0;
  op.template setup<G>(rs, par);
  const PS rho = (PS)op.rho;
  PS rz_part = 0, pdp_part = 0;
  for (int64_t q = tid; q < chunk; q += kThreads) {
    if (!op.valid(q)) { w[q] = (PS)0; continue; }
    const int64_t gi = gb + q, ni = op.natural(q);
    const double u = pd.zs_in[ni], v = pd.zs_in[n + ni], su = pd.zs_in[2 * n + ni], sv = pd.zs_in[3 * n + ni];
    P2 d, r;
    d.x = (PS)(su / u);
    d.y = (PS)(sv / v);
    r.x = (PS)pd.gx[ni];
    r.y = -r.x;
    const P2 p = precond<PS>(d, r, rho);
    Dv[gi] = d;
    Rv[gi] = r;
    Pv[gi] = p;
    w[q] = p.x - p.y;
    rz_part += r.x * p.x + r.y * p.y;
    pdp_part += d.x * p.x * p.x + d.y * p.y * p.y;
  }
  __syncthreads();
  // the derivative needs a tighter solve than a Newton direction
  const double tol = fmin(prm.tol_pcg, 1e-6);
  const int k = pcg_solve<G>(op, rs, sh, par, Y, Rv, Pv, Dv, w, rho, tol, prm.max_iter_pcg, rz_part, pdp_part, nmat);
  double tsum = 0.0;
  for (int64_t q = tid; q < chunk; q += kThreads) {
    if (!op.valid(q)) { buf[q] = 0.0; continue; }
    const P2 y = Y[gb + q];
    buf[q] = (double)y.x - (double)y.y;
    tsum += (double)y.x + (double)y.y;
  }
  __syncthreads();
  op.apply_A_out(pd);
  ++nmat;
  if (pd.grad_A) op.grad_A_out(pd, Y);
  double v[1] = {tsum};
  cluster_reduce<G, 1>(rs, par, v, [&](const double (&t)[1]) {
    if (op.rank == 0) {
      *pd.grad_tau = -t[0];
      mfipm_info info{};
      info.status = MFIPM_OK;
      info.pcg_iters = k;
      info.n_mat = nmat;
      *pd.info = info;
    }
  });
}

template <int G, class Op, class PS>
__global__ void __launch_bounds__(kThreads, 1) bwd_kernel(KernelArgs a) {
  extern __shared__ __align__(256) unsigned char smem[];
  __shared__ RedSmem rs;
  __shared__ IpmShared<PS, double> sh;
  int par = 0;
  int rank = 0;
  if constexpr (G > 1) rank = (int)cg::this_cluster().block_rank();
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) rs.fetched = atomicAdd(a.queue, 1);
    cluster_barrier<G>();
    int pid;
    if constexpr (G == 1) {
      pid = rs.fetched;
    } else {
      pid = cg::this_cluster().map_shared_rank(&rs, 0)->fetched;
    }
    if (pid >= a.batch) break;
    const ProbDesc pd = a.probs[pid];
    Op op;
    op.init(pd, a, smem, rank);
    backward_one<G, Op, PS>(pd, a, op, rs, sh, par);
    cluster_barrier<G>();
  }
  cluster_barrier<G>();
}

template <int G, class Op, class PS>
inline cudaError_t launch_bwd_t(const KernelArgs& a, size_t smem, int grid_clusters, cudaStream_t st) {
  auto kern = bwd_kernel<G, Op, PS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (G > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_clusters * G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int G, class Op, class PS>
inline int occupancy_bwd_t(size_t smem) {
  auto kern = bwd_kernel<G, Op, PS>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (G > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Persistent solver kernel.  Phase 1: whole clusters take problems [0, nbig) from queue[0]
// (the problems whose vectors need the shared memory of G CTAs).  Phase 2: every CTA on its
// own takes problems [nbig, batch) from queue[1] and solves them with no cross-CTA traffic
// (one problem per CTA uses the SMs more efficiently than a cluster per problem).  There is
// no grid-wide barrier between the phases: a cluster that runs out of large problems
// starts on small ones while others finish theirs.
template <int G, class Op, class Op1, class PS, class S>
__global__ void __launch_bounds__(kThreads, 1) ipm_kernel(KernelArgs a) {
  extern __shared__ __align__(256) unsigned char smem[];
  __shared__ RedSmem rs;
  __shared__ IpmShared<PS, typename S::T> sh;
  int par = 0;
  int rank = 0;
  if constexpr (G > 1) rank = (int)cg::this_cluster().block_rank();
  for (; !a.phase2_only;) {
    if (rank == 0 && threadIdx.x == 0) rs.fetched = atomicAdd(a.queue, 1);
    cluster_barrier<G>();
    int pid;
    if constexpr (G == 1) {
      pid = rs.fetched;
    } else {
      pid = cg::this_cluster().map_shared_rank(&rs, 0)->fetched;
    }
    if (pid >= a.nbig) break;
    const ProbDesc pd = a.probs[pid];
    Op op;
    op.init(pd, a, smem, rank);
    solve_one<G, Op, PS, S>(pd, a, op, rs, sh, par);
    cluster_barrier<G>();
  }
  cluster_barrier<G>();  // every CTA has read rank 0's last fetch before it is reused
  for (;;) {
    if (threadIdx.x == 0) rs.fetched = a.nbig + atomicAdd(a.queue + 1, 1);
    __syncthreads();
    const int pid = rs.fetched;
    if (pid >= a.batch) break;
    const ProbDesc pd = a.probs[pid];
    Op1 op;
    op.init(pd, a, smem, 0);
    solve_one<1, Op1, PS, S>(pd, a, op, rs, sh, par);
    __syncthreads();
  }
  cluster_barrier<G>();  // no CTA leaves while another may still read its shared memory
}

template <int G, class Op, class Op1, class PS, class S>
inline cudaError_t launch_t(const KernelArgs& a, size_t smem, int grid_clusters, cudaStream_t st) {
  auto kern = ipm_kernel<G, Op, Op1, PS, S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (G > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_clusters * G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int G, class Op, class Op1, class PS, class S>
inline int occupancy_t(size_t smem) {
  auto kern = ipm_kernel<G, Op, Op1, PS, S>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (G > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}


#define MFIPM_G_SWITCH(G, CALL) \
  switch (G) {                  \
    case 1: return CALL(1);     \
    case 2: return CALL(2);     \
    case 4: return CALL(4);     \
    case 8: return CALL(8);     \
    case 16: return CALL(16);   \
    default: break;             \
  }

}  // namespace mfipm
