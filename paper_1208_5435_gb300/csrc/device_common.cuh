// Device building blocks of the mfIPM kernels: complex arithmetic, CTA/cluster
// reductions through distributed shared memory, and the shared-memory radix-4 FFT
// used by the partial-DCT operator.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cg = cooperative_groups;

namespace mfipm {

constexpr int kThreads = 512;          // threads per CTA of every solver kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRed = 8;             // values per fused cluster reduction

// ------------------------------------------------------------------ double-float
// A double-float value is the unevaluated sum hi + lo of two float32 numbers with
// |lo| <= ulp(hi)/2: about 48 significant bits on the float32 pipes.  Built from the
// error-free transformations TwoSum (Knuth) and Fast2Sum (Dekker) and the FMA-based exact
// product; addition is the cheap "sloppy" double-double addition of Hida, Li and Bailey,
// whose absolute error is bounded by about 2^-46 (|a| + |b|) -- what an FFT needs.
// The _rn intrinsics keep the compiler from contracting or reordering these steps.
struct df {
  float hi, lo;
  __host__ __device__ constexpr df() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr df(float h, float l = 0.f) : hi(h), lo(l) {}
};
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {  // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
  const df s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df to_df(double x) {
  const float h = __double2float_rn(x);
  return df(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double to_double(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }
__device__ __forceinline__ double to_double(double a) { return a; }

struct dfc {
  df x, y;
};

__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ df shfl_xor(df v, int m) {
  return df(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ dfc mk(df a, df b) { return dfc{a, b}; }
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <class C> __device__ __forceinline__ C cmul_i(C a) { return mk(-a.y, a.x); }     // i*a
template <class C> __device__ __forceinline__ C cmul_mi(C a) { return mk(a.y, -a.x); }    // -i*a
template <class C, class R> __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }

// Twiddle tables, level-ordered: tw[2^l + j] = exp(-2 pi i j / 2^l) for 0 <= j < 2^l and
// 1 <= l <= log2_tw (built once per call by a setup kernel with sincospi).  Roots of one
// order sit contiguously, so the lanes of a warp that need consecutive j read consecutive
// entries (one cache line serves 8-16 lanes).
template <class C> struct Twiddle {
  const C* tw;
  int log2_tw;
  // exp(-2 pi i j / 2^logB) for 0 <= j < 2^logB
  __device__ __forceinline__ C root(int64_t j, int logB) const { return __ldg(&tw[((int64_t)1 << logB) + j]); }
};
template <> struct Twiddle<dfc> {
  const float4* tw;  // {re.hi, re.lo, im.hi, im.lo}
  int log2_tw;
  __device__ __forceinline__ dfc root(int64_t j, int logB) const {
    const float4 t = __ldg(&tw[((int64_t)1 << logB) + j]);
    return dfc{df(t.x, t.y), df(t.z, t.w)};
  }
};

// ------------------------------------------------------------------ reductions
template <class V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Shared state of the cluster reductions (lives in static shared memory).
struct RedSmem {
  double warp_part[kWarps][kMaxRed];
  double cta_part[2][kMaxRed];  // double-buffered: read remotely by the other CTAs
  double sd[8];                 // scalars derived by thread 0 from the last reduction
  float sf[8];
  int flag;
  int fetched;                  // problem index broadcast by CTA rank 0
};

// Reduce K per-thread values over the cluster of G CTAs (sum, or min when kMin).  Thread 0
// of every CTA receives identical totals (the G partials are combined in rank order) and
// runs fin(totals), which stores derived scalars in rs.sd / rs.sf / rs.flag; the function
// ends with a CTA barrier, after which every thread may read them.  `parity` alternates so
// that a CTA can publish new partials while a slower CTA still reads the previous ones;
// between two uses of one buffer lies the cluster barrier of the call in between.
template <int G, int K, bool kMin = false, class V, class Fin>
__device__ __forceinline__ void cluster_reduce(RedSmem& rs, int& parity, const V (&v)[K], Fin&& fin) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    V w = v[k];
    if constexpr (kMin) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w = fmin(w, __shfl_xor_sync(0xffffffffu, w, o));
    } else {
      w = warp_sum(w);
    }
    if (lane == 0) rs.warp_part[warp][k] = (double)w;
  }
  __syncthreads();
  double mine[K];
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < kWarps ? rs.warp_part[lane][k] : (kMin ? INFINITY : 0.0);
      if constexpr (kMin) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
      } else {
        t = warp_sum(t);
      }
      mine[k] = t;
      if (G > 1 && lane == 0) rs.cta_part[parity][k] = t;
    }
  }
  if constexpr (G > 1) cg::this_cluster().sync();
  if (threadIdx.x == 0) {
    double tot[K];
    if constexpr (G == 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] = mine[k];
    } else {
      cg::cluster_group cl = cg::this_cluster();
#pragma unroll
      for (int k = 0; k < K; ++k) tot[k] = kMin ? INFINITY : 0.0;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const RedSmem* r = cl.map_shared_rank(&rs, g);
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = kMin ? fmin(tot[k], r->cta_part[parity][k]) : tot[k] + r->cta_part[parity][k];
      }
    }
    fin(tot);
  }
  __syncthreads();
  parity ^= 1;
}

template <int G> __device__ __forceinline__ void cluster_barrier() {
  if constexpr (G == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

// ------------------------------------------------------------------ shared-memory FFT
// Shared-memory slot of complex element p of an M = 2^logM point buffer: the low four bits
// of p are XORed with four higher bits (bits max(logM - 4, 4) and up).  An involution that
// keeps every aligned run of 16 consecutive p on 16 distinct slots of one 16-slot group (the
// FFT stages and the per-index passes stay conflict-free), and spreads the bit-reversed
// column accesses of the DCT exchange step over distinct banks: consecutive columns k2 sit
// at positions bitrev(k2) that differ only in their top bits, which without the XOR all
// fall into one bank.
__device__ __forceinline__ int swz(int p, int logM) {
  const int sh = logM > 8 ? logM - 4 : 4;
  return p ^ ((p >> sh) & 15);
}

// Radix-4 butterflies of the two transforms, in registers: the forward (DIF) one takes a0..a3
// at stride S of a block and twiddles w, w^2, w^3 of the block's order; the inverse (DIT) one
// undoes it with the conjugate twiddles.
template <class C>
__device__ __forceinline__ void bfly4_dif(C& a0, C& a1, C& a2, C& a3, C w1, C w2, C w3) {
  const C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  a0 = cadd(s02, s13);
  a1 = cmul(csub(s02, s13), w2);
  a2 = cmul(cadd(d02, cmul_mi(d13)), w1);
  a3 = cmul(cadd(d02, cmul_i(d13)), w3);
}
template <class C>
__device__ __forceinline__ void bfly4_dit(C& a0, C& a1, C& a2, C& a3, C w1, C w2, C w3) {
  const C b1 = cmulc(a1, w2), b2 = cmulc(a2, w1), b3 = cmulc(a3, w3);
  const C Ss = cadd(a0, b1), D = csub(a0, b1), E = cadd(b2, b3), F = csub(b3, b2);
  a0 = cadd(Ss, E);
  a1 = cadd(D, cmul_mi(F));
  a2 = csub(Ss, E);
  a3 = cadd(D, cmul_i(F));
}

// Two consecutive radix-4 stages of the forward transform (blocks of 2^logB, then of
// 2^(logB-2)) in one pass over shared memory: each group of 16 points (stride 2^(logB-4) in
// one block) is loaded once, both stages run in registers, and it is stored once -- half the
// barriers and shared-memory traffic of two single stages, and 16 independent loads per
// thread to cover their latency.
template <class C>
__device__ __forceinline__ void fft_dif_pass16(C* buf, int logM, int logB, const Twiddle<C>& tw) {
  const int logS2 = logB - 4, S2 = 1 << logS2, S1 = S2 << 2;
  for (int g = threadIdx.x; g < (1 << (logM - 4)); g += kThreads) {
    const int blk = g >> logS2, t2 = g & (S2 - 1);
    const int base = (blk << logB) + t2;
    C x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = buf[swz(base + j * S2, logM)];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = t2 + i * S2;
      bfly4_dif(x[i], x[i + 4], x[i + 8], x[i + 12], tw.root(t, logB), tw.root(2 * t, logB), tw.root(3 * t, logB));
    }
    const C v1 = tw.root(t2, logB - 2), v2 = tw.root(2 * t2, logB - 2), v3 = tw.root(3 * t2, logB - 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) bfly4_dif(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3], v1, v2, v3);
#pragma unroll
    for (int j = 0; j < 16; ++j) buf[swz(base + j * S2, logM)] = x[j];
    (void)S1;
  }
}
// The inverse of two consecutive forward stages: blocks of 2^(logB-2), then of 2^logB.
template <class C>
__device__ __forceinline__ void fft_dit_pass16(C* buf, int logM, int logB, const Twiddle<C>& tw) {
  const int logS2 = logB - 4, S2 = 1 << logS2;
  for (int g = threadIdx.x; g < (1 << (logM - 4)); g += kThreads) {
    const int blk = g >> logS2, t2 = g & (S2 - 1);
    const int base = (blk << logB) + t2;
    C x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = buf[swz(base + j * S2, logM)];
    const C v1 = tw.root(t2, logB - 2), v2 = tw.root(2 * t2, logB - 2), v3 = tw.root(3 * t2, logB - 2);
#pragma unroll
    for (int q = 0; q < 4; ++q) bfly4_dit(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3], v1, v2, v3);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = t2 + i * S2;
      bfly4_dit(x[i], x[i + 4], x[i + 8], x[i + 12], tw.root(t, logB), tw.root(2 * t, logB), tw.root(3 * t, logB));
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) buf[swz(base + j * S2, logM)] = x[j];
  }
}
// The fused passes are used for 8-byte complex values (float32 chains) when every thread has a
// group of 16 points; 16-byte values (double-float, float64) keep single stages (register room).
template <class C> __device__ __forceinline__ bool use_pass16(int logM) {
  return sizeof(C) == 8 && (1 << (logM - 4)) >= kThreads;
}

// In-place radix-4 decimation-in-frequency FFT of M = 2^logM points held in shared
// memory (element p in slot swz(p)): natural-order input, bit-reversed output, forward sign
// exp(-2 pi i jk/M).  Each radix-4 group is two radix-2 stages, so the output order is
// plain bit reversal.
template <class C, class R>
__device__ void fft_dif(C* buf, int logM, const Twiddle<C>& tw) {
  const int M = 1 << logM;
  int logB = logM;
  if (use_pass16<C>(logM)) {
    for (; logB >= 4; logB -= 4) {
      fft_dif_pass16(buf, logM, logB, tw);
      __syncthreads();
    }
  }
  for (; logB >= 2; logB -= 2) {
    const int logS = logB - 2, S = 1 << logS;
    for (int gi = threadIdx.x; gi < (M >> 2); gi += kThreads) {
      const int blk = gi >> logS, t = gi & (S - 1);
      const int p = (blk << logB) + t;
      const int q0 = swz(p, logM), q1 = swz(p + S, logM), q2 = swz(p + 2 * S, logM), q3 = swz(p + 3 * S, logM);
      C a0 = buf[q0], a1 = buf[q1], a2 = buf[q2], a3 = buf[q3];
      C w1 = tw.root(t, logB), w2 = tw.root(2 * t, logB), w3 = tw.root(3 * t, logB);
      C s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
      buf[q0] = cadd(s02, s13);
      buf[q1] = cmul(csub(s02, s13), w2);
      buf[q2] = cmul(cadd(d02, cmul_mi(d13)), w1);
      buf[q3] = cmul(cadd(d02, cmul_i(d13)), w3);
    }
    __syncthreads();
  }
  if (logB == 1) {
    for (int gi = threadIdx.x; gi < (M >> 1); gi += kThreads) {
      const int q0 = swz(2 * gi, logM), q1 = swz(2 * gi + 1, logM);
      C a0 = buf[q0], a1 = buf[q1];
      buf[q0] = cadd(a0, a1);
      buf[q1] = csub(a0, a1);
    }
    __syncthreads();
  }
}

// Unnormalised inverse of fft_dif: bit-reversed input, natural output, sign +,
// result = M * IDFT (same slot layout).
template <class C, class R>
__device__ void fft_dit_inv(C* buf, int logM, const Twiddle<C>& tw) {
  const int M = 1 << logM;
  int logB = 2;
  if (logM & 1) {
    for (int gi = threadIdx.x; gi < (M >> 1); gi += kThreads) {
      const int q0 = swz(2 * gi, logM), q1 = swz(2 * gi + 1, logM);
      C a0 = buf[q0], a1 = buf[q1];
      buf[q0] = cadd(a0, a1);
      buf[q1] = csub(a0, a1);
    }
    __syncthreads();
    logB = 3;
  }
  // the forward transform fused its first stages in pairs from the top: the single stages
  // it ran last (the small blocks) are undone first, then the fused pairs
  if (use_pass16<C>(logM)) {
    const int fused = (logM - (logM & 1)) / 4;  // pairs the forward transform fused
    const int single_top = logM - 4 * fused;    // largest block size of its single stages
    for (; logB <= single_top; logB += 2) {
      const int logS = logB - 2, S = 1 << logS;
      for (int gi = threadIdx.x; gi < (M >> 2); gi += kThreads) {
        const int blk = gi >> logS, t = gi & (S - 1);
        const int p = (blk << logB) + t;
        const int q0 = swz(p, logM), q1 = swz(p + S, logM), q2 = swz(p + 2 * S, logM), q3 = swz(p + 3 * S, logM);
        C a0 = buf[q0], a1 = buf[q1], a2 = buf[q2], a3 = buf[q3];
        bfly4_dit(a0, a1, a2, a3, tw.root(t, logB), tw.root(2 * t, logB), tw.root(3 * t, logB));
        buf[q0] = a0;
        buf[q1] = a1;
        buf[q2] = a2;
        buf[q3] = a3;
      }
      __syncthreads();
    }
    for (logB = single_top + 4; logB <= logM; logB += 4) {
      fft_dit_pass16(buf, logM, logB, tw);
      __syncthreads();
    }
    return;
  }
  for (; logB <= logM; logB += 2) {
    const int logS = logB - 2, S = 1 << logS;
    for (int gi = threadIdx.x; gi < (M >> 2); gi += kThreads) {
      const int blk = gi >> logS, t = gi & (S - 1);
      const int p = (blk << logB) + t;
      const int q0 = swz(p, logM), q1 = swz(p + S, logM), q2 = swz(p + 2 * S, logM), q3 = swz(p + 3 * S, logM);
      C o0 = buf[q0];
      C b1 = cmulc(buf[q1], tw.root(2 * t, logB));
      C b2 = cmulc(buf[q2], tw.root(t, logB));
      C b3 = cmulc(buf[q3], tw.root(3 * t, logB));
      C Ss = cadd(o0, b1), D = csub(o0, b1), E = cadd(b2, b3), F = csub(b3, b2);
      buf[q0] = cadd(Ss, E);
      buf[q1] = cadd(D, cmul_mi(F));
      buf[q2] = csub(Ss, E);
      buf[q3] = cadd(D, cmul_i(F));
    }
    __syncthreads();
  }
}

// G-point DFT of a register array (G a compile-time power of two), natural order in and
// out.  inverse=true uses the + sign and does not normalise.
template <int G, class C>
__device__ __forceinline__ void small_dft(C (&a)[G], bool inverse, const Twiddle<C>& tw) {
  if constexpr (G == 1) {
    return;
  } else {
    constexpr int logG = (G == 2) ? 1 : (G == 4) ? 2 : (G == 8) ? 3 : 4;
    // bit-reversal permutation (compile-time indices)
#pragma unroll
    for (int i = 0; i < G; ++i) {
      int r = 0;
#pragma unroll
      for (int bbit = 0; bbit < logG; ++bbit) r |= ((i >> bbit) & 1) << (logG - 1 - bbit);
      if (r > i) { C t = a[i]; a[i] = a[r]; a[r] = t; }
    }
#pragma unroll
    for (int ls = 0; ls < logG; ++ls) {
      const int s = 1 << ls;
#pragma unroll
      for (int j = 0; j < G; j += 2 * s) {
#pragma unroll
        for (int t = 0; t < s; ++t) {
          C w = tw.root(t, ls + 1);
          if (inverse) w = cconj(w);
          C u = a[j + t], v = cmul(a[j + t + s], w);
          a[j + t] = cadd(u, v);
          a[j + t + s] = csub(u, v);
        }
      }
    }
  }
}

__device__ __forceinline__ int bitrev(int x, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)x) >> (32 - bits));
}

}  // namespace mfipm
