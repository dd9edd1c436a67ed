// Partial DCT of any even length n whose half L = n/2 has no prime factor above 5 (the
// n = 1000 of the phase-transition experiment, Sec. 5.8; the 200 x 1000 DCT problem of the
// test set, Table 3).  The chain is the power-of-two operator's (Makhoul's even/odd
// reordering, the length-L complex FFT of the packed pairs, the real-DCT untangling, the row
// mask, and the exact inverse of all of it; Sec. 2, A = R C with orthonormal rows), with the
// FFT done as an in-place mixed-radix transform (radices 4, 2, 3, 5) in one CTA's shared
// memory.  One CTA per problem (n <= 16384: 24 bytes of shared memory per complex point, as
// for the power-of-two chain); the IPM around it is the persistent kernel's solve_one.
#include "dct_gen.h"
#include "solver_impl.cuh"

namespace mfipm {

// Radices of L, first stage first: n4 fours, then n2 (0 or 1) twos, n3 threes and n5 fives
// (the host admits only lengths whose half has no other prime factor).
struct GenPlan {
  int L, n4, n2, n3, n5;
};
__device__ __forceinline__ GenPlan gen_plan(int L) {
  GenPlan p{L, 0, 0, 0, 0};
  int r = L;
  while (r % 4 == 0) { ++p.n4; r /= 4; }
  if (r % 2 == 0) { p.n2 = 1; r /= 2; }
  while (r % 3 == 0) { ++p.n3; r /= 3; }
  while (r % 5 == 0) { ++p.n5; r /= 5; }
  return p;
}

// Roots of one length: three runs of L entries, exp(-2 pi i e / L), exp(-2 pi i k / n) and
// exp(-i pi k / (2 n)) (the FFT's twiddles, and w_N^k and eps^k of the untangling), and the
// shared-memory position of every frequency after the forward transform (digit reversal).
template <class C> struct GenTw {
  const C* t;
  const int* pos;
  int L;
  __device__ __forceinline__ C at(int i) const { return __ldg(t + i); }
  __device__ __forceinline__ C root(int e) const { return at(e); }
  __device__ __forceinline__ C wN(int k) const { return at(L + k); }
  __device__ __forceinline__ C eps(int k) const { return at(2 * L + k); }
};
template <> struct GenTw<dfc> {
  const float4* t;  // {re.hi, re.lo, im.hi, im.lo}
  const int* pos;
  int L;
  __device__ __forceinline__ dfc at(int i) const {
    const float4 v = __ldg(t + i);
    return dfc{df(v.x, v.y), df(v.z, v.w)};
  }
  __device__ __forceinline__ dfc root(int e) const { return at(e); }
  __device__ __forceinline__ dfc wN(int k) const { return at(L + k); }
  __device__ __forceinline__ dfc eps(int k) const { return at(2 * L + k); }
};

// R-point DFT in registers, natural order in and out; inv: + sign, no normalisation.  w1, w2 =
// exp(-2 pi i / R), exp(-4 pi i / R) (R = 3, 5): the real parts cos and the imaginary parts
// -sin of the two roots the closed forms need.
template <int R, class C>
__device__ __forceinline__ void gen_dft(C (&x)[R], bool inv, C w1, C w2) {
  if constexpr (R == 2) {
    const C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const C s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]), s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
    const C j13 = inv ? cmul_i(d13) : cmul_mi(d13);  // (-+ i)(x1 - x3)
    x[0] = cadd(s02, s13);
    x[2] = csub(s02, s13);
    x[1] = cadd(d02, j13);
    x[3] = csub(d02, j13);
  } else if constexpr (R == 3) {
    // y1,2 = x0 + cos(2pi/3) t -+ i sin(2pi/3) (x1 - x2), t = x1 + x2
    const C t = cadd(x[1], x[2]);
    const C b = cadd(x[0], cscale(t, w1.x));
    const C d = cscale(csub(x[1], x[2]), w1.y);  // -sin(2 pi / 3) (x1 - x2)
    const C jd = inv ? cmul_mi(d) : cmul_i(d);
    x[0] = cadd(x[0], t);
    x[1] = cadd(b, jd);
    x[2] = csub(b, jd);
  } else {
    static_assert(R == 5, "radices 2, 3, 4, 5");
    // with c1, c2 = cos(2pi/5), cos(4pi/5) and s1, s2 = sin(2pi/5), sin(4pi/5):
    // y1,4 = x0 + c1 t1 + c2 t2 -+ i (s1 t3 + s2 t4), y2,3 = x0 + c2 t1 + c1 t2 -+ i (s2 t3 - s1 t4)
    const C t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]), t3 = csub(x[1], x[4]), t4 = csub(x[2], x[3]);
    const C b1 = cadd(x[0], cadd(cscale(t1, w1.x), cscale(t2, w2.x)));
    const C b2 = cadd(x[0], cadd(cscale(t1, w2.x), cscale(t2, w1.x)));
    // w1.y = -s1, w2.y = -s2
    const C d1 = cadd(cscale(t3, w1.y), cscale(t4, w2.y));  // -(s1 t3 + s2 t4)
    const C d2 = csub(cscale(t3, w2.y), cscale(t4, w1.y));  // -(s2 t3 - s1 t4)
    const C j1 = inv ? cmul_mi(d1) : cmul_i(d1);
    const C j2 = inv ? cmul_mi(d2) : cmul_i(d2);
    x[0] = cadd(x[0], cadd(t1, t2));
    x[1] = cadd(b1, j1);
    x[4] = csub(b1, j1);
    x[2] = cadd(b2, j2);
    x[3] = csub(b2, j2);
  }
}

// One decimation-in-frequency stage on blocks of Ls points (m = Ls / R): the R points
// j + t m of a block go through an R-point DFT, output q is multiplied by exp(-2 pi i j q / Ls)
// and stored back at j + q m.  INV undoes it exactly (conjugate twiddles first, then the
// inverse DFT), up to the factor R.
template <int R, bool INV, class C>
__device__ void gen_stage(C* buf, int Ls, const GenTw<C>& tw) {
  const int L = tw.L, m = Ls / R, step = L / Ls, nb = L / R;
  C w1 = tw.root(0), w2 = w1;
  if constexpr (R == 3 || R == 5) {
    w1 = tw.root(L / R);
    w2 = tw.root(2 * (L / R));
  }
  for (int u = threadIdx.x; u < nb; u += kThreads) {
    const int blk = u / m, j = u - blk * m;
    C* p = buf + blk * Ls + j;
    C x[R];
#pragma unroll
    for (int t = 0; t < R; ++t) x[t] = p[t * m];
    if constexpr (!INV) {
      gen_dft<R>(x, false, w1, w2);
      if (j != 0) {
#pragma unroll
        for (int t = 1; t < R; ++t) x[t] = cmul(x[t], tw.root(j * t * step));
      }
    } else {
      if (j != 0) {
#pragma unroll
        for (int t = 1; t < R; ++t) x[t] = cmulc(x[t], tw.root(j * t * step));
      }
      gen_dft<R>(x, true, w1, w2);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) p[t * m] = x[t];
  }
}

// Forward transform (natural order in, digit-reversed out, sign -) or its unnormalised
// inverse (digit-reversed in, natural out; L times the inverse DFT): the forward stages on
// blocks of L, L / r_0, ..., r_(S-1); the inverse undoes them from the last.
template <bool INV, class C>
__device__ void gen_fft(C* buf, const GenPlan& pl, const GenTw<C>& tw) {
  if constexpr (!INV) {
    int Ls = pl.L;
    for (int i = 0; i < pl.n4; ++i, Ls /= 4) { gen_stage<4, false>(buf, Ls, tw); __syncthreads(); }
    if (pl.n2) { gen_stage<2, false>(buf, Ls, tw); Ls /= 2; __syncthreads(); }
    for (int i = 0; i < pl.n3; ++i, Ls /= 3) { gen_stage<3, false>(buf, Ls, tw); __syncthreads(); }
    for (int i = 0; i < pl.n5; ++i, Ls /= 5) { gen_stage<5, false>(buf, Ls, tw); __syncthreads(); }
  } else {
    int Ls = 5;
    for (int i = 0; i < pl.n5; ++i, Ls *= 5) { gen_stage<5, true>(buf, Ls, tw); __syncthreads(); }
    Ls = Ls / 5 * 3;
    for (int i = 0; i < pl.n3; ++i, Ls *= 3) { gen_stage<3, true>(buf, Ls, tw); __syncthreads(); }
    Ls = Ls / 3 * 2;
    if (pl.n2) { gen_stage<2, true>(buf, Ls, tw); Ls *= 2; __syncthreads(); }
    Ls = Ls / 2 * 4;
    for (int i = 0; i < pl.n4; ++i, Ls *= 4) { gen_stage<4, true>(buf, Ls, tw); __syncthreads(); }
  }
}

// The untangling, mask and inverse for every frequency: thread k takes k and its partner
// L - k (0 and, for even L, L/2 pair with themselves).  Returns this CTA's share of the masked
// coefficient energy.  MODE_FORWARD writes the orthonormal DCT-II coefficients to fwd
// instead (every one of the n exactly once) and leaves buf as it is.
template <class C, int MODE>
__device__ double gen_pointwise(C* buf, const DctGeom& geo, const GenPlan& pl, const GenTw<C>& tw, double inv_n,
                                double* fwd) {
  using R = decltype(C().x);
  const PwConst<R> pc(inv_n);
  R acc = pc.zero;
  const int L = pl.L;
  for (int k = threadIdx.x; k <= L / 2; k += kThreads) {
    const int kb = k == 0 ? 0 : L - k;
    const int pa = __ldg(tw.pos + k), pb = __ldg(tw.pos + kb);
    const unsigned ma = __ldg(geo.mcode + k), mb = __ldg(geo.mcode + kb);
    const C wa = tw.wN(k), ea = tw.eps(k), wb = tw.wN(kb), eb = tw.eps(kb);
    const C a = buf[pa], b = buf[pb];
    const C na = dct_pointwise_w<C, MODE, R>(k, a, b, wa, ea, ma, geo, pc, true, acc, fwd);
    if (kb != k) {
      const C nb = dct_pointwise_w<C, MODE, R>(kb, b, a, wb, eb, mb, geo, pc, true, acc, fwd);
      if constexpr (MODE != MODE_FORWARD) buf[pb] = nb;
    }
    if constexpr (MODE != MODE_FORWARD) buf[pa] = na;
  }
  return to_double(acc);
}

template <class C, int MODE>
__device__ double gen_chain(C* buf, const DctGeom& geo, const GenPlan& pl, const GenTw<C>& tw, double inv_n,
                            double* fwd = nullptr) {
  __syncthreads();
  gen_fft<false>(buf, pl, tw);
  const double acc = gen_pointwise<C, MODE>(buf, geo, pl, tw, inv_n, fwd);
  __syncthreads();
  if constexpr (MODE != MODE_FORWARD) gen_fft<true>(buf, pl, tw);
  return acc;
}

// Storage order: position q of the n-vectors holds v_q of Makhoul's reordering
// (v_j = x_2j, v_(n-1-j) = x_(2j+1)), and the complex point j of the FFT is (v_2j, v_(2j+1)).
struct DctGenOp {
  DctGeom geo;
  GenPlan pl;
  double2* buf64;
  float2* buf32;
  GenTw<double2> tw64;
  GenTw<float2> tw32;
  GenTw<dfc> twdf;
  int64_t chunk, gbase;
  double rho, inv_n;
  int rank;

  __device__ void init(const ProbDesc& pd, const KernelArgs& a, unsigned char* smem, int) {
    rank = 0;
    geo = DctGeom{};
    geo.N = pd.n;
    geo.mask = pd.mask;
    geo.bsu = pd.bsu;
    geo.bsu_df = pd.bsu_df;
    geo.mcode = pd.mcode;
    geo.bpk = pd.bpk;
    geo.bpk_f64 = a.prm.resid_fp64 != 0;
    const int L = (int)(pd.n >> 1);
    pl = gen_plan(L);
    buf64 = reinterpret_cast<double2*>(smem);
    buf32 = reinterpret_cast<float2*>(smem + (size_t)16 * L);
    const char* t = static_cast<const char*>(pd.twg);
    const int* pos = reinterpret_cast<const int*>(t + gen_tw_offpos(L));
    tw64 = GenTw<double2>{reinterpret_cast<const double2*>(t), pos, L};
    tw32 = GenTw<float2>{reinterpret_cast<const float2*>(t + gen_tw_off32(L)), pos, L};
    twdf = GenTw<dfc>{reinterpret_cast<const float4*>(t + gen_tw_offdf(L)), pos, L};
    chunk = pd.n;
    gbase = 0;
    rho = (double)pd.m / (double)pd.n;  // A A^T = I: rho = m/n (Eq. eq:ne2_P)
    inv_n = 1.0 / (double)pd.n;
  }
  __device__ __forceinline__ bool valid(int64_t) const { return true; }
  template <class T> __device__ __forceinline__ T* rbuf() const { return reinterpret_cast<T*>(buf64); }
  template <class PS> __device__ __forceinline__ PS* wbuf() const {
    if constexpr (sizeof(PS) == 8) {
      return reinterpret_cast<PS*>(buf64);
    } else {
      return reinterpret_cast<PS*>(buf32);
    }
  }
  template <class T> __device__ double resid_t() {
    if constexpr (std::is_same<T, df>::value) {
      return gen_chain<dfc, MODE_RESID>(reinterpret_cast<dfc*>(buf64), geo, pl, twdf, inv_n);
    } else {
      return gen_chain<double2, MODE_RESID>(buf64, geo, pl, tw64, inv_n);
    }
  }
  template <class PS> __device__ double normal(PS*) {
    if constexpr (sizeof(PS) == 8) {
      return gen_chain<double2, MODE_NORMAL>(buf64, geo, pl, tw64, inv_n);
    } else {
      return gen_chain<float2, MODE_NORMAL>(buf32, geo, pl, tw32, inv_n);
    }
  }
  static constexpr bool kLowpResid = true;
  template <class T> __device__ double resid_lowp() {
    T* rb = rbuf<T>();
    float* wb = wbuf<float>();
    for (int64_t q = threadIdx.x; q < chunk; q += kThreads) wb[q] = to_float(rb[q]);
    const double acc = gen_chain<float2, MODE_RESID>(buf32, geo, pl, tw32, inv_n);
    for (int64_t q = threadIdx.x; q < chunk; q += kThreads) rb[q] = from_float<T>(wb[q]);
    __syncthreads();
    return acc;
  }
  // grad_b = A w for w in rbuf<double>() (float64 chain): all n DCT coefficients go to
  // pd.scratch, then the sampled rows are gathered.  Overwrites rbuf.
  __device__ void apply_A_out(const ProbDesc& pd) {
    gen_chain<double2, MODE_FORWARD>(buf64, geo, pl, tw64, inv_n, pd.scratch);
    __threadfence();
    __syncthreads();
    if (pd.grad_b)
      for (int64_t i = threadIdx.x; i < pd.m; i += kThreads) pd.grad_b[i] = pd.scratch[pd.rows[i]];
  }
  __device__ void grad_A_out(const ProbDesc&, const void*) {}
  __device__ int64_t natural(int64_t q) const { return q < geo.N / 2 ? 2 * q : 2 * geo.N - 1 - 2 * q; }
  template <int GG> __device__ void setup(RedSmem&, int&) {}
};

// ------------------------------------------------------------------ tables and launchers
__global__ void gen_twiddle_kernel(char* base, int L) {
  double2* t64 = reinterpret_cast<double2*>(base);
  float2* t32 = reinterpret_cast<float2*>(base + gen_tw_off32(L));
  float4* tdf = reinterpret_cast<float4*>(base + gen_tw_offdf(L));
  int* pos = reinterpret_cast<int*>(base + gen_tw_offpos(L));
  const GenPlan pl = gen_plan(L);
  const double N = 2.0 * (double)L;
  // digit reversal: k = k_0 + r_0 k_1 + r_0 r_1 k_2 + ... sits at k_0 L/r_0 + k_1 L/(r_0 r_1) + ...
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    int q = k, span = L, p = 0;
    auto digit = [&](int r) { span /= r; p += (q % r) * span; q /= r; };
    for (int i = 0; i < pl.n4; ++i) digit(4);
    if (pl.n2) digit(2);
    for (int i = 0; i < pl.n3; ++i) digit(3);
    for (int i = 0; i < pl.n5; ++i) digit(5);
    pos[k] = p;
  }
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 3 * L; e += gridDim.x * blockDim.x) {
    const int which = e / L, i = e - which * L;
    // exp(-i pi x): x = 2i/L, 2i/N, i/(2N)
    const double x = which == 0 ? 2.0 * (double)i / (double)L : which == 1 ? 2.0 * (double)i / N : (double)i / (2.0 * N);
    double s, c;
    sincospi(x, &s, &c);
    t64[e] = make_double2(c, -s);
    t32[e] = make_float2((float)c, (float)-s);
    const df re = to_df(c), im = to_df(-s);
    tdf[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

cudaError_t launch_gen_twiddles(void* base, int64_t n, cudaStream_t st) {
  const int L = (int)(n / 2);
  const int blocks = (3 * L + 255) / 256 < 256 ? (3 * L + 255) / 256 : 256;
  gen_twiddle_kernel<<<blocks, 256, 0, st>>>(static_cast<char*>(base), L);
  return cudaGetLastError();
}

size_t dct_gen_smem_bytes(int64_t max_n) { return (size_t)(max_n / 2) * 24; }

cudaError_t launch_dct_gen_solver(int variant, const KernelArgs& a, int64_t max_n, int ctas, cudaStream_t st) {
  const size_t smem = dct_gen_smem_bytes(max_n);
  switch (variant) {
    case kGenDF: return launch_t<1, DctGenOp, DctGenOp, float, StateDF>(a, smem, ctas, st);
    case kGenF64: return launch_t<1, DctGenOp, DctGenOp, float, StateF64>(a, smem, ctas, st);
    case kGenF64Pcg: return launch_t<1, DctGenOp, DctGenOp, double, StateF64>(a, smem, ctas, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bwd_dct_gen(const KernelArgs& a, int64_t max_n, int ctas, cudaStream_t st) {
  return launch_bwd_t<1, DctGenOp, float>(a, dct_gen_smem_bytes(max_n), ctas, st);
}
int max_active_ctas_bwd_dct_gen(int64_t max_n) { return occupancy_bwd_t<1, DctGenOp, float>(dct_gen_smem_bytes(max_n)); }

int max_active_ctas_dct_gen(int variant, int64_t max_n) {
  const size_t smem = dct_gen_smem_bytes(max_n);
  switch (variant) {
    case kGenDF: return occupancy_t<1, DctGenOp, DctGenOp, float, StateDF>(smem);
    case kGenF64: return occupancy_t<1, DctGenOp, DctGenOp, float, StateF64>(smem);
    case kGenF64Pcg: return occupancy_t<1, DctGenOp, DctGenOp, double, StateF64>(smem);
    default: return 0;
  }
}

}  // namespace mfipm
