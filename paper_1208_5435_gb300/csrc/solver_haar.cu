// Partial Haar operator for the persistent IPM kernel: A = m rows of the orthonormal n x n
// Haar matrix (Sec. 2 lists Haar wavelets among the orthonormal systems whose sampled rows
// give CS matrices with A A^T = I and O(n) products).  Coefficient 0 is the scaling
// coefficient; coefficient 2^j + k is the wavelet of scale j (0 coarsest) at position k.
//
//     A^T A w = H^T M H w,     A^T (A x - b) = H^T (M H x - b_u)
//
// with M the row mask and b_u the measurements placed at their rows (orthonormal rows, so
// rho = m/n as for the DCT).  The analysis H runs as a pyramid of pairwise sums and
// differences / sqrt(2): finest scales inside each thread, then across the threads of the
// CTA (warp-synchronous while the pairs stay in one warp), then across the G CTAs of the
// cluster by CTA 0 through distributed shared memory.  Each detail is masked (minus b_u)
// as it is produced; the synthesis H^T retraces the pyramid.
//
// Storage order inside a CTA's chunk of c = n/G values: slot i * Tc + t holds natural index
// gbase + t * V + i (Tc = min(c, threads), V = c / Tc), so the V values of thread t's block
// are its own and every level inside a thread touches consecutive shared-memory banks.
#include "solver_impl.cuh"

namespace mfipm {

__device__ __forceinline__ int ilog2_dev(int64_t v) { return 63 - __clzll((unsigned long long)v); }

template <int G> struct HaarOp {
  int64_t chunk, gbase;
  double rho;
  int rank, logN, Tc, logTc, logV;
  const uint8_t* mask;
  const double* bsu;
  const float2* bsu_df;
  unsigned char* rb;  // chunk values of the residual buffer (8 bytes each)
  double* fwd;        // MODE_FORWARD: the n coefficients (reverse mode's A w)
  float* wb;          // chunk float32 values of the PCG operator input

  __device__ void init(const ProbDesc& pd, const KernelArgs&, unsigned char* smem, int rank_) {
    rank = rank_;
    logN = pd.log2n;
    chunk = pd.n / G;
    gbase = (int64_t)rank_ * chunk;
    Tc = (int)(chunk < kThreads ? chunk : kThreads);
    logTc = ilog2_dev(Tc);
    logV = ilog2_dev(chunk) - logTc;
    mask = pd.mask;
    bsu = pd.bsu;
    bsu_df = pd.bsu_df;
    rb = smem;
    wb = reinterpret_cast<float*>(smem + 8 * chunk);
    rho = (double)pd.m / (double)pd.n;  // A A^T = I: rho = m/n (Eq. eq:ne2_P)
  }
  __device__ __forceinline__ bool valid(int64_t) const { return true; }
  __device__ __forceinline__ int64_t natural(int64_t q) const {
    const int64_t t = q & (Tc - 1), i = q >> logTc;
    return gbase + (t << logV) + i;
  }
  template <class T> __device__ __forceinline__ T* rbuf() const { return reinterpret_cast<T*>(rb); }
  // float32 PCG input in its own buffer; the float64 PCG shares the residual buffer (every PCG
  // initialisation reads the residual of an index before writing that index's input)
  template <class PS> __device__ __forceinline__ PS* wbuf() const {
    if constexpr (sizeof(PS) == 8) {
      return reinterpret_cast<PS*>(rb);
    } else {
      return reinterpret_cast<PS*>(wb);
    }
  }
  template <class T> __device__ double resid_t() { return chain<T, MODE_RESID>(rbuf<T>()); }
  static constexpr bool kLowpResid = false;
  template <class T> __device__ double resid_lowp() { return resid_t<T>(); }
  template <class PS> __device__ double normal(PS* w) { return chain<PS, MODE_NORMAL>(w); }
  // grad_b = A w for w in rbuf<double>(): the analysis pyramid in float64 writes all n Haar
  // coefficients to pd.scratch, then the sampled rows are gathered.  Overwrites rbuf.
  __device__ void apply_A_out(const ProbDesc& pd) {
    fwd = pd.scratch;
    chain<double, MODE_FORWARD>(rbuf<double>());
    __threadfence();
    cluster_barrier<G>();
    if (pd.grad_b)
      for (int64_t i = (int64_t)rank * kThreads + threadIdx.x; i < pd.m; i += (int64_t)G * kThreads)
        pd.grad_b[i] = pd.scratch[pd.rows[i]];
  }
  __device__ void grad_A_out(const ProbDesc&, const void*) {}
  template <int GG> __device__ void setup(RedSmem&, int&) {}

  __device__ __forceinline__ float load_b(int64_t i, float) const { return 0.f; }
  __device__ __forceinline__ double load_b(int64_t i, double) const { return bsu[i]; }
  __device__ __forceinline__ df load_b(int64_t i, df) const {
    const float2 v = bsu_df[i];
    return df(v.x, v.y);
  }
  // detail or scaling coefficient of index idx: masked (minus b_u), energy into acc
  template <class R, int MODE> __device__ __forceinline__ R coef(R d, int64_t idx, R& acc) const {
    if constexpr (MODE == MODE_FORWARD) {
      fwd[idx] = to_double(d);
      return d;
    }
    if (!mask[idx]) return R();
    if constexpr (MODE == MODE_RESID) d = d - load_b(idx, R());
    acc = acc + d * d;
    return d;
  }

  // buf := H^T M H buf (MODE_NORMAL) or H^T (M H buf - b_u) (MODE_RESID); returns this
  // thread's share of the masked coefficient energy (||A w||^2 or ||A x - b||^2)
  template <class R, int MODE> __device__ double chain(R* buf) {
    const int t = threadIdx.x;
    const int V = 1 << logV;
    const R r2 = rsqrt2<R>();
    R acc = R();
    const bool act = t < Tc;
    const int64_t base_t = gbase + ((int64_t)t << logV);  // natural index of thread t's block
    __syncthreads();
    // analysis inside the thread, finest scale first
    if (act) {
      for (int l = 0; l < logV; ++l) {
        const int s = 1 << l;
        const int64_t jbit = (int64_t)1 << (logN - 1 - l);
        for (int i = 0; i < V; i += 2 * s) {
          const R x0 = buf[i * Tc + t], x1 = buf[(i + s) * Tc + t];
          buf[i * Tc + t] = (x0 + x1) * r2;
          buf[(i + s) * Tc + t] = coef<R, MODE>((x0 - x1) * r2, jbit + ((base_t + i) >> (l + 1)), acc);
        }
      }
    }
    __syncwarp();
    // across the threads: thread t's block average sits in slot t
    for (int lam = 0; lam < logTc; ++lam) {
      const int s = 1 << lam;
      if (act && (t & (2 * s - 1)) == 0) {
        const int lev = logV + lam;
        const R x0 = buf[t], x1 = buf[t + s];
        buf[t] = (x0 + x1) * r2;
        buf[t + s] = coef<R, MODE>((x0 - x1) * r2, ((int64_t)1 << (logN - 1 - lev)) + (base_t >> (lev + 1)), acc);
      }
      // the next level pairs t and t + 2s (t a multiple of 4s): one warp while 4s <= 32
      if (4 * s <= 32) __syncwarp(); else __syncthreads();
    }
    __syncthreads();
    // across the cluster: CTA 0 combines the G block averages (G = 1: the scaling coefficient)
    if constexpr (G == 1) {
      if (t == 0) buf[0] = coef<R, MODE>(buf[0], 0, acc);
    } else {
      constexpr int logG = G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : 4;
      cg::this_cluster().sync();
      if (rank == 0 && t == 0) {
        cg::cluster_group cl = cg::this_cluster();
        R v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) v[g] = cl.map_shared_rank(buf, g)[0];
#pragma unroll
        for (int lam = 0; lam < logG; ++lam) {
          const int s = 1 << lam;
#pragma unroll
          for (int g = 0; g < G; g += 2 * s) {
            const R x0 = v[g], x1 = v[g + s];
            v[g] = (x0 + x1) * r2;
            v[g + s] = coef<R, MODE>((x0 - x1) * r2, ((int64_t)1 << (logG - 1 - lam)) + (g >> (lam + 1)), acc);
          }
        }
        v[0] = coef<R, MODE>(v[0], 0, acc);
        if constexpr (MODE != MODE_FORWARD) {
#pragma unroll
          for (int lam = logG - 1; lam >= 0; --lam) {
            const int s = 1 << lam;
#pragma unroll
            for (int g = 0; g < G; g += 2 * s) {
              const R a0 = v[g], d0 = v[g + s];
              v[g] = (a0 + d0) * r2;
              v[g + s] = (a0 - d0) * r2;
            }
          }
#pragma unroll
          for (int g = 0; g < G; ++g) cl.map_shared_rank(buf, g)[0] = v[g];
        }
      }
      cg::this_cluster().sync();
    }
    __syncthreads();
    if constexpr (MODE != MODE_FORWARD) {  // MODE_FORWARD: analysis only
      // synthesis across the threads, coarsest first
      for (int lam = logTc - 1; lam >= 0; --lam) {
        const int s = 1 << lam;
        if (act && (t & (2 * s - 1)) == 0) {
          const R a0 = buf[t], d0 = buf[t + s];
          buf[t] = (a0 + d0) * r2;
          buf[t + s] = (a0 - d0) * r2;
        }
        // the next level reads slot t + s (written here by thread t): one warp while 2s <= 32
        if (2 * s <= 32) __syncwarp(); else __syncthreads();
      }
      // synthesis inside the thread
      if (act) {
        for (int l = logV - 1; l >= 0; --l) {
          const int s = 1 << l;
          for (int i = 0; i < V; i += 2 * s) {
            const R a0 = buf[i * Tc + t], d0 = buf[(i + s) * Tc + t];
            buf[i * Tc + t] = (a0 + d0) * r2;
            buf[(i + s) * Tc + t] = (a0 - d0) * r2;
          }
        }
      }
    }
    __syncthreads();
    return to_double(acc);
  }
};

// shared memory: the residual buffer (8 bytes per value) and the PCG input (4 bytes)
size_t haar_smem_bytes(int G, int64_t max_n) { return (size_t)(max_n / G) * 12; }

cudaError_t launch_haar_solver(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define L_(g) launch_t<g, HaarOp<g>, HaarOp<1>, float, StateDF>(a, smem, grid_clusters, st)
  MFIPM_G_SWITCH(G, L_)
#undef L_
  return cudaErrorInvalidValue;
}

int max_active_clusters_haar(int G, int64_t max_n) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define O_(g) occupancy_t<g, HaarOp<g>, HaarOp<1>, float, StateDF>(smem)
  MFIPM_G_SWITCH(G, O_)
#undef O_
  return 0;
}

// The same solver with a float64 PCG (MFIPM_PREC_FP64): operator products, PCG vectors and
// preconditioner in float64, iterate in double-float.
cudaError_t launch_haar_solver_f64pcg(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define L_(g) launch_t<g, HaarOp<g>, HaarOp<1>, double, StateDF>(a, smem, grid_clusters, st)
  MFIPM_G_SWITCH(G, L_)
#undef L_
  return cudaErrorInvalidValue;
}

int max_active_clusters_haar_f64pcg(int G, int64_t max_n) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define O_(g) occupancy_t<g, HaarOp<g>, HaarOp<1>, double, StateDF>(smem)
  MFIPM_G_SWITCH(G, O_)
#undef O_
  return 0;
}

}  // namespace mfipm

namespace mfipm {

// Reverse mode (mfipm_backward) on the partial Haar operator: float32 adjoint PCG, float64 A w.
cudaError_t launch_bwd_haar(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define L_(g) launch_bwd_t<g, HaarOp<g>, float>(a, smem, grid_clusters, st)
  MFIPM_G_SWITCH(G, L_)
#undef L_
  return cudaErrorInvalidValue;
}

int max_active_clusters_bwd_haar(int G, int64_t max_n) {
  const size_t smem = haar_smem_bytes(G, max_n);
#define O_(g) occupancy_bwd_t<g, HaarOp<g>, float>(smem)
  MFIPM_G_SWITCH(G, O_)
#undef O_
  return 0;
}

}  // namespace mfipm
