// Structures shared by the C-ABI layer (capi.cu) and the kernels (solver.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/mfipm.h"

namespace mfipm {

// Parameters of the IPM as the kernels read them (copied from mfipm_params).
struct SolveParams {
  double tol, tol_pcg, sigma1, sigma2, sigma3, alpha_bar, alpha_tilde, eta;
  double f32_gap;  // relative gap above which the partial-DCT outer residual runs in float32
  double mcc_beta_min, mcc_beta_max, mcc_delta, mcc_gamma;  // centrality correctors (reading R19)
  int32_t max_iter, max_iter_pcg, equal_steps, resid_fp64;
  int32_t mcc;     // multiple centrality correctors per iteration (0: the single corrector)
};

// One problem of a launch.  Vectors of length n live in the caller's workspace, in the
// operator's storage order (the partial DCT keeps its vectors permuted so that the FFT
// reads them in place; see solver.cu).
struct ProbDesc {
  int64_t n, m;
  int32_t kind;           // mfipm_op_kind
  int32_t log2n;          // partial DCT
  double tau;
  const double* b;        // DEVICE m
  double* x_out;          // DEVICE n (natural order)
  double* zs_out;         // DEVICE 4n or null
  // partial DCT
  const int64_t* rows;    // DEVICE m
  uint8_t* mask;          // DEVICE n: 1 where the DCT row is sampled
  double* bsu;            // DEVICE n: b scattered to its rows, divided by the row's DCT scale
  float2* bsu_df;         // DEVICE n: bsu as double-float (hi, lo)
  // partial DCT, persistent kernel: per frequency k < n/2 of the half-length FFT, the row-mask
  // bits of the four DCT rows k, n-k (k > 0), n/2-k, n/2+k (bits 0..3), and their four b_u
  // values as one 32-byte record (double-float: hi[4] then lo[4] as float32; float64: the
  // four values); the exchange step reads one code and at most one record per frequency
  uint8_t* mcode;         // DEVICE n/2 or null
  void* bpk;              // DEVICE n/2 records of 32 bytes or null
  // partial DCT of a general even length (mixed-radix chain): the roots table of this n
  // (gen_tw_bytes(n/2) bytes, shared by the problems of equal n), else null
  const void* twg;
  // dense
  const void* A;
  int32_t a_dtype;
  int32_t pad0;
  double a_scale;
  int64_t lda;
  // state
  double* zs;             // DEVICE 4n: per index {u, v, s_u, s_v}
  double* scratch;        // DEVICE n doubles: operator output scratch
  // mfipm_backward only
  const double* zs_in;    // DEVICE 4n: final [u; v; s_u; s_v] of the forward solve (natural order)
  const double* gx;       // DEVICE n: dL/dx
  const double* x_in;     // DEVICE n: the forward solution (dense dL/dA)
  double* grad_b;         // DEVICE m or null
  double* grad_A;         // DEVICE m x n or null (dense)
  double* grad_tau;       // DEVICE 1
  void* pcg;              // DEVICE 6 vectors of n pairs (x1, x2, r, p, d, xc), float or double pairs
  mfipm_info* info;       // DEVICE
};

struct KernelArgs {
  const ProbDesc* probs;
  int32_t batch;
  int32_t nbig;           // problems [0, nbig) are solved by a whole cluster, the rest by one CTA each
  int* queue;             // DEVICE work counters (cluster queue, CTA queue), zero at launch
  int* err;               // DEVICE error word (first failing problem's status)
  const double2* tw64;    // exp(-2 pi i j / 2^log2_tw)
  const float2* tw32;
  const float4* twdf;     // the same roots as double-float {re.hi, re.lo, im.hi, im.lo}
  int32_t log2_tw;
  int32_t phase2_only;    // a helper launch of single CTAs that takes the per-CTA queue only
  SolveParams prm;
};

// Roots table of the general-length partial DCT (L = n/2): three runs of L roots
// (exp(-2 pi i e / L), exp(-2 pi i k / n), exp(-i pi k / (2n))) in float64 pairs, then the
// same in float32 pairs, then in double-float quadruples, then the L int32 positions of the
// frequencies after the forward FFT; each part 256-byte aligned.
__host__ __device__ inline size_t gen_tw_al(size_t x) { return (x + 255) & ~(size_t)255; }
__host__ __device__ inline size_t gen_tw_off32(int64_t L) { return gen_tw_al((size_t)3 * L * 16); }
__host__ __device__ inline size_t gen_tw_offdf(int64_t L) { return gen_tw_off32(L) + gen_tw_al((size_t)3 * L * 8); }
__host__ __device__ inline size_t gen_tw_offpos(int64_t L) { return gen_tw_offdf(L) + gen_tw_al((size_t)3 * L * 16); }
__host__ __device__ inline size_t gen_tw_bytes(int64_t L) { return gen_tw_offpos(L) + gen_tw_al((size_t)L * 4); }
// Variants of the general-length partial-DCT kernel: float32 PCG with the double-float or
// the float64 iterate, and the float64 PCG.
enum { kGenDF = 0, kGenF64 = 1, kGenF64Pcg = 2 };
cudaError_t launch_gen_twiddles(void* base, int64_t n, cudaStream_t st);
cudaError_t launch_dct_gen_solver(int variant, const KernelArgs& a, int64_t max_n, int ctas, cudaStream_t st);
int max_active_ctas_dct_gen(int variant, int64_t max_n);

// Launchers implemented in solver.cu.  Return cudaError_t of the launch.
cudaError_t launch_twiddles(double2* tw64, float2* tw32, float4* twdf, int log2_tw, cudaStream_t st);
cudaError_t launch_dct_setup(const ProbDesc* probs_dev, int batch, int64_t max_n, int* err, cudaStream_t st,
                             bool pack_fp64 = false);

// Products with A and the KKT residual of a candidate x (apply.cu): what = 0: out = A in,
// 1: out = A^T in, 2: *kkt = kkt_rel(in) for (b, tau).  Synchronises st.
size_t apply_workspace_bytes(const mfipm_operator& op);
int apply_operator(int what, const mfipm_operator& op, const double* in, const double* b, double tau, double* out,
                   double* kkt, void* workspace, size_t ws_bytes, cudaStream_t st, std::string* msg);
cudaError_t launch_dct_solver_df(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
cudaError_t launch_haar_solver(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
int max_active_clusters_haar(int G, int64_t max_n);
cudaError_t launch_haar_solver_f64pcg(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
int max_active_clusters_haar_f64pcg(int G, int64_t max_n);
size_t haar_smem_bytes(int G, int64_t max_n);
cudaError_t launch_dct_solver_f64(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
cudaError_t launch_dense_solver(int G, bool fp64_pcg, const KernelArgs& a, int64_t max_n, int64_t max_m,
                                int grid_clusters, cudaStream_t st);
cudaError_t launch_dct_solver_f64pcg(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
int max_active_clusters_dct_f64pcg(int G, int64_t max_n);
int max_active_clusters_dct_df(int G, int64_t max_n);
int max_active_clusters_dct_f64(int G, int64_t max_n);
int max_active_clusters_dense(int G, bool fp64_pcg, int64_t max_n, int64_t max_m);
size_t dct_smem_bytes(int G, int64_t max_n);
size_t dense_smem_bytes(int G, bool fp64_pcg, int64_t max_n, int64_t max_m);

cudaError_t launch_bwd_dct(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
cudaError_t launch_bwd_dense(int G, bool fp64_pcg, const KernelArgs& a, int64_t max_n, int64_t max_m,
                             int grid_clusters, cudaStream_t st);
int max_active_clusters_bwd_dct(int G, int64_t max_n);
cudaError_t launch_bwd_haar(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st);
int max_active_clusters_bwd_haar(int G, int64_t max_n);
int max_active_clusters_bwd_dense(int G, bool fp64_pcg, int64_t max_n, int64_t max_m);

// Operator-only kernels for mfipm_apply_A / mfipm_apply_At / mfipm_kkt_residual:
// mode 0 = A x (out m), 1 = A^T y (out n), 2 = kkt_rel (out 1 double, device).
cudaError_t launch_apply(int mode, int G, const KernelArgs& a, const double* in, double* out,
                         cudaStream_t st);

// Measured FP32 FMA rate of the current device in TFLOP/s (probe.cu).
cudaError_t measure_fp32_fma_peak(double* tflops, cudaStream_t st);

}  // namespace mfipm
