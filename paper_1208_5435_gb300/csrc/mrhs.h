// Host interface of the shared-A multi-right-hand-side solver (mrhs.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "internal.h"

namespace mfipm {

// C[c][r] = sum_k Aop[r][k] * Bop[c][k]: Aop rows x K and Bop N x K, both bf16 row-major
// (K-major); C is N x rows float32.
// With split-K the result is `splits` slices of N x rows (their sum is the product).
using GemmFn = cudaError_t (*)(void* ctx, const void* Aop, const void* Bop, float* C, int rows, int N, int K,
                               int splits, cudaStream_t st, int stages);

struct MrhsCall {
  int64_t m, n, lda;
  int R;
  const void* A;          // DEVICE bf16 m x n
  double a_scale, rho;
  const double* const* b; // HOST array of DEVICE pointers
  const double* tau;      // HOST
  double* const* x;       // HOST array of DEVICE pointers
  double* const* zs_out;  // HOST array or null
  mfipm_info* infos_dev;  // DEVICE
  void* workspace;
  size_t ws_bytes;
  SolveParams prm;
  cudaStream_t stream;
  GemmFn gemm;
  void* gemm_ctx;
  int splits1, splits2;   // split-K slices of T = A W and Y = A^T T
  int stages1, stages2;   // their tcgen05 ring stages (3 or 4)
  int* err_dev;           // DEVICE error word of the GEMMs (MFIPM_TIMEOUT)
  int resid_tc;           // residual by exact digit slices on the tcgen05 GEMM (else FP32 pipes)
};

constexpr int kMaxSplits = 8;

size_t mrhs_workspace_bytes(int64_t m, int64_t n, int R);
// whether the tensor-core residual can run for these shapes (GEMM N = R <= 256, K % 8 == 0)
bool mrhs_resid_tc_supported(int64_t m, int64_t n, int R);

// Partial-DCT problems of one length n above the cluster solver's reach: the same lockstep
// IPM with the multi-pass operator of large_dct.cu.
struct LdCall {
  int64_t n;
  int R;
  const int64_t* m;              // HOST, rows per problem
  const int64_t* const* rows;    // HOST array of DEVICE pointers
  const double* const* b;        // HOST array of DEVICE pointers
  const double* tau;             // HOST (solve)
  double* const* x;              // HOST array of DEVICE pointers (solve output)
  double* const* zs_out;         // HOST array or null (solve)
  const double* const* zs_in;    // backward: final iterates of the forward solve
  const double* const* gx;       // backward: dL/dx
  double* const* grad_b;         // backward: HOST array or null
  double* grad_tau;              // backward: HOST or null
  mfipm_info* infos;             // HOST, R entries
  void* workspace;
  size_t ws_bytes;
  SolveParams prm;
  cudaStream_t stream;
};
size_t large_dct_workspace_bytes(int64_t n, int R);
int large_dct_solve(const LdCall& call, std::string* msg);
int large_dct_backward(const LdCall& call, std::string* msg);
// CUDA-event time of the operator products A^T A w of the last large_dct_solve / _backward
// on this thread (ms = -1 if none), their algorithmic bytes (8 per index per product) and
// the number of kernels that solve launched
void large_dct_set_timing(bool on);
void large_dct_timing(double* ms, double* bytes, int64_t* products, int64_t* launches);
int mrhs_solve(const MrhsCall& call, std::string* msg);
cudaError_t gemm_simple(void*, const void* Aop, const void* Bop, float* C, int rows, int N, int K, int splits,
                        cudaStream_t st, int stages);
// tensor-core GEMM (tc_gemm.cu)
bool tc_gemm_supported(int rows, int N, int K);
int tc_gemm_splits(int rows, int K, int num_sms);
cudaError_t tc_gemm(const void* Aop, const void* Bop, float* C, int rows, int N, int K, int splits, int* err,
                    cudaStream_t st, int stages = 4);
// ||A||_F^2 of a bf16 matrix (device result in *out)
cudaError_t bf16_fro2(const void* A, int64_t m, int64_t n, int64_t lda, double* out, cudaStream_t st);

}  // namespace mfipm
