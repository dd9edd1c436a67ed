// Host interface of the multi-pass partial-DCT operator (large_dct.cu) for R problems of
// one length n (a power of two), vectors stored problem after problem (R x n).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lockstep.h"

namespace mfipm {

constexpr int64_t kLdMinN = 1024;         // four-step split needs N2 >= 16 columns
constexpr int64_t kLdMaxN = 1 << 20;      // double-float column block must fit shared memory

struct LdShape {
  int logN, logL, logN1, logN2;  // n = 2^logN, L = n/2 = N1 N2
};
LdShape ld_shape(int64_t n);
bool ld_supported(int64_t n);

struct LdArgs {
  int logN, logL, logN1, logN2, log2_tw;
  int gate;                  // GATE_ALL / GATE_ACTIVE / GATE_LIVE on col[j]
  const Col* col;
  const float2* pin;         // normal: (p_u, p_v) pairs, w = p_u - p_v
  float* yout;               // normal: A^T A w
  const float2* din;         // resid / forward: x, double-float (hi, lo)
  float2* dout;              // resid: A^T (A x - b), double-float
  void* inter;               // R x L complex intermediate (double-float size)
  const uint8_t* mask;       // R x n sampled-row mask
  uint8_t* mcode;            // R x (N1/2) x (N2+1) mask bits per pass-B work item (ld_mask_codes)
  const double* bsu;         // R x n  b scattered / DCT scale
  const float2* bsu_df;      // the same, double-float
  double* fwd;               // forward: R x n orthonormal DCT-II coefficients
  double* part2;             // per (problem, row-pair block) masked energy, stride kpart
  int nb2, kpart;
  const float2* tw32;        // level-ordered twiddles up to level logN + 2
  const float4* twdf;
};

// once per solve, after the mask is built
cudaError_t ld_mask_codes(const LdArgs& a, int R, cudaStream_t st);
size_t ld_mask_code_bytes(int64_t n, int R);
cudaError_t ld_normal(const LdArgs& a, int R, cudaStream_t st);
cudaError_t ld_resid(const LdArgs& a, int R, cudaStream_t st);
cudaError_t ld_resid_f32(const LdArgs& a, int R, cudaStream_t st);  // float32 chain, same output
cudaError_t ld_forward(const LdArgs& a, int R, cudaStream_t st);

}  // namespace mfipm
