// Setup kernels of the mfIPM launches: twiddle table, partial-DCT row mask and scaled b.
#include "solver_impl.cuh"

namespace mfipm {

// ------------------------------------------------------------------ setup kernels
__global__ void twiddle_kernel(double2* tw64, float2* tw32, float4* twdf, int log2_tw) {
  // level-ordered: entry 2^l + j holds exp(-2 pi i j / 2^l), 1 <= l <= log2_tw, j < 2^l
  const int64_t T = (int64_t)2 << log2_tw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < T; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < 2) continue;
    const int l = 63 - __clzll((unsigned long long)e);
    const int64_t j = e - ((int64_t)1 << l);
    double s, c;
    // exp(-2 pi i j / 2^l) = cos(pi * 2j/2^l) - i sin(pi * 2j/2^l)
    sincospi(2.0 * (double)j / (double)((int64_t)1 << l), &s, &c);
    if (tw64) tw64[e] = make_double2(c, -s);
    tw32[e] = make_float2((float)c, (float)-s);
    const df re = to_df(c), im = to_df(-s);
    twdf[e] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// mask[j] = 1 and bsu[j] = b_i / alpha_j (DCT) or b_i (Haar) for j = rows[i]; validates rows.
__global__ void dct_setup_kernel(const ProbDesc* probs, int batch, int* err) {
  const ProbDesc pd = probs[blockIdx.y];
  const int64_t n = pd.n;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    pd.mask[j] = 0;
    pd.bsu[j] = 0.0;
    pd.bsu_df[j] = make_float2(0.f, 0.f);
  }
}
__global__ void dct_scatter_kernel(const ProbDesc* probs, int batch, int* err) {
  const ProbDesc pd = probs[blockIdx.y];
  const int64_t n = pd.n, m = pd.m;
  const double sc0 = sqrt((double)n), scj = sqrt(0.5 * (double)n);  // 1/alpha
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = pd.rows[i];
    const bool ok = r >= 0 && r < n && (i == 0 || pd.rows[i - 1] < r);
    if (!ok) {
      atomicCAS(err, 0, -1);  // invalid rows: reported by the host as MFIPM_INVALID_ARG
      continue;
    }
    const double bi = pd.b ? pd.b[i] : 0.0;  // no b: the mask alone
    if (!isfinite(bi)) atomicCAS(err, 0, -2);
    pd.mask[r] = 1;
    // the DCT chain works on the unnormalised transform (b over the row's scale); the Haar
    // chain on the orthonormal coefficients themselves
    const double v = pd.kind == MFIPM_OP_PARTIAL_HAAR ? bi : bi * (r == 0 ? sc0 : scj);
    pd.bsu[r] = v;
    const df vd = to_df(v);
    pd.bsu_df[r] = make_float2(vd.hi, vd.lo);
  }
}

// Per-frequency packing for the persistent kernel's exchange step (problems with mcode set):
// code[k] = mask bits of rows k, N-k (k > 0), L-k, L+k; bpk[k] = their b_u values.
__global__ void dct_pack_kernel(const ProbDesc* probs, int batch, bool fp64) {
  const ProbDesc pd = probs[blockIdx.y];
  if (!pd.mcode) return;
  const int64_t N = pd.n, L = N >> 1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i2 = k > 0 ? N - k : 0;
    const bool m1 = pd.mask[k], m2 = k > 0 && pd.mask[i2], m3 = pd.mask[L - k], m4 = pd.mask[L + k];
    pd.mcode[k] = (uint8_t)((m1 ? 1u : 0u) | (m2 ? 2u : 0u) | (m3 ? 4u : 0u) | (m4 ? 8u : 0u));
    const double b1 = m1 ? pd.bsu[k] : 0.0, b2 = m2 ? pd.bsu[i2] : 0.0;
    const double b3 = m3 ? pd.bsu[L - k] : 0.0, b4 = m4 ? pd.bsu[L + k] : 0.0;
    if (fp64) {
      double2* r = static_cast<double2*>(pd.bpk) + 2 * k;
      r[0] = make_double2(b1, b2);
      r[1] = make_double2(b3, b4);
    } else {
      const df d1 = to_df(b1), d2 = to_df(b2), d3 = to_df(b3), d4 = to_df(b4);
      float4* r = static_cast<float4*>(pd.bpk) + 2 * k;
      r[0] = make_float4(d1.hi, d2.hi, d3.hi, d4.hi);
      r[1] = make_float4(d1.lo, d2.lo, d3.lo, d4.lo);
    }
  }
}

// ------------------------------------------------------------------ launchers
size_t dct_smem_bytes(int G, int64_t max_n) {
  const int64_t M = max_n / 2 / G;
  return (size_t)M * 16 + (size_t)M * 8;
}
size_t dense_smem_bytes(int G, bool, int64_t max_n, int64_t max_m) {
  const int64_t chunk = (max_n + G - 1) / G;
  const size_t c8 = ((size_t)chunk * 8 + 255) & ~(size_t)255;
  return 2 * c8 + 3 * (size_t)((max_m + 31) & ~31) * 8;
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, float4* twdf, int log2_tw, cudaStream_t st) {
  const int64_t T = (int64_t)2 << log2_tw;
  const int blocks = (int)((T + 255) / 256 < 1024 ? (T + 255) / 256 : 1024);
  twiddle_kernel<<<blocks, 256, 0, st>>>(tw64, tw32, twdf, log2_tw);
  return cudaGetLastError();
}

cudaError_t launch_dct_setup(const ProbDesc* probs_dev, int batch, int64_t max_n, int* err, cudaStream_t st,
                             bool pack_fp64) {
  const int bx = (int)((max_n + 255) / 256 < 64 ? (max_n + 255) / 256 : 64);
  dct_setup_kernel<<<dim3(bx, batch), 256, 0, st>>>(probs_dev, batch, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  dct_scatter_kernel<<<dim3(bx, batch), 256, 0, st>>>(probs_dev, batch, err);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  dct_pack_kernel<<<dim3(bx, batch), 256, 0, st>>>(probs_dev, batch, pack_fp64);
  return cudaGetLastError();
}

}  // namespace mfipm
