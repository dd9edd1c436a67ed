// bf16 "TN" GEMM on the 5th-generation tensor cores (tcgen05) for the shared-A solver:
//     C_s[c][r] = sum_{k in split s} Aop[r][k] * Bop[c][k]
// Aop (rows x K) and Bop (N x K) are bf16 row-major, i.e. both K-major; C has `splits`
// slices of N x rows float32 (the consumer adds them, which keeps the sum deterministic).
//
// One CTA computes a 128-row x BN tile: one thread issues TMA loads (128-byte swizzle) into a
// three- or four-stage shared-memory ring, one thread issues tcgen05.mma (M = 128, N = BN, K = 16, bf16
// in, float32 accumulators in tensor memory), and all four warps read the accumulators back
// with tcgen05.ld and store them.  Stages are handed over with mbarriers; every wait is
// bounded and, on expiry, records an error code and abandons the tile (no hang).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "mrhs.h"

namespace mfipm {
namespace tc {

constexpr int kBM = 128, kBK = 64, kThreadsTc = 128;
constexpr uint32_t kTileA = kBM * kBK * 2;  // 16 KiB
constexpr long long kSpinLimit = 1ll << 22;  // polls of an mbarrier before giving up (well above 1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the phase did not complete within kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), tile base 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);     // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}
// instruction descriptor: float32 accumulators, bf16 A and B, both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t idesc_bf16(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

// ST ring stages: 4 by default; 3 leaves room for two CTAs per SM at BN = 128 (autotuned)
template <int BN, int ST>
__global__ void __launch_bounds__(kThreadsTc, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float* C,
                   int rows, int N, int K, int kt_per_split, int* err) {
  constexpr uint32_t kTileB = BN * kBK * 2;
  constexpr int kTmemCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + ST * kTileA;
  __shared__ __align__(8) uint64_t full_bar[ST], empty_bar[ST], done_bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, split = blockIdx.y;
  const int kt0 = split * kt_per_split;
  const int ktiles = min(kt_per_split, (K + kBK - 1) / kBK - kt0);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (ktiles > 0) {
    if (warp == 0 && lane == 0) {
      // producer: TMA loads of the A and B tiles of each k-step
      int issued = 0;
      for (int kt = 0; kt < ktiles; ++kt) {
        const int s = kt % ST;
        const uint32_t ph = (uint32_t)(kt / ST) & 1u;
        if (kt >= ST && !mbar_wait(&empty_bar[s], ph ^ 1u)) {
          atomicCAS(err, 0, MFIPM_TIMEOUT);
          break;
        }
        mbar_expect_tx(&full_bar[s], kTileA + kTileB);
        const int kx = (kt0 + kt) * kBK;
        tma_load_2d(sA + s * kTileA, &mapA, kx, m0, &full_bar[s]);
        tma_load_2d(sB + s * kTileB, &mapB, kx, 0, &full_bar[s]);
        issued = kt + 1;
      }
      // no copy may still be in flight when the CTA leaves: wait (bounded) for the last load
      // of every stage (phases of one stage complete in order)
      for (int kt = (issued > ST ? issued - ST : 0); kt < issued; ++kt)
        if (!mbar_wait(&full_bar[kt % ST], (uint32_t)(kt / ST) & 1u)) atomicCAS(err, 0, MFIPM_TIMEOUT);
    } else if (warp == 1 && lane == 0) {
      // MMA issuer: four K=16 steps per stage, accumulate in tensor memory
      constexpr uint32_t idesc = idesc_bf16(BN);
      bool ok = true;
      for (int kt = 0; kt < ktiles && ok; ++kt) {
        const int s = kt % ST;
        const uint32_t ph = (uint32_t)(kt / ST) & 1u;
        if (!mbar_wait(&full_bar[s], ph)) {
          atomicCAS(err, 0, MFIPM_TIMEOUT);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA + s * kTileA), b0 = smem_u32(sB + s * kTileB);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint64_t ad = smem_desc_sw128(a0 + kk * 32), bd = smem_desc_sw128(b0 + kk * 32);
          const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty_bar[s]))
                     : "memory");
      }
      if (ok)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done_bar))
                     : "memory");
    }
  }
  __syncwarp();
  // epilogue: every thread owns one accumulator row (tensor-memory lane 32*warp + lane)
  bool have = ktiles > 0;
  if (have) {
    if (!mbar_wait(&done_bar, 0)) {
      if (lane == 0) atomicCAS(err, 0, MFIPM_TIMEOUT);
      have = false;
    }
  }
  have = __all_sync(0xffffffffu, have);  // tcgen05.ld is warp-collective
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r = m0 + warp * 32 + lane;
  float* Cs = C + (size_t)split * N * rows;
#pragma unroll
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    if (have) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = 0u;
    }
    if (r < rows) {
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int c = c0 + q;
        if (c < N) Cs[(size_t)c * rows + r] = __uint_as_float(v[q]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2D bf16 tensor (rows x K, K contiguous), box = box_rows x 64, 128-byte swizzle
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t K, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int ST>
cudaError_t launch_bn(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int rows, int N, int K, int splits,
                      int kt_per, int* err, cudaStream_t st) {
  const size_t smem = 1024 + (size_t)ST * (kTileA + BN * kBK * 2);
  auto kern = tc_gemm_kernel<BN, ST>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e) return e;
  kern<<<dim3((unsigned)((rows + kBM - 1) / kBM), (unsigned)splits), kThreadsTc, smem, st>>>(ma, mb, C, rows, N, K,
                                                                                            kt_per, err);
  return cudaGetLastError();
}

}  // namespace tc

bool tc_gemm_supported(int rows, int N, int K) { return N >= 1 && N <= 256 && K % 8 == 0 && rows >= 1 && tc::encode_fn(); }

// Split count for a GEMM: enough CTAs to cover the SMs, at least 8 k-steps per split.
int tc_gemm_splits(int rows, int K, int num_sms) {
  const int mt = (rows + tc::kBM - 1) / tc::kBM, kt = (K + tc::kBK - 1) / tc::kBK;
  int s = 1;
  while (mt * s * 2 <= num_sms && kt / (s * 2) >= 8) s *= 2;
  return s;
}

cudaError_t tc_gemm(const void* Aop, const void* Bop, float* C, int rows, int N, int K, int splits, int* err,
                    cudaStream_t st, int stages) {
  const int bn = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  CUtensorMap ma, mb;
  if (!tc::make_map(&ma, Aop, rows, K, tc::kBM) || !tc::make_map(&mb, Bop, N, K, bn)) return cudaErrorInvalidValue;
  const int kt = (K + tc::kBK - 1) / tc::kBK;
  const int kt_per = (kt + splits - 1) / splits;
  if (stages == 3) {
    switch (bn) {
      case 32: return tc::launch_bn<32, 3>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
      case 64: return tc::launch_bn<64, 3>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
      case 128: return tc::launch_bn<128, 3>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
      default: return tc::launch_bn<256, 3>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
    }
  }
  switch (bn) {
    case 32: return tc::launch_bn<32, 4>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
    case 64: return tc::launch_bn<64, 4>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
    case 128: return tc::launch_bn<128, 4>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
    default: return tc::launch_bn<256, 4>(ma, mb, C, rows, N, K, splits, kt_per, err, st);
  }
}

}  // namespace mfipm
