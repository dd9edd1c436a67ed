// Host interface of the reverse mode of the general-length partial DCT (solver_dct_gen.cu):
// the adjoint kernel of mfipm_backward on the mixed-radix chain, one CTA per problem.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace mfipm {

cudaError_t launch_bwd_dct_gen(const KernelArgs& a, int64_t max_n, int ctas, cudaStream_t st);
int max_active_ctas_bwd_dct_gen(int64_t max_n);

}  // namespace mfipm
