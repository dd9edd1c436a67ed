// Instantiations of the reverse-mode (adjoint) kernel.
#include "solver_impl.cuh"

namespace mfipm {

cudaError_t launch_bwd_dct(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st) {
  const size_t smem = dct_smem_bytes(G, max_n);
#define L_(g) launch_bwd_t<g, DctOp<g>, float>(a, smem, grid_clusters, st)
  MFIPM_G_SWITCH(G, L_)
#undef L_
  return cudaErrorInvalidValue;
}

int max_active_clusters_bwd_dct(int G, int64_t max_n) {
  const size_t smem = dct_smem_bytes(G, max_n);
#define O_(g) occupancy_bwd_t<g, DctOp<g>, float>(smem)
  MFIPM_G_SWITCH(G, O_)
#undef O_
  return 0;
}

cudaError_t launch_bwd_dense(int G, bool fp64_pcg, const KernelArgs& a, int64_t max_n, int64_t max_m,
                             int grid_clusters, cudaStream_t st) {
  const size_t smem = dense_smem_bytes(G, fp64_pcg, max_n, max_m);
  if (fp64_pcg) {
#define L_(g) launch_bwd_t<g, DenseOp<g>, double>(a, smem, grid_clusters, st)
    MFIPM_G_SWITCH(G, L_)
#undef L_
  } else {
#define L_(g) launch_bwd_t<g, DenseOp<g>, float>(a, smem, grid_clusters, st)
    MFIPM_G_SWITCH(G, L_)
#undef L_
  }
  return cudaErrorInvalidValue;
}

int max_active_clusters_bwd_dense(int G, bool fp64_pcg, int64_t max_n, int64_t max_m) {
  const size_t smem = dense_smem_bytes(G, fp64_pcg, max_n, max_m);
  if (fp64_pcg) {
#define O_(g) occupancy_bwd_t<g, DenseOp<g>, double>(smem)
    MFIPM_G_SWITCH(G, O_)
#undef O_
  } else {
#define O_(g) occupancy_bwd_t<g, DenseOp<g>, float>(smem)
    MFIPM_G_SWITCH(G, O_)
#undef O_
  }
  return 0;
}

}  // namespace mfipm
