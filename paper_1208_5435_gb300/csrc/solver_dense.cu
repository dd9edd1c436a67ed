// Instantiations of the persistent IPM kernel for dense float64 A.
#include "solver_impl.cuh"

namespace mfipm {

cudaError_t launch_dense_solver(int G, bool fp64_pcg, const KernelArgs& a, int64_t max_n, int64_t max_m,
                                int grid_clusters, cudaStream_t st) {
  const size_t smem = dense_smem_bytes(G, fp64_pcg, max_n, max_m);
  if (fp64_pcg) {
#define L_(g) launch_t<g, DenseOp<g>, DenseOp<1>, double, StateF64>(a, smem, grid_clusters, st)
    MFIPM_G_SWITCH(G, L_)
#undef L_
  } else {
#define L_(g) launch_t<g, DenseOp<g>, DenseOp<1>, float, StateF64>(a, smem, grid_clusters, st)
    MFIPM_G_SWITCH(G, L_)
#undef L_
  }
  return cudaErrorInvalidValue;
}

int max_active_clusters_dense(int G, bool fp64_pcg, int64_t max_n, int64_t max_m) {
  const size_t smem = dense_smem_bytes(G, fp64_pcg, max_n, max_m);
  if (fp64_pcg) {
#define O_(g) occupancy_t<g, DenseOp<g>, DenseOp<1>, double, StateF64>(smem)
    MFIPM_G_SWITCH(G, O_)
#undef O_
  } else {
#define O_(g) occupancy_t<g, DenseOp<g>, DenseOp<1>, float, StateF64>(smem)
    MFIPM_G_SWITCH(G, O_)
#undef O_
  }
  return 0;
}

}  // namespace mfipm
