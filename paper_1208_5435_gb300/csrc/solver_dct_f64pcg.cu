// Instantiations of the persistent IPM kernel for the partial-DCT operator with a float64 PCG
// (operator products, PCG vectors and preconditioner in float64) and a float64 iterate: the
// tight PCG tolerances of basis pursuit through a tiny tau (Sec. 5.4, tolpcg down to 1e-6),
// which a float32 PCG cannot reach.
#include "solver_impl.cuh"

namespace mfipm {

cudaError_t launch_dct_solver_f64pcg(int G, const KernelArgs& a, int64_t max_n, int grid_clusters, cudaStream_t st) {
  const size_t smem = dct_smem_bytes(G, max_n);
#define L_(g) launch_t<g, DctOp<g>, DctOp<1>, double, StateF64>(a, smem, grid_clusters, st)
  MFIPM_G_SWITCH(G, L_)
#undef L_
  return cudaErrorInvalidValue;
}

int max_active_clusters_dct_f64pcg(int G, int64_t max_n) {
  const size_t smem = dct_smem_bytes(G, max_n);
#define O_(g) occupancy_t<g, DctOp<g>, DctOp<1>, double, StateF64>(smem)
  MFIPM_G_SWITCH(G, O_)
#undef O_
  return 0;
}

}  // namespace mfipm
