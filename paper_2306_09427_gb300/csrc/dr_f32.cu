// Fused batched kernel, mixed precision (FP32 forces/updates, FP64 sums), viscous damping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_viscous(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<float, VAR_VISCOUS>(a, bin, s);
}
int cluster_capacity_f32(int npt, int cl, size_t smem, int* n_clusters) {
  if (npt == 1) return cluster_capacity<float, 1>(cl, smem, n_clusters);
  if (npt == 2) return cluster_capacity<float, 2>(cl, smem, n_clusters);
  *n_clusters = 0;
  return RVE_OK;
}
}  // namespace rvegpu
