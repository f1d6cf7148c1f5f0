// Fused batched kernel, mixed precision (FP32 forces/updates, FP64 sums), viscous damping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_viscous(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<float, VAR_VISCOUS>(a, bin, s);
}
}  // namespace rvegpu
