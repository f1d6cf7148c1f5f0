// Fused batched kernel, FP64 throughout, viscous damping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_viscous(const DrArgs<double>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<double, VAR_VISCOUS>(a, bin, s);
}
}  // namespace rvegpu
