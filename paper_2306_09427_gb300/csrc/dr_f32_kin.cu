// Fused batched kernel, mixed precision, kinetic damping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_kinetic(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<float, VAR_KINETIC>(a, bin, s);
}
}  // namespace rvegpu
