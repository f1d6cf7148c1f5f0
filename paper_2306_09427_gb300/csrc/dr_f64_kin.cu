// Fused batched kernel, FP64 throughout, kinetic damping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_kinetic(const DrArgs<double>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<double, VAR_KINETIC>(a, bin, s);
}
}  // namespace rvegpu
