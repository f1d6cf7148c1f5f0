// Fused batched kernel, FP64 throughout, viscous damping with the energy-balance bookkeeping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_energy(const DrArgs<double>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<double, VAR_ENERGY>(a, bin, s);
}
}  // namespace rvegpu
