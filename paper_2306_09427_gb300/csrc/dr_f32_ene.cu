// Fused batched kernel, mixed precision, viscous damping with the energy-balance bookkeeping.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin_energy(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) {
  return launch_bin_t<float, VAR_ENERGY>(a, bin, s);
}
}  // namespace rvegpu
