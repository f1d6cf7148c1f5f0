// Fused batched kernel, FP64 throughout.
#include "dr_launch.cuh"

namespace rvegpu {
int launch_bin(const DrArgs<double>& a, const Bin& bin, cudaStream_t s) { return launch_bin_t<double>(a, bin, s); }
}  // namespace rvegpu
