// Instantiation and launch of the fused kernel for one bin.
#pragma once

#include <mutex>

#include "batch.h"
#include "dr_fused.cuh"

namespace rvegpu {

// Opt a kernel in to `smem` bytes of dynamic shared memory (once per size
// and device).  The check and the attribute call stay together under one
// lock, so no thread launches on a size another thread has recorded but not
// yet set.
template <typename K>
int set_smem(K fn, size_t smem, int (&smem_set)[64], std::mutex& mu) {
  int dev = 0;
  RVE_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 64 || smem_set[dev] < int(smem)) {
    RVE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    if (dev < 64) smem_set[dev] = int(smem);
  }
  return RVE_OK;
}

// Launch fn<<<grid, block, smem, s>>>(arg); with pdl, as a programmatic
// dependent of the launch before it on s: it may start once every CTA of
// that launch has signalled (griddepcontrol.launch_dependents, at the top of
// the DR kernels) instead of when that launch ends.  It reads nothing that
// launch writes.  Graph capture keeps the edge.
template <typename K, typename Arg>
int launch_k(K fn, unsigned grid, unsigned block, size_t smem, cudaStream_t s, bool pdl, const Arg& arg) {
  if (!pdl) {
    fn<<<grid, block, smem, s>>>(arg);
    RVE_CUDA_TRY(cudaGetLastError());
    return RVE_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RVE_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, arg));
  return RVE_OK;
}

// The node-centric and cluster kernels are instantiated in translation
// units of their own (dr_node_launch.cu), compiled in parallel with these.
int launch_node_any(const DrArgs<float>& a, const Bin& bin, cudaStream_t s);
int launch_node_any(const DrArgs<double>& a, const Bin& bin, cudaStream_t s);
int launch_cluster_any(const DrArgs<float>& a, const Bin& bin, cudaStream_t s);

template <typename T, int NT, int NPT, int MODE, int VAR>
int launch_variant(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  if constexpr (MODE == 0 && VAR == VAR_VISCOUS) {
    if (a.node_kernel && bin.smem_node > 0) return launch_node_any(a, bin, s);
  }
  auto fn = dr_fused_kernel<T, NT, NPT, MODE, VAR>;
  // largest dynamic shared memory opted in so far, per device ordinal; the
  // check and the attribute call stay together under one lock, so no thread
  // launches on a size another thread has recorded but not yet set
  static int smem_set[64] = {};
  static std::mutex smem_mu;
  int dev = 0;
  RVE_CUDA_TRY(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lock(smem_mu);
    if (dev >= 64 || smem_set[dev] < int(bin.smem)) {
      RVE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bin.smem)));
      if (dev < 64) smem_set[dev] = int(bin.smem);
    }
  }
  DrArgs<T> b = a;
  b.work = bin.d_work;
  b.n_work = bin.n;
  if (bin.check_every > 0) b.check_every = bin.check_every;
  return launch_k(fn, unsigned(bin.n), NT, bin.smem, s, bin.pdl, b);
}

template <typename T, int NT, int NPT, int VAR>
int launch_mode(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  if constexpr (VAR == VAR_VISCOUS && std::is_same<T, float>::value) {
    if (bin.mode != 0 && bin.cl > 0 && a.node_kernel) return launch_cluster_any(a, bin, s);
  }
  switch (bin.mode) {
    case 0: return launch_variant<T, NT, NPT, 0, VAR>(a, bin, s);
    case 1:
      if constexpr (NT >= 512 && NPT >= 2) return launch_variant<T, NT, NPT, 1, VAR>(a, bin, s);
      break;
    case 2:
      if constexpr (NT >= 512 && NPT >= 2) return launch_variant<T, NT, NPT, 2, VAR>(a, bin, s);
      break;
  }
  return fail(RVE_EINVAL, "no kernel variant for this bin");
}

template <typename T, int NT, int VAR>
int launch_npt(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  switch (bin.npt) {
    case 1: return launch_mode<T, NT, 1, VAR>(a, bin, s);
    case 2: return launch_mode<T, NT, 2, VAR>(a, bin, s);
    case 4: return launch_mode<T, NT, 4, VAR>(a, bin, s);
  }
  return fail(RVE_EINVAL, "nodes per thread must be 1, 2 or 4");
}

template <typename T, int VAR>
int launch_bin_t(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  if (bin.n == 0) return RVE_OK;
  switch (bin.nt) {
    case 64: return launch_npt<T, 64, VAR>(a, bin, s);
    case 128: return launch_npt<T, 128, VAR>(a, bin, s);
    case 256: return launch_npt<T, 256, VAR>(a, bin, s);
    case 512: return launch_npt<T, 512, VAR>(a, bin, s);
    case 1024: return launch_npt<T, 1024, VAR>(a, bin, s);
  }
  return fail(RVE_EINVAL, "threads per CTA must be 64, 128, 256, 512 or 1024");
}

}  // namespace rvegpu
