// Instantiation and launch of the node-centric kernel (resident RVEs) and
// of the thread-block-cluster kernel (large RVEs, mixed precision), in a
// translation unit of their own so that the build compiles them in parallel
// with the two-phase kernel's.
#include <mutex>

#include "dr_cluster.cuh"
#include "dr_launch.cuh"
#include "dr_node.cuh"

namespace rvegpu {

template <typename T, int NT, int NPT>
int launch_node(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  auto fn = dr_node_kernel<T, NT, NPT>;
  static int smem_set[64] = {};
  static std::mutex smem_mu;
  const int rc = set_smem(fn, bin.smem_node, smem_set, smem_mu);
  if (rc != RVE_OK) return rc;
  DrArgs<T> b = a;
  b.work = bin.d_work;
  b.n_work = bin.n;
  if (bin.check_every > 0) b.check_every = bin.check_every;
  return launch_k(fn, unsigned(bin.n), NT, bin.smem_node, s, bin.pdl, b);
}

template <typename T, int NT>
int launch_node_npt(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  switch (bin.npt) {
    case 1: return launch_node<T, NT, 1>(a, bin, s);
    case 2: return launch_node<T, NT, 2>(a, bin, s);
    case 4: return launch_node<T, NT, 4>(a, bin, s);
  }
  return fail(RVE_EINVAL, "nodes per thread must be 1, 2 or 4");
}

template <typename T>
int launch_node_nt(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  switch (bin.nt) {
    case 64: return launch_node_npt<T, 64>(a, bin, s);
    case 128: return launch_node_npt<T, 128>(a, bin, s);
    case 256: return launch_node_npt<T, 256>(a, bin, s);
    case 512: return launch_node_npt<T, 512>(a, bin, s);
    case 1024: return launch_node_npt<T, 1024>(a, bin, s);
  }
  return fail(RVE_EINVAL, "threads per CTA must be 64, 128, 256, 512 or 1024");
}

int launch_node_any(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) { return launch_node_nt(a, bin, s); }
int launch_node_any(const DrArgs<double>& a, const Bin& bin, cudaStream_t s) { return launch_node_nt(a, bin, s); }

// One cluster of bin.cl CTAs per work item (streamed-size RVEs held in the
// cluster's distributed shared memory).
// Opt the cluster kernel in to at least `smem` bytes of dynamic shared
// memory; one cache per instantiation for the launches and the capacity
// queries alike, so the attribute is only ever raised.
template <typename T, int NPT>
int cluster_smem(size_t smem) {
  static int smem_set[64] = {};
  static std::mutex smem_mu;
  return set_smem(dr_cluster_kernel<T, CLUSTER_NT, NPT>, smem, smem_set, smem_mu);
}

template <typename T, int NPT>
int launch_cluster(const DrArgs<T>& a, const Bin& bin, cudaStream_t s) {
  auto fn = dr_cluster_kernel<T, CLUSTER_NT, NPT>;
  const int rc = cluster_smem<T, NPT>(bin.smem_cluster);
  if (rc != RVE_OK) return rc;
  DrArgs<T> b = a;
  b.work = bin.d_work;
  b.n_work = bin.n;
  if (bin.check_every > 0) b.check_every = bin.check_every;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(bin.n) * unsigned(bin.cl), 1, 1);
  cfg.blockDim = dim3(CLUSTER_NT, 1, 1);
  cfg.dynamicSmemBytes = bin.smem_cluster;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(bin.cl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RVE_CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, b));
  return RVE_OK;
}

// Clusters of `cl` CTAs of the cluster kernel with `smem` bytes each that
// the device can hold at once (0: the configuration cannot run).
template <typename T, int NPT>
int cluster_capacity(int cl, size_t smem, int* n_clusters) {
  auto fn = dr_cluster_kernel<T, CLUSTER_NT, NPT>;
  const int rc = cluster_smem<T, NPT>(smem);
  if (rc != RVE_OK) return rc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(cl), 1, 1);
  cfg.blockDim = dim3(CLUSTER_NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = unsigned(cl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RVE_CUDA_TRY(cudaOccupancyMaxActiveClusters(n_clusters, fn, &cfg));
  return RVE_OK;
}

int launch_cluster_any(const DrArgs<float>& a, const Bin& bin, cudaStream_t s) {
  if (bin.cl_npt == 1) return launch_cluster<float, 1>(a, bin, s);
  if (bin.cl_npt == 2) return launch_cluster<float, 2>(a, bin, s);
  return fail(RVE_EINVAL, "cluster bins hold 1 or 2 free nodes per thread");
}

int cluster_capacity_f32(int npt, int cl, size_t smem, int* n_clusters) {
  if (npt == 1) return cluster_capacity<float, 1>(cl, smem, n_clusters);
  if (npt == 2) return cluster_capacity<float, 2>(cl, smem, n_clusters);
  *n_clusters = 0;
  return RVE_OK;
}

}  // namespace rvegpu
