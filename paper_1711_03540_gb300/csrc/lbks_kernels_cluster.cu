// Two-block work groups (thread block clusters of 2) of the register-resident
// kernel (lbks_resident.cuh): whole lattices of up to 2 NT S sites, with the
// values crossing the block edge read from the other block's shared memory.
#include "lbks_resident.cuh"

namespace lbks {

namespace {

template <int Q, int ST, int S>
cudaLaunchConfig_t cluster_config(int grid, int NT, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2 * grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem_bytes_t<Q, ST, S>(NT);
  cfg.stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = 2;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int Q, int ST, int S>
cudaError_t prepare_t(int NT, int* max_clusters) {
  if (NT > ResidentCfg<ST, S>::kMaxThreads || NT % 32 != 0) return cudaErrorInvalidValue;
  // the opt-in covers the largest block of this instantiation (see the single-block one)
  cudaError_t e = cudaFuncSetAttribute(resident_kernel<Q, ST, S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes_t<Q, ST, S>(ResidentCfg<ST, S>::kMaxThreads));
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr;
  const cudaLaunchConfig_t cfg = cluster_config<Q, ST, S>(1, NT, nullptr, &attr);
  return cudaOccupancyMaxActiveClusters(max_clusters, resident_kernel<Q, ST, S, 2>, &cfg);
}

template <int Q, int ST, int S>
cudaError_t launch_t(const ResidentLaunch& L, cudaStream_t s) {
  const ResidentArgs a{L.src, L.dst, L.runs, L.pieces, L.bundles, L.nbundles, L.queue, L.ksteps, L.flags, L.kx, L.wait_limit, L.withhold_step};
  cudaLaunchAttribute attr;
  const cudaLaunchConfig_t cfg = cluster_config<Q, ST, S>(L.grid, L.NT, s, &attr);
  return cudaLaunchKernelEx(&cfg, resident_kernel<Q, ST, S, 2>, a);
}

}  // namespace

cudaError_t resident_cluster_prepare(int Q, int storage, int S, int NT, int* max_clusters) {
  if (!resident_supported(Q, storage, S, NT)) return cudaErrorInvalidValue;
  LBKS_RESIDENT_DISPATCH(return (prepare_t<Qc, STc, Sc>(NT, max_clusters)));
  return cudaErrorInvalidValue;
}

cudaError_t launch_resident_cluster(const ResidentLaunch& L, cudaStream_t s) {
  const int Q = L.Q, storage = L.storage, S = L.S;
  if (!resident_supported(Q, storage, S, L.NT) || L.cl != 2) return cudaErrorInvalidValue;
  if (L.nbundles == 0 || L.grid == 0) return cudaSuccess;
  LBKS_RESIDENT_DISPATCH(return (launch_t<Qc, STc, Sc>(L, s)));
  return cudaErrorInvalidValue;
}

}  // namespace lbks
