// Single-block work groups of the register-resident kernel (lbks_resident.cuh):
// whole lattices of up to NT S sites and segments of longer ones.
#include "lbks_resident.cuh"

namespace lbks {

namespace {

template <int Q, int ST, int S>
cudaError_t prepare_t(int NT, int* blocks_per_sm) {
  if (NT > ResidentCfg<ST, S>::kMaxThreads || NT % 32 != 0) return cudaErrorInvalidValue;
  // the opt-in covers the largest block of this instantiation, so that preparing a
  // smaller tiling later never lowers it under a larger one already prepared
  const size_t smem = smem_bytes_t<Q, ST, S>(NT);
  cudaError_t e = cudaFuncSetAttribute(resident_kernel<Q, ST, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes_t<Q, ST, S>(ResidentCfg<ST, S>::kMaxThreads));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, resident_kernel<Q, ST, S, 1>, NT, smem);
}

template <int Q, int ST, int S>
cudaError_t launch_t(const ResidentLaunch& L, cudaStream_t s) {
  ResidentArgs a{L.src, L.dst, L.runs, L.pieces, L.bundles, L.nbundles, L.queue, L.ksteps, L.flags, L.kx, L.wait_limit, L.withhold_step};
  resident_kernel<Q, ST, S, 1><<<L.grid, L.NT, smem_bytes_t<Q, ST, S>(L.NT), s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool resident_supported(int Q, int storage, int S, int NT) {
  if (Q != 5 && Q != 7) return false;
  if (storage != kF64 && storage != kF32 && storage != kF16S) return false;
  if (S != 4 && S != 6 && S != 8 && S != 12 && S != 16 && S != 18 && S != 20) return false;
  if (storage == kF64 && S > 8) return false;
  const int maxt = storage == kF64 ? 256 : (S <= 8 ? 512 : (S <= 12 ? 384 : 256));
  return NT >= 32 && NT <= maxt && NT % 32 == 0;
}

cudaError_t resident_prepare(int Q, int storage, int S, int NT, int* blocks_per_sm) {
  if (!resident_supported(Q, storage, S, NT)) return cudaErrorInvalidValue;
  LBKS_RESIDENT_DISPATCH(return (prepare_t<Qc, STc, Sc>(NT, blocks_per_sm)));
  return cudaErrorInvalidValue;
}

cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s) {
  if (L.collapse) return launch_collapse_resident(L, s);
  const int Q = L.Q, storage = L.storage, S = L.S;
  if (!resident_supported(Q, storage, S, L.NT)) return cudaErrorInvalidValue;
  if (L.nbundles == 0 || L.grid == 0) return cudaSuccess;
  if (L.cl == 2) return launch_resident_cluster(L, s);
  if (L.cl != 1) return cudaErrorInvalidValue;
  LBKS_RESIDENT_DISPATCH(return (launch_t<Qc, STc, Sc>(L, s)));
  return cudaErrorInvalidValue;
}

}  // namespace lbks
