// lb_ks_mass_energy_noalloc: the FP64 mass/energy reduction of the guard for
// callers that cannot allocate device memory.  Its per-block partial sums live
// in a fixed file-scope device array instead of memory from cudaMalloc.
#include <mutex>

#include "../../include/lb_ks.h"
#include "lbks_device.cuh"

namespace lbks {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaTileSites = 1024;
constexpr int kNaMaxTiles = 16384;  // lattices of up to 2^24 sites
constexpr int kMaxDevices = 64;

// Scratch shared by every call on a device: (mass, energy) partials of each
// 1024-site tile, then the two totals.  256 KB; every device that loads the
// library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNaMaxTiles + 2];

std::mutex g_na_mutex;
double* g_na_addr[kMaxDevices] = {};

template <int Q, int ST>
__global__ void __launch_bounds__(kNaThreads) na_partials_kernel(const void* __restrict__ fv, int64_t plane, int64_t N,
                                                                double rhobar, double scale,
                                                                double* __restrict__ scratch) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  const T* f = static_cast<const T*>(fv);
  const int64_t x0 = (int64_t)blockIdx.x * kNaTileSites;
  const int len = (N - x0 < kNaTileSites) ? (int)(N - x0) : kNaTileSites;
  double m = 0.0, e = 0.0;
  for (int k = threadIdx.x; k < len; k += blockDim.x) {
    double rho = rhobar;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      rho += static_cast<double>(to_compute(f[(int64_t)i * plane + x0 + k], static_cast<CT>(scale)));
    m += rho;
    e = __fma_rn(rho, rho, e);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  __shared__ double sm[2][kNaThreads / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sm[0][w] = m; sm[1][w] = e; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0, ee = 0.0;
    for (int i = 0; i < kNaThreads / 32; ++i) { mm += sm[0][i]; ee += sm[1][i]; }
    scratch[2 * blockIdx.x] = mm;
    scratch[2 * blockIdx.x + 1] = ee;
  }
}

// One warp adds the tile partials in a fixed order; totals go to the last two slots.
__global__ void na_total_kernel(int ntiles, double* __restrict__ scratch) {
  const int lane = threadIdx.x;
  double m = 0.0, e = 0.0;
  for (int t = lane; t < ntiles; t += 32) {
    m += scratch[2 * t];
    e += scratch[2 * t + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  if (lane == 0) {
    scratch[2 * kNaMaxTiles] = m;
    scratch[2 * kNaMaxTiles + 1] = e;
  }
}

// Device address of the scratch array on the current device, looked up once per device
// and kept for the life of the process (it does not survive cudaDeviceReset of that
// device, after which the module, and the array, are loaded anew).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = static_cast<double*>(p);
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lbks

using namespace lbks;

extern "C" int lb_ks_mass_energy_noalloc(int scheme, int precision, const void* f, int64_t plane, int64_t N,
                                         double rhobar, double scale, double* out, void* stream) {
  if ((scheme != LB_KS_D1Q5 && scheme != LB_KS_D1Q7) || precision < LB_KS_F64 || precision > LB_KS_F16S)
    return LB_KS_EINVAL;
  if (!f || !out || N < 1 || plane < N || !(scale > 0.0)) return LB_KS_EINVAL;
  if (precision != LB_KS_F16S && scale != 1.0) return LB_KS_EINVAL;  // only FP16 storage is scaled
  if (N > (int64_t)kNaTileSites * kNaMaxTiles) return LB_KS_EINVAL;  // beyond the static scratch
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return LB_KS_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ntiles = (int)((N + kNaTileSites - 1) / kNaTileSites);
#define LBKS_NA_CASE(Qv, STv)                                                                                   \
  if (scheme == Qv && precision == STv)                                                                        \
    na_partials_kernel<Qv, STv><<<ntiles, kNaThreads, 0, s>>>(f, plane, N, rhobar, scale, scratch);
  LBKS_NA_CASE(5, kF64) LBKS_NA_CASE(5, kF32) LBKS_NA_CASE(5, kF16S)
  LBKS_NA_CASE(7, kF64) LBKS_NA_CASE(7, kF32) LBKS_NA_CASE(7, kF16S)
#undef LBKS_NA_CASE
  na_total_kernel<<<1, 32, 0, s>>>(ntiles, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return LB_KS_ECUDA;
  if ((e = cudaMemcpyAsync(out, scratch + 2 * kNaMaxTiles, 2 * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess)
    return LB_KS_ECUDA;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return LB_KS_ECUDA;
  return LB_KS_OK;
}
