// HBM-streaming fused step for large lattices (one launch per step).
//
// A block owns a tile of kTile consecutive sites of one run.  Each thread
// loads kVec consecutive sites of every plane with one vector load, collides
// them in registers and writes f* to a shared-memory copy of the tile that
// also holds c_max post-collision halo sites on each side (computed by a few
// threads from the neighbouring sites, periodic wrap).  After one barrier
// every thread reads the shifted values f*_i(x - c_i) for lane-contiguous
// sites and stores them coalesced.  HBM traffic per site-update: one read and
// one write of the Q populations (plus 2 c_max halo sites per tile).
#include "lbks_device.cuh"

namespace lbks {

namespace {

constexpr int kStreamThreads = 256;
constexpr int kVec = 4;
constexpr int kTile = kStreamThreads * kVec;  // 1024 sites
constexpr int kHalo = 4;                      // >= c_max, keeps float4 stores aligned

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[kVec]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[kVec]) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct Vec4<__half> {
  static __device__ __forceinline__ void load(const __half* p, __half (&v)[kVec]) {
    const uint2 q = __ldcs(reinterpret_cast<const uint2*>(p));
    const __half2 a = *reinterpret_cast<const __half2*>(&q.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&q.y);
    v[0] = __low2half(a); v[1] = __high2half(a); v[2] = __low2half(b); v[3] = __high2half(b);
  }
};

// Aligned 16-byte shared-memory stores of kVec post-collision values of plane i
// (conflict-free; the tile row stride Q*W*sizeof(CT) is a multiple of 16 bytes).
template <int Q>
__device__ __forceinline__ void store4(float* p, const float (&g)[kVec][Q], int i) {
  *reinterpret_cast<float4*>(p) = make_float4(g[0][i], g[1][i], g[2][i], g[3][i]);
}
template <int Q>
__device__ __forceinline__ void store4(double* p, const double (&g)[kVec][Q], int i) {
  reinterpret_cast<double2*>(p)[0] = make_double2(g[0][i], g[1][i]);
  reinterpret_cast<double2*>(p)[1] = make_double2(g[2][i], g[3][i]);
}

template <int Q, int ST>
__global__ void __launch_bounds__(kStreamThreads) stream_step_kernel(Arena src, Arena dst,
                                                                     const RunDesc* __restrict__ runs,
                                                                     const Tile* __restrict__ tiles) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  constexpr int C = cmax_of(Q);
  constexpr int W = kTile + 2 * kHalo;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT* sm = reinterpret_cast<CT*>(smem_raw);  // [Q][W], tile site k at column kHalo + k

  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  const Coef<CT, Q> k = load_coef<CT, Q>(d);
  const T* fs = static_cast<const T*>(src.f) + d.off;
  T* fd = static_cast<T*>(dst.f) + d.off;
  const int len = tl.len;
  const int64_t x0 = tl.x0;

  // Phase 1: kVec consecutive sites per thread.
  {
    const int k0 = threadIdx.x * kVec;
    if (k0 < len) {
      CT g[kVec][Q];
      if (k0 + kVec <= len) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          T v[kVec];
          Vec4<T>::load(fs + (int64_t)i * src.plane + x0 + k0, v);
#pragma unroll
          for (int u = 0; u < kVec; ++u) g[u][i] = to_compute(v[u], k.scale);
        }
      } else {
#pragma unroll
        for (int u = 0; u < kVec; ++u)
#pragma unroll
          for (int i = 0; i < Q; ++i)
            g[u][i] = (k0 + u < len) ? to_compute(fs[(int64_t)i * src.plane + x0 + k0 + u], k.scale) : CT(0);
      }
#pragma unroll
      for (int u = 0; u < kVec; ++u) collide<Q, CT>(g[u], k);
      if (k0 + kVec <= len) {
#pragma unroll
        for (int i = 0; i < Q; ++i) store4(sm + i * W + kHalo + k0, g, i);
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
          for (int u = 0; u < kVec; ++u)
            if (k0 + u < len) sm[i * W + kHalo + k0 + u] = g[u][i];
      }
    }
    // Halo: C sites left of the tile and C sites right of it (periodic in the run).
    if (threadIdx.x < 2 * C) {
      const int h = threadIdx.x;
      const int col = h < C ? (kHalo - C + h) : (kHalo + len + (h - C));
      const int64_t xs = h < C ? wrap_site(x0 - C + h, d.N) : wrap_site(x0 + len + (h - C), d.N);
      CT g[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) g[i] = to_compute(fs[(int64_t)i * src.plane + xs], k.scale);
      collide<Q, CT>(g, k);
#pragma unroll
      for (int i = 0; i < Q; ++i) sm[i * W + col] = g[i];
    }
  }
  __syncthreads();
  // Phase 2: pull f*_i(x - c_i), lane-contiguous sites, coalesced stores.
#pragma unroll
  for (int u = 0; u < kVec; ++u) {
    const int kk = threadIdx.x + u * kStreamThreads;
    if (kk < len) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const CT v = sm[i * W + kHalo + kk - speed(i)];
        T out;
        from_compute(v, k.inv_scale, &out);
        __stcs(fd + (int64_t)i * dst.plane + x0 + kk, out);
      }
    }
  }
}

template <int Q, int ST>
size_t stream_smem() {
  using CT = typename StorageType<ST>::compute;
  return sizeof(CT) * Q * (kTile + 2 * kHalo);
}

template <int Q, int ST>
cudaError_t prepare_stream_t() {
  return cudaFuncSetAttribute(stream_step_kernel<Q, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)stream_smem<Q, ST>());
}

template <int Q, int ST>
cudaError_t launch_stream_t(Arena src, Arena dst, const RunDesc* runs, const Tile* tiles, int ntiles, cudaStream_t s) {
  stream_step_kernel<Q, ST><<<ntiles, kStreamThreads, stream_smem<Q, ST>(), s>>>(src, dst, runs, tiles);
  return cudaGetLastError();
}

}  // namespace

int stream_tile_sites() { return kTile; }

// Opt in to more than 48 KB of dynamic shared memory (FP64 tiles); call before any launch.
cudaError_t stream_prepare(int Q, int storage) {
  if (Q == 5 && storage == kF64) return prepare_stream_t<5, kF64>();
  if (Q == 5 && storage == kF32) return prepare_stream_t<5, kF32>();
  if (Q == 5 && storage == kF16S) return prepare_stream_t<5, kF16S>();
  if (Q == 7 && storage == kF64) return prepare_stream_t<7, kF64>();
  if (Q == 7 && storage == kF32) return prepare_stream_t<7, kF32>();
  if (Q == 7 && storage == kF16S) return prepare_stream_t<7, kF16S>();
  return cudaErrorInvalidValue;
}

cudaError_t launch_stream_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs, const Tile* tiles,
                               int ntiles, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (Q == 5 && storage == kF64) return launch_stream_t<5, kF64>(src, dst, runs, tiles, ntiles, s);
  if (Q == 5 && storage == kF32) return launch_stream_t<5, kF32>(src, dst, runs, tiles, ntiles, s);
  if (Q == 5 && storage == kF16S) return launch_stream_t<5, kF16S>(src, dst, runs, tiles, ntiles, s);
  if (Q == 7 && storage == kF64) return launch_stream_t<7, kF64>(src, dst, runs, tiles, ntiles, s);
  if (Q == 7 && storage == kF32) return launch_stream_t<7, kF32>(src, dst, runs, tiles, ntiles, s);
  if (Q == 7 && storage == kF16S) return launch_stream_t<7, kF16S>(src, dst, runs, tiles, ntiles, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbks
