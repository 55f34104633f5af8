// HBM-streaming fused step for large lattices (one launch per step).
//
// A block owns a tile of kTile consecutive sites of one run.  Each thread
// loads VEC consecutive sites of every plane with one 16-byte load (4 sites of
// FP32, 8 of FP16 with half as many threads per block; FP64: two loads), collides
// them in registers and writes f* to a shared-memory copy of the tile that
// also holds c_max post-collision halo sites on each side (computed by a few
// threads from the neighbouring sites, periodic wrap).  After one barrier
// every thread reads the shifted values f*_i(x - c_i) for lane-contiguous
// sites and stores them coalesced.  HBM traffic per site-update: one read and
// one write of the Q populations (plus 2 c_max halo sites per tile).  Scaled
// FP16 storage keeps the tile in shared memory as halves (rounded once, in the
// collision phase) and stores two adjacent sites per thread with one 4-byte store.
#include <type_traits>

#include "lbks_device.cuh"

namespace lbks {

namespace {

constexpr int kTile = 1024;  // sites per block (the host's streaming tiles)
constexpr int kHalo = 4;     // >= c_max, keeps the vector stores aligned

// Sites per thread and threads per block of a storage type: 16-byte loads of each
// plane (FP64 two of them), the same tile of kTile sites.
template <int ST> struct StreamShape {
  static constexpr int kVec = ST == kF16S ? 8 : 4;
  static constexpr int kThreads = kTile / kVec;
};

template <typename T> struct VecLoad;
template <> struct VecLoad<float> {
  static __device__ __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
};
template <> struct VecLoad<double> {
  static __device__ __forceinline__ void load(const double* p, double (&v)[4]) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
template <> struct VecLoad<__half> {
  static __device__ __forceinline__ void load(const __half* p, __half (&v)[8]) {
    const uint4 q = __ldcs(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __half2 a = *reinterpret_cast<const __half2*>(&w[j]);
      v[2 * j] = __low2half(a);
      v[2 * j + 1] = __high2half(a);
    }
  }
};

// Compile-time loop over I = B..E-1 (keeps every plane's speed a constant expression).
template <int B, int E> struct StaticFor {
  template <typename F> __device__ __forceinline__ static void run(F&& fn) {
    if constexpr (B < E) {
      fn(std::integral_constant<int, B>{});
      StaticFor<B + 1, E>::run(fn);
    }
  }
};

// Element type of the shared-memory tile: the storage type for scaled FP16 (the
// value is rounded to it once, where it is computed), else the compute type.
template <int ST>
using TileType = typename std::conditional<ST == kF16S, typename StorageType<ST>::type,
                                           typename StorageType<ST>::compute>::type;

// Aligned 16-byte shared-memory stores of kVec post-collision values of plane i
// (conflict-free; the tile row stride Q*W*sizeof(CT) is a multiple of 16 bytes).
template <int Q>
__device__ __forceinline__ void store4(float* p, const float (&g)[4][Q], int i) {
  *reinterpret_cast<float4*>(p) = make_float4(g[0][i], g[1][i], g[2][i], g[3][i]);
}
template <int Q>
__device__ __forceinline__ void store4(double* p, const double (&g)[4][Q], int i) {
  reinterpret_cast<double2*>(p)[0] = make_double2(g[0][i], g[1][i]);
  reinterpret_cast<double2*>(p)[1] = make_double2(g[2][i], g[3][i]);
}

// Eight scaled FP16 values of plane i, rounded to storage, as two aligned 8-byte stores
// (the tile column kHalo + 8 t is 8-byte aligned).
template <int Q>
__device__ __forceinline__ void store4(__half* p, const float (&g)[8][Q], int i, float inv_scale) {
  __half o[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) from_compute(g[u][i], inv_scale, &o[u]);
  uint32_t w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __half2 a = __halves2half2(o[2 * j], o[2 * j + 1]);
    w[j] = *reinterpret_cast<const uint32_t*>(&a);
  }
  reinterpret_cast<uint2*>(p)[0] = make_uint2(w[0], w[1]);
  reinterpret_cast<uint2*>(p)[1] = make_uint2(w[2], w[3]);
}

template <int Q, int ST>
__device__ __forceinline__ void stream_step(Arena src, Arena dst, const RunDesc* __restrict__ runs,
                                            const Tile* __restrict__ tiles) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  using ET = TileType<ST>;
  constexpr bool kHalf = ST == kF16S;
  constexpr int kVec = StreamShape<ST>::kVec;
  constexpr int kStreamThreads = StreamShape<ST>::kThreads;
  constexpr int C = cmax_of(Q);
  constexpr int W = kTile + 2 * kHalo;
  static_assert(W % 8 == 0, "tile rows of halves must start 16-byte aligned");
  static_assert(C < kHalo, "the paired FP16 reads reach column kHalo - c_max - 1");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ET* sm = reinterpret_cast<ET*>(smem_raw);  // [Q][W], tile site k at column kHalo + k
  // one tile value, rounded to the tile's element type
  auto put = [&](ET* p, CT v, CT inv_scale) {
    if constexpr (kHalf) from_compute(v, inv_scale, p);
    else *p = v;
  };

  wait_prior_grid();
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
          VecLoad<T>::load(fs + (int64_t)i * src.plane + x0 + k0, v);
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
        for (int i = 0; i < Q; ++i) {
          if constexpr (kHalf) store4(sm + i * W + kHalo + k0, g, i, k.inv_scale);
          else store4(sm + i * W + kHalo + k0, g, i);
        }
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i)
#pragma unroll
          for (int u = 0; u < kVec; ++u)
            if (k0 + u < len) put(&sm[i * W + kHalo + k0 + u], g[u][i], k.inv_scale);
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
      for (int i = 0; i < Q; ++i) put(&sm[i * W + col], g[i], k.inv_scale);
    }
  }
  __syncthreads();
  // Phase 2: pull f*_i(x - c_i), lane-contiguous sites, coalesced stores.
  if constexpr (kHalf) {
    // Sites kk .. kk + 7 (kk = 8 t) of plane i sit at tile columns e0 .. e0 + 7,
    // e0 = i W + kHalo + kk - c_i, whose offset from 8 t is a compile-time constant: the
    // eight halves come from one 16-byte, two 8-byte or four 4-byte shared loads (e0
    // a multiple of 8, 4 or 2), or, for odd c_i, from five words, each output word the
    // high half of one and the low half of the next; one 16-byte streaming store writes
    // them.  Columns read stay in [kHalo - 4, kHalo + kTile + 3] = [0, W) of the row
    // (c_max <= 3 <= kHalo - 1); values read past a ragged tile's end or its halo are
    // not stored.  Rows, run offsets, the plane stride and tile starts are multiples of
    // 8 halves, so the 16-byte global stores are aligned.
    static_assert(W % 8 == 0, "tile rows of halves start 16-byte aligned");
    const int kk = kVec * threadIdx.x;
    if (kk < len) {
      StaticFor<0, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int off = i * W + kHalo - speed(i);  // e0 = off + kk
        const unsigned char* row = smem_raw + (size_t)(off & ~1) * sizeof(__half) + (size_t)kk * sizeof(__half);
        uint32_t w[4];
        if constexpr (off % 8 == 0) {
          const uint4 v = *reinterpret_cast<const uint4*>(row);
          w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
        } else if constexpr (off % 4 == 0) {
          const uint2 a = reinterpret_cast<const uint2*>(row)[0], b = reinterpret_cast<const uint2*>(row)[1];
          w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
        } else if constexpr (off % 2 == 0) {
#pragma unroll
          for (int j = 0; j < 4; ++j) w[j] = reinterpret_cast<const uint32_t*>(row)[j];
        } else {
          uint32_t x[5];
#pragma unroll
          for (int j = 0; j < 5; ++j) x[j] = reinterpret_cast<const uint32_t*>(row)[j];
#pragma unroll
          for (int j = 0; j < 4; ++j) w[j] = __byte_perm(x[j], x[j + 1], 0x5432);
        }
        T* p = fd + (int64_t)i * dst.plane + x0 + kk;
        if (kk + kVec <= len) {
          __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
        } else {
#pragma unroll
          for (int j = 0; j < kVec; ++j)
            if (kk + j < len) __stcs(p + j, __ushort_as_half((unsigned short)((w[j >> 1] >> (16 * (j & 1))) & 0xffffu)));
        }
      });
    }
  } else {
#pragma unroll
    for (int u = 0; u < kVec; ++u) {
      const int kk = threadIdx.x + u * kStreamThreads;
      if (kk < len) {
#pragma unroll
        for (int i = 0; i < Q; ++i) __stcs(fd + (int64_t)i * dst.plane + x0 + kk, sm[i * W + kHalo + kk - speed(i)]);
      }
    }
  }
}

template <int Q, int ST>
__global__ void __launch_bounds__(StreamShape<ST>::kThreads) stream_step_kernel(Arena src, Arena dst,
                                                                                 const RunDesc* __restrict__ runs,
                                                                                 const Tile* __restrict__ tiles) {
  stream_step<Q, ST>(src, dst, runs, tiles);
}

// Scaled FP16: registers for 8 blocks (32 warps) per SM.  The kernel is bound by load
// latency; at 64 registers a few values spill, and the occupancy outweighs them (5.61 ->
// 5.93 TB/s on the 2^24-site lattice).  (An explicit minimum for FP32 and FP64 changes
// the compiler's choice even where it does not bind: FP32 took 80 registers instead of
// 48 with a minimum of one block and ran 8 % slower.)
template <int Q>
__global__ void __launch_bounds__(StreamShape<kF16S>::kThreads, 8) stream_step_kernel_f16(Arena src, Arena dst,
                                                                                       const RunDesc* __restrict__ runs,
                                                                                       const Tile* __restrict__ tiles) {
  stream_step<Q, kF16S>(src, dst, runs, tiles);
}

template <int Q, int ST>
size_t stream_smem() {
  return sizeof(TileType<ST>) * Q * (kTile + 2 * kHalo);
}

template <int Q, int ST>
cudaError_t prepare_stream_t() {
  if constexpr (ST == kF16S)
    return cudaFuncSetAttribute(stream_step_kernel_f16<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stream_smem<Q, ST>());
  else
    return cudaFuncSetAttribute(stream_step_kernel<Q, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stream_smem<Q, ST>());
}

template <int Q, int ST>
cudaError_t launch_stream_t(Arena src, Arena dst, const RunDesc* runs, const Tile* tiles, int ntiles, cudaStream_t s) {
  if constexpr (ST == kF16S)
    return launch_early(stream_step_kernel_f16<Q>, ntiles, StreamShape<ST>::kThreads, stream_smem<Q, ST>(), s, src, dst,
                        runs, tiles);
  else
    return launch_early(stream_step_kernel<Q, ST>, ntiles, StreamShape<ST>::kThreads, stream_smem<Q, ST>(), s, src, dst,
                        runs, tiles);
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
