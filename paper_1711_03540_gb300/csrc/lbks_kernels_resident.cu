// Register-resident, temporally blocked fused step for ensembles of lattices
// (one persistent launch runs ksteps steps of every lattice of the batch).
//
// Work unit ("piece"): a whole periodic lattice (ring) or, for lattices larger
// than one block holds, a stretch of one with c_max * ksteps halo sites on
// each side (segment).  A piece occupies V consecutive threads of a block;
// thread j holds S or S-1 consecutive sites (all Q planes) in registers, so
// any lattice length n with V (S-1) < n <= V S is held exactly.  Pieces of
// different runs (different N, tau, alpha, beta) are packed into the same
// block by the host ("bundle").
//
// One step = collide every held site in registers (Eq. LB_equation_ordinary),
// then shift plane i by c_i: inside a thread by register renaming, across
// threads by writing the c_i values that leave a thread into shared memory,
// one barrier, and reading the ones that enter from the neighbour thread
// (the neighbour of the piece's last thread is its first: periodic wrap).
// For a segment the wrap injects unrelated values at its two ends; they
// travel at most c_max sites per step and never reach the stored middle.
//
// Blocks take bundles from a global counter (atomicAdd), largest first, until
// the queue is empty: a persistent grid with a ragged work queue.  There are no
// waits on other blocks.
#include <type_traits>

#include "lbks_device.cuh"

namespace lbks {

namespace {

template <int ST, int S> struct ResidentCfg {
  // Upper bound of threads per block; sets the register budget per thread.
  static constexpr int kMaxThreads = (ST == kF64) ? 256 : (S <= 8 ? 512 : (S <= 12 ? 384 : 256));
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

struct ResidentArgs {
  Arena src, dst;
  const RunDesc* runs;
  const Piece* pieces;
  const int2* bundles;
  int nbundles;
  int* queue;
  int ksteps;
};

template <int Q, int ST, int S>
__global__ void __launch_bounds__(ResidentCfg<ST, S>::kMaxThreads, 1) resident_kernel(const ResidentArgs a) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  constexpr int C = cmax_of(Q);
  constexpr int NX = C * (C + 1) / 2;  // values leaving a thread per direction per step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  CT* xR = reinterpret_cast<CT*>(smem_raw);  // [2 parities][NX][NT]: right-moving values
  CT* xL = xR + 2 * NX * NT;                  // [2 parities][NX][NT]: left-moving values
  __shared__ int s_bundle;
  const int t = threadIdx.x;

  for (;;) {
    if (t == 0) s_bundle = atomicAdd(a.queue, 1);
    __syncthreads();
    const int b = s_bundle;
    __syncthreads();
    if (b >= a.nbundles) break;
    const int2 bd = a.bundles[b];

    int pidx = -1;
    for (int p = bd.x; p < bd.x + bd.y; ++p) {
      const int t0 = a.pieces[p].t0;
      if (t >= t0 && t < t0 + a.pieces[p].nthr) { pidx = p; break; }
    }
    const bool active = pidx >= 0;

    CT f[Q][S];
    Coef<CT, Q> k;
    bool full = true;
    int start = 0, left = t, right = t;
    Piece pc;
    int64_t N = 1;
    if (active) {
      pc = a.pieces[pidx];
      const RunDesc& d = a.runs[pc.run];
      k = load_coef<CT, Q>(d);
      N = d.N;
      const int j = t - pc.t0;
      const int V = pc.nthr;
      const int mfull = pc.n - V * (S - 1);  // threads holding S sites; the rest hold S-1
      full = j < mfull;
      start = full ? j * S : mfull * S + (j - mfull) * (S - 1);
      left = pc.t0 + (j == 0 ? V - 1 : j - 1);
      right = pc.t0 + (j == V - 1 ? 0 : j + 1);
      const T* fs = static_cast<const T*>(a.src.f) + d.off;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (s < S - 1 || full) {
          const int64_t x = (pc.x0 + start + s) % N;
#pragma unroll
          for (int i = 0; i < Q; ++i) f[i][s] = to_compute(fs[(int64_t)i * a.src.plane + x], k.scale);
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) f[i][s] = CT(0);
        }
      }
    }

    for (int step = 0; step < a.ksteps; ++step) {
      CT* xr = xR + (step & 1) * NX * NT;
      CT* xl = xL + (step & 1) * NX * NT;
      if (active) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          CT g[Q];
#pragma unroll
          for (int i = 0; i < Q; ++i) g[i] = f[i][s];
          collide<Q, CT>(g, k);
#pragma unroll
          for (int i = 0; i < Q; ++i) f[i][s] = g[i];
        }
        // Values leaving the thread: the last c (c > 0) or first |c| (c < 0) held sites.
        StaticFor<1, Q>::run([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          constexpr int c = speed(i);
          constexpr int kk = c > 0 ? c : -c;
          constexpr int base = kk * (kk - 1) / 2;
#pragma unroll
          for (int jj = 0; jj < kk; ++jj) {
            if constexpr (c > 0) xr[(base + jj) * NT + t] = full ? f[i][S - kk + jj] : f[i][S - 1 - kk + jj];
            else xl[(base + jj) * NT + t] = f[i][jj];
          }
        });
      }
      __syncthreads();
      if (active) {
        StaticFor<1, Q>::run([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          constexpr int c = speed(i);
          constexpr int kk = c > 0 ? c : -c;
          constexpr int base = kk * (kk - 1) / 2;
          CT rv[kk];
#pragma unroll
          for (int jj = 0; jj < kk; ++jj)
            rv[jj] = (c > 0) ? xr[(base + jj) * NT + left] : xl[(base + jj) * NT + right];
          if constexpr (c > 0) {
            // f_i(x + c) <- f*_i(x): slot s takes slot s - c, the first c slots come from the left thread.
#pragma unroll
            for (int s = S - 1; s >= kk; --s) f[i][s] = f[i][s - kk];
#pragma unroll
            for (int s = 0; s < kk; ++s) f[i][s] = rv[s];
          } else {
            // c < 0: slot s takes slot s + |c|; the last |c| held slots come from the right thread.
#pragma unroll
            for (int s = 0; s < S; ++s) {
              if (s + kk < S - 1) {
                f[i][s] = f[i][s + kk];
              } else if (s + kk == S - 1) {
                f[i][s] = full ? f[i][S - 1] : rv[0];
              } else {
                const int jf = s - (S - kk);  // source index when the thread holds S sites
                const int js = jf + 1;        // ... and when it holds S - 1 (slot S-1 unused then)
                f[i][s] = full ? rv[jf] : (js < kk ? rv[js < kk ? js : 0] : CT(0));
              }
            }
          }
        });
      }
    }

    if (active) {
      const RunDesc& d = a.runs[pc.run];
      T* fd = static_cast<T*>(a.dst.f) + d.off;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int li = start + s;
        if ((s < S - 1 || full) && li >= pc.st_lo && li < pc.st_hi) {
          const int64_t x = (pc.x0 + li) % N;
#pragma unroll
          for (int i = 0; i < Q; ++i) from_compute(f[i][s], k.inv_scale, fd + (int64_t)i * a.dst.plane + x);
        }
      }
    }
  }
}

template <int Q, int ST, int S>
size_t smem_bytes_t(int NT) {
  using CT = typename StorageType<ST>::compute;
  constexpr int C = cmax_of(Q);
  return sizeof(CT) * 2 * 2 * (C * (C + 1) / 2) * (size_t)NT;
}

template <int Q, int ST, int S>
cudaError_t prepare_t(int NT, int* blocks_per_sm) {
  if (NT > ResidentCfg<ST, S>::kMaxThreads || NT % 32 != 0) return cudaErrorInvalidValue;
  const size_t smem = smem_bytes_t<Q, ST, S>(NT);
  cudaError_t e = cudaFuncSetAttribute(resident_kernel<Q, ST, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, resident_kernel<Q, ST, S>, NT, smem);
}

template <int Q, int ST, int S>
cudaError_t launch_t(const ResidentLaunch& L, cudaStream_t s) {
  ResidentArgs a{L.src, L.dst, L.runs, L.pieces, L.bundles, L.nbundles, L.queue, L.ksteps};
  resident_kernel<Q, ST, S><<<L.grid, L.NT, smem_bytes_t<Q, ST, S>(L.NT), s>>>(a);
  return cudaGetLastError();
}

#define LBKS_RESIDENT_CASES(Q_, ST_, OP)                                              \
  if (Q == Q_ && storage == ST_) {                                                    \
    constexpr int Qc = Q_, STc = ST_;                                                 \
    switch (S) {                                                                      \
      case 4: { constexpr int Sc = 4; OP; }                                           \
      case 6: { constexpr int Sc = 6; OP; }                                           \
      case 8: { constexpr int Sc = 8; OP; }                                           \
      case 12: if constexpr (STc != kF64) { constexpr int Sc = 12; OP; } break;       \
      case 16: if constexpr (STc != kF64) { constexpr int Sc = 16; OP; } break;       \
      default: break;                                                                 \
    }                                                                                 \
  }

#define LBKS_RESIDENT_DISPATCH(OP)       \
  LBKS_RESIDENT_CASES(5, kF64, OP)       \
  LBKS_RESIDENT_CASES(5, kF32, OP)       \
  LBKS_RESIDENT_CASES(5, kF16S, OP)      \
  LBKS_RESIDENT_CASES(7, kF64, OP)       \
  LBKS_RESIDENT_CASES(7, kF32, OP)       \
  LBKS_RESIDENT_CASES(7, kF16S, OP)

}  // namespace

bool resident_supported(int Q, int storage, int S, int NT) {
  if (Q != 5 && Q != 7) return false;
  if (storage != kF64 && storage != kF32 && storage != kF16S) return false;
  if (S != 4 && S != 6 && S != 8 && S != 12 && S != 16) return false;
  if (storage == kF64 && S > 8) return false;
  const int maxt = storage == kF64 ? 256 : (S <= 8 ? 512 : (S <= 12 ? 384 : 256));
  return NT >= 32 && NT <= maxt && NT % 32 == 0;
}

size_t resident_smem_bytes(int Q, int storage, int NT) {
  const int C = (Q - 1) / 2;
  const size_t es = storage == kF64 ? 8 : 4;
  return es * 2 * 2 * (C * (C + 1) / 2) * (size_t)NT;
}

cudaError_t resident_prepare(int Q, int storage, int S, int NT, int* blocks_per_sm) {
  if (!resident_supported(Q, storage, S, NT)) return cudaErrorInvalidValue;
  LBKS_RESIDENT_DISPATCH(return (prepare_t<Qc, STc, Sc>(NT, blocks_per_sm)));
  return cudaErrorInvalidValue;
}

cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s) {
  const int Q = L.Q, storage = L.storage, S = L.S;
  if (!resident_supported(Q, storage, S, L.NT)) return cudaErrorInvalidValue;
  if (L.nbundles == 0 || L.grid == 0) return cudaSuccess;
  LBKS_RESIDENT_DISPATCH(return (launch_t<Qc, STc, Sc>(L, s)));
  return cudaErrorInvalidValue;
}

}  // namespace lbks
