// Register-resident, temporally blocked fused step for ensembles of lattices
// (one persistent launch runs ksteps steps of every lattice it is given).
//
// Work unit ("piece"): a whole periodic lattice (ring) or, for lattices larger
// than one block holds, a stretch of one with c_max * ksteps halo sites on
// each side (segment).  A piece occupies V consecutive threads of a block;
// thread j holds S or S-1 consecutive sites (all Q planes) in registers, so
// any lattice length n with V (S-1) < n <= V S is held exactly.  Pieces of
// different runs (different N, tau, alpha, beta) are packed into the same
// block by the host ("bundle").
//
// One step of Eq. LB_equation_ordinary:
//  A. per held site: s_g = sum_i g_i, rho = rhobar + s_g, rho^2;
//  B. per plane i >= 1, the post-collision value of every site is written
//     straight into the register of the site it streams to (c_i > 0: sites
//     visited from the last one down, c_i < 0: from the first one up, so the
//     destination register's old value has already been used); the c_i values
//     that leave the thread go to shared memory;  g_0 = s_g - sum of the others
//     (mass conservation; the same arithmetic, in the same order, as collide());
//  C. one barrier, then the values entering from the neighbour thread are read
//     (the neighbour of a piece's last thread is its first: periodic wrap).
// For a segment the wrap injects unrelated values at its two ends; they travel
// at most c_max sites per step and never reach the stored middle.
//
// Loads and stores at the launch edges go through shared memory so that
// global accesses are coalesced (consecutive threads, consecutive sites).
//
// Blocks take bundles from a global counter (atomicAdd), largest first, until
// the queue is empty: a persistent grid with a ragged work queue.  No block
// waits on another.
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

// Shared memory per thread (elements): the exchange buffers
// [2 parities][2 directions][NX], reused at the launch edges as a staging area
// of Q planes x S sites.
__host__ __device__ constexpr int exchange_elems(int Q) { return 4 * ((Q - 1) / 2) * ((Q - 1) / 2 + 1) / 2; }
__host__ __device__ constexpr int smem_elems_per_thread(int Q, int S) {
  return exchange_elems(Q) > Q * S ? exchange_elems(Q) : Q * S;
}

template <int Q, int ST, int S>
__global__ void __launch_bounds__(ResidentCfg<ST, S>::kMaxThreads, 1) resident_kernel(const ResidentArgs a) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  constexpr int C = cmax_of(Q);
  constexpr int NX = C * (C + 1) / 2;  // values leaving a thread per direction per step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  CT* const xbase = reinterpret_cast<CT*>(smem_raw);  // [parity][R|L][NX][NT]
  CT* const stage = xbase;                             // [NT * S] at the launch edges
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
    int j = 0, V = 1, start = 0, left = t, right = t;
    Piece pc{};
    int64_t N = 1, x_first = 0;
    const T* fs = nullptr;
    T* fd = nullptr;
    if (active) {
      pc = a.pieces[pidx];
      const RunDesc& d = a.runs[pc.run];
      k = load_coef<CT, Q>(d);
      N = d.N;
      j = t - pc.t0;
      V = pc.nthr;
      const int mfull = pc.n - V * (S - 1);  // threads holding S sites; the rest hold S-1
      full = j < mfull;
      start = full ? j * S : mfull * S + (j - mfull) * (S - 1);
      left = pc.t0 + (j == 0 ? V - 1 : j - 1);
      right = pc.t0 + (j == V - 1 ? 0 : j + 1);
      x_first = (pc.x0 + j) % N;
      fs = static_cast<const T*>(a.src.f) + d.off;
      fd = static_cast<T*>(a.dst.f) + d.off;
    }

    // ---- load: coalesced global reads of all planes into the staging area, then registers
    const int sbase = pc.t0 * S;  // this piece's sites in each staged plane
    if (active) {
      int64_t x = x_first;
      for (int li = j; li < pc.n; li += V) {
#pragma unroll
        for (int i = 0; i < Q; ++i) stage[i * NT * S + sbase + li] = to_compute(fs[(int64_t)i * a.src.plane + x], k.scale);
        x += V;
        while (x >= N) x -= N;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s) f[i][s] = (s < S - 1 || full) ? stage[i * NT * S + sbase + start + s] : CT(0);
    }
    __syncthreads();

    for (int step = 0; step < a.ksteps; ++step) {
      CT* const xr = xbase + (step & 1) * 2 * NX * NT;  // right-moving values leaving threads
      CT* const xl = xr + NX * NT;                       // left-moving values leaving threads
      if (active) {
        // A. per-site sums
        CT acc[S], rho[S], rho2[S], tt[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          CT sg = f[0][s];
#pragma unroll
          for (int i = 1; i < Q; ++i) sg = add_rn(sg, f[i][s]);
          acc[s] = sg;
          rho[s] = add_rn(k.rhobar, sg);
          rho2[s] = mul_rn(rho[s], rho[s]);
        }
        // B. plane by plane: collide, write to the destination site's register or send.
        StaticFor<1, Q>::run([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          constexpr int c = speed(i);
          constexpr int kk = c > 0 ? c : -c;
          constexpr int base = kk * (kk - 1) / 2;
          if constexpr (c > 0) {
#pragma unroll
            for (int s = S - 1; s >= 0; --s) {
              tt[s] = mul_rn(rho[s], k.a[i]);  // shared with the -c plane that follows
              const CT v = post_collision(k.r, f[i][s], rho[s], rho2[s], k.b[i], tt[s]);
              acc[s] = add_rn(acc[s], -v);
              if (s + kk <= S - 2) {
                f[i][s + kk] = v;
              } else if (s + kk == S - 1) {
                if (full) f[i][S - 1] = v;
                else xr[base * NT + t] = v;
              } else if (s <= S - 2) {
                xr[(base + (full ? s + kk - S : s + kk - S + 1)) * NT + t] = v;
              } else if (full) {  // s == S - 1 holds a site only in threads with S sites
                xr[(base + s + kk - S) * NT + t] = v;
              }
            }
          } else {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const CT v = post_collision(k.r, f[i][s], rho[s], rho2[s], k.b[i], tt[s]);
              acc[s] = add_rn(acc[s], -v);
              if (s >= kk) f[i][s - kk] = v;
              else xl[(base + s) * NT + t] = v;
            }
          }
        });
#pragma unroll
        for (int s = 0; s < S; ++s) f[0][s] = acc[s];
      }
      __syncthreads();
      if (active) {
        // C. values entering from the neighbours
        StaticFor<1, Q>::run([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          constexpr int c = speed(i);
          constexpr int kk = c > 0 ? c : -c;
          constexpr int base = kk * (kk - 1) / 2;
          if constexpr (c > 0) {
#pragma unroll
            for (int jj = 0; jj < kk; ++jj) f[i][jj] = xr[(base + jj) * NT + left];
          } else {
            // threads with S sites fill slots S-kk .. S-1, threads with S-1 sites S-1-kk .. S-2
#pragma unroll
            for (int jj = 0; jj < kk; ++jj) {
              const CT v = xl[(base + jj) * NT + right];
              if (full) f[i][S - kk + jj] = v;
              else f[i][S - 1 - kk + jj] = v;
            }
          }
        });
      }
    }
    __syncthreads();  // the last step's exchange reads finish before the staging area is reused

    // ---- store: registers into the staging area, then coalesced global writes of all planes
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s)
          if (s < S - 1 || full) stage[i * NT * S + sbase + start + s] = f[i][s];
    }
    __syncthreads();
    if (active) {
      int64_t x = x_first;
      for (int li = j; li < pc.n; li += V) {
        if (li >= pc.st_lo && li < pc.st_hi) {
#pragma unroll
          for (int i = 0; i < Q; ++i)
            from_compute(stage[i * NT * S + sbase + li], k.inv_scale, fd + (int64_t)i * a.dst.plane + x);
        }
        x += V;
        while (x >= N) x -= N;
      }
    }
    __syncthreads();
  }
}

template <int Q, int ST, int S>
size_t smem_bytes_t(int NT) {
  using CT = typename StorageType<ST>::compute;
  return sizeof(CT) * (size_t)smem_elems_per_thread(Q, S) * (size_t)NT;
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
