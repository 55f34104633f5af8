// Kernels of the tau = 1 collapse (lbks_collapse.cuh): initialisation of the one
// stored plane and the streaming stencil step (one launch per step; HBM-bound:
// one read and one write of the plane per site-update, the halo from the tile's
// neighbours through shared memory).
#include "lbks_collapse.cuh"

namespace lbks {

namespace {

constexpr int kCollapseThreads = 256;
constexpr int kCollapseTile = 1024;  // sites per tile (the streaming tiles of the handle)

// delta(x) = rho0(x) - rhobar over one tile of nodes; with reservoir ends, nodes
// x <= 0 and x >= N - 1 (and the c_max ghost nodes beyond) hold the end values.
template <int ST>
__global__ void __launch_bounds__(kCollapseThreads) collapse_init_kernel(Arena dst, const RunDesc* __restrict__ runs,
                                                                         const Tile* __restrict__ tiles,
                                                                         const double* __restrict__ rho0,
                                                                         const int64_t* __restrict__ rho_off) {
  using T = typename StorageType<ST>::type;
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
    const int64_t x = (int64_t)tl.x0 + k;
    double v;
    if (d.reservoir && x <= 0) v = d.rho_left;
    else if (d.reservoir && x >= d.N - 1) v = d.rho_right;
    else v = rho0[rho_off[tl.run] + x];
    static_cast<T*>(dst.f)[d.off + x] = static_cast<T>(__dsub_rn(v, d.rhobar));
  }
}

// One collapsed step over one tile of a run: nodes [x0, x0 + len) from nodes
// [x0 - C, x0 + len + C) (periodic wrap, or the reservoir ghosts).  Reservoir end
// nodes are not written: both arenas hold their fixed values.
template <int C, int ST>
__global__ void __launch_bounds__(kCollapseThreads) collapse_step_kernel(Arena src, Arena dst,
                                                                         const RunDesc* __restrict__ runs,
                                                                         const Tile* __restrict__ tiles) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  __shared__ CT buf[kCollapseTile + 2 * C];
  wait_prior_grid();
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  const T* fs = static_cast<const T*>(src.f) + d.off;
  T* fd = static_cast<T*>(dst.f) + d.off;
  const int t = threadIdx.x;
  constexpr int kPer = kCollapseTile / kCollapseThreads;
  CT v[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {  // all loads in flight before the shared-memory stores
    const int k = t + j * kCollapseThreads;
    v[j] = k < tl.len ? static_cast<CT>(__ldcs(fs + tl.x0 + k)) : CT(0);
  }
  if (t < 2 * C) {  // halo: C nodes on each side of the tile
    const int64_t x = t < C ? (int64_t)tl.x0 - C + t : (int64_t)tl.x0 + tl.len + (t - C);
    const int64_t y = d.reservoir ? x : wrap_site(x, d.N);
    buf[t < C ? t : C + tl.len + (t - C)] = static_cast<CT>(fs[y]);
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = t + j * kCollapseThreads;
    if (k < tl.len) buf[C + k] = v[j];
  }
  __syncthreads();
  const CollapseCoef<CT, C> kc = load_collapse_coef<CT, C>(d);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = t + j * kCollapseThreads;
    if (k >= tl.len) continue;
    const int64_t x = (int64_t)tl.x0 + k;
    if (d.reservoir && (x == 0 || x == d.N - 1)) continue;
    CT dl[C + 1], dr[C + 1];
#pragma unroll
    for (int c = 1; c <= C; ++c) {
      dl[c] = buf[C + k - c];
      dr[c] = buf[C + k + c];
    }
    dl[0] = dr[0] = CT(0);
    __stcs(fd + x, static_cast<T>(collapse_site<CT, C>(buf[C + k], dl, dr, kc)));
  }
}

}  // namespace

int collapse_tile_sites() { return kCollapseTile; }

cudaError_t launch_collapse_init(int storage, Arena dst, const RunDesc* runs, const Tile* tiles, int ntiles,
                                 const double* rho0, const int64_t* rho_off, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (storage == kF64) collapse_init_kernel<kF64><<<ntiles, kCollapseThreads, 0, s>>>(dst, runs, tiles, rho0, rho_off);
  else if (storage == kF32) collapse_init_kernel<kF32><<<ntiles, kCollapseThreads, 0, s>>>(dst, runs, tiles, rho0, rho_off);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_collapse_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs, const Tile* tiles,
                                 int ntiles, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (Q == 5 && storage == kF64) return launch_early(collapse_step_kernel<2, kF64>, ntiles, kCollapseThreads, 0, s, src, dst, runs, tiles);
  if (Q == 5 && storage == kF32) return launch_early(collapse_step_kernel<2, kF32>, ntiles, kCollapseThreads, 0, s, src, dst, runs, tiles);
  if (Q == 7 && storage == kF64) return launch_early(collapse_step_kernel<3, kF64>, ntiles, kCollapseThreads, 0, s, src, dst, runs, tiles);
  if (Q == 7 && storage == kF32) return launch_early(collapse_step_kernel<3, kF32>, ntiles, kCollapseThreads, 0, s, src, dst, runs, tiles);
  return cudaErrorInvalidValue;
}

}  // namespace lbks

// ---------------------------------------------------------------- register-resident

namespace lbks {

namespace {

// Register-resident collapsed step, many steps per launch, for whole periodic
// lattices (rings) and stretches of longer ones with c_max * ksteps halo sites per
// side (segments), with the piece / bundle / work-queue layout of the resident LB
// kernel: thread j of a piece holds S or S-1 consecutive sites of rho - rhobar in
// registers, as e[C + s], with C halo slots on each side.  One step:
//  1. the thread's first C values go to the left-going exchange row and its last
//     C values to the right-going one (shared memory, double-buffered by parity);
//  2. one block barrier;
//  3. the left halo e[0 .. C-1] is read from the left neighbour thread's last C
//     values and the right halo from the right neighbour's first C (the
//     neighbour of a piece's last thread is its first: periodic wrap);
//  4. every held site takes collapse_site() of its window.
constexpr int kCRThreads = 512;  // upper bound of threads per block

struct CollapseResidentArgs {
  Arena src, dst;
  const RunDesc* runs;
  const Piece* pieces;
  const int2* bundles;
  int nbundles;
  int* queue;
  int ksteps;
};

template <int C, int ST, int S>
__global__ void __launch_bounds__(kCRThreads, 1) collapse_resident_kernel(const CollapseResidentArgs a) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  CT* const stage = reinterpret_cast<CT*>(smem_raw);  // [NT * S] at the launch edges
  // [parity][R|L][C][kCRThreads]: a compile-time row length, so that every exchange
  // access is a base address plus an immediate offset
  constexpr int XS = kCRThreads;
  CT* const xbase = stage + NT * S;
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

    CT e[S + 2 * C];
    CollapseCoef<CT, C> k;
    // where the thread's sites sit (computed before the load and again, from the piece
    // read anew, before the store, so that none of it is held through the steps)
    struct Geom {
      int64_t N, x_first;
      int j, V, start, sbase;
      bool full;
    };
    auto geom = [&](const Piece& pc, int64_t N) {
      Geom G;
      G.N = N;
      G.j = t - pc.t0;
      G.V = pc.nthr;
      const int mfull = pc.n - G.V * (S - 1);  // threads holding S sites; the rest hold S-1
      G.full = G.j < mfull;
      G.start = G.full ? G.j * S : mfull * S + (G.j - mfull) * (S - 1);
      G.x_first = (pc.x0 + G.j) % N;
      G.sbase = pc.t0 * S;
      return G;
    };
    bool full = true;
    int left = t, right = t;
    Geom G{};
    int n = 0;
    const T* fs = nullptr;
    if (active) {
      const Piece pc = a.pieces[pidx];
      const RunDesc& d = a.runs[pc.run];
      k = load_collapse_coef<CT, C>(d);
      G = geom(pc, d.N);
      full = G.full;
      n = pc.n;
      left = pc.t0 + (G.j == 0 ? G.V - 1 : G.j - 1);
      right = pc.t0 + (G.j == G.V - 1 ? 0 : G.j + 1);
      fs = static_cast<const T*>(a.src.f) + d.off;
    }

    // ---- load: coalesced global reads into the staging area, then registers
    if (active) {
      int64_t x = G.x_first;
      for (int li = G.j; li < n; li += G.V) {
        stage[G.sbase + li] = static_cast<CT>(fs[x]);
        x += G.V;
        while (x >= G.N) x -= G.N;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int s = 0; s < S; ++s) e[C + s] = (s < S - 1 || full) ? stage[G.sbase + G.start + s] : CT(0);
    }
    __syncthreads();

    for (int step = 0; step < a.ksteps; ++step) {
      CT* const xr = xbase + (step & 1) * 2 * C * XS;  // a thread's last C values (read by its right neighbour)
      CT* const xl = xr + C * XS;                       // its first C values (read by its left neighbour)
      if (active) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          xl[c * XS + t] = e[C + c];
          xr[c * XS + t] = full ? e[S + c] : e[S - 1 + c];  // own sites end at C + S - 1 or C + S - 2
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          e[c] = xr[c * XS + left];
          const CT v = xl[c * XS + right];
          if (full) e[C + S + c] = v;
          else e[C + S - 1 + c] = v;
        }
        CT nw[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          CT dl[C + 1], dr[C + 1];
          dl[0] = dr[0] = CT(0);
#pragma unroll
          for (int c = 1; c <= C; ++c) {
            dl[c] = e[C + s - c];
            dr[c] = e[C + s + c];
          }
          nw[s] = collapse_site<CT, C>(e[C + s], dl, dr, k);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) e[C + s] = nw[s];
      }
    }

    // ---- store: registers into the staging area, then coalesced global writes
    Piece pc{};
    if (active) {
      pc = a.pieces[pidx];  // read anew (after the barriers of the steps)
      G = geom(pc, a.runs[pc.run].N);
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (s < S - 1 || G.full) stage[G.sbase + G.start + s] = e[C + s];
    }
    __syncthreads();
    if (active) {
      T* const fd = static_cast<T*>(a.dst.f) + a.runs[pc.run].off;
      int64_t x = G.x_first;
      for (int li = G.j; li < pc.n; li += G.V) {
        if (li >= pc.st_lo && li < pc.st_hi) fd[x] = static_cast<T>(stage[G.sbase + li]);
        x += G.V;
        while (x >= G.N) x -= G.N;
      }
    }
    __syncthreads();
  }
}

template <int C, int ST, int S>
size_t cr_smem_bytes(int NT) {
  using CT = typename StorageType<ST>::compute;
  return sizeof(CT) * ((size_t)NT * S + (size_t)4 * C * kCRThreads);
}

#define LBKS_COLLAPSE_CASES(OP)                                                         \
  if (Q == 5 && storage == kF64) { constexpr int Cc = 2, STc = kF64; LBKS_CR_S(OP) }    \
  if (Q == 5 && storage == kF32) { constexpr int Cc = 2, STc = kF32; LBKS_CR_S(OP) }    \
  if (Q == 7 && storage == kF64) { constexpr int Cc = 3, STc = kF64; LBKS_CR_S(OP) }    \
  if (Q == 7 && storage == kF32) { constexpr int Cc = 3, STc = kF32; LBKS_CR_S(OP) }
#define LBKS_CR_S(OP)                                  \
  switch (S) {                                         \
    case 8: { constexpr int Sc = 8; OP; }              \
    case 16: { constexpr int Sc = 16; OP; }            \
    case 32: if constexpr (STc != kF64) { constexpr int Sc = 32; OP; } break; \
    default: break;                                    \
  }

template <int C, int ST, int S>
cudaError_t cr_prepare_t(int NT, int* blocks_per_sm) {
  // the opt-in covers the largest block (kCRThreads), so that preparing a smaller tiling
  // later never lowers it under a larger one already prepared
  const size_t smem = cr_smem_bytes<C, ST, S>(NT);
  cudaError_t e = cudaFuncSetAttribute(collapse_resident_kernel<C, ST, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)cr_smem_bytes<C, ST, S>(kCRThreads));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, collapse_resident_kernel<C, ST, S>, NT, smem);
}

template <int C, int ST, int S>
cudaError_t cr_launch_t(const ResidentLaunch& L, cudaStream_t s) {
  const CollapseResidentArgs a{L.src, L.dst, L.runs, L.pieces, L.bundles, L.nbundles, L.queue, L.ksteps};
  collapse_resident_kernel<C, ST, S><<<L.grid, L.NT, cr_smem_bytes<C, ST, S>(L.NT), s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool collapse_resident_supported(int Q, int storage, int S, int NT) {
  if (Q != 5 && Q != 7) return false;
  if (storage != kF64 && storage != kF32) return false;
  if (S != 8 && S != 16 && S != 32) return false;
  if (storage == kF64 && S > 16) return false;  // 128 registers per thread at 512 threads
  return NT >= 32 && NT <= kCRThreads && NT % 32 == 0;
}

cudaError_t collapse_resident_prepare(int Q, int storage, int S, int NT, int* blocks_per_sm) {
  if (!collapse_resident_supported(Q, storage, S, NT)) return cudaErrorInvalidValue;
  LBKS_COLLAPSE_CASES(return (cr_prepare_t<Cc, STc, Sc>(NT, blocks_per_sm)));
  return cudaErrorInvalidValue;
}

cudaError_t launch_collapse_resident(const ResidentLaunch& L, cudaStream_t s) {
  const int Q = L.Q, storage = L.storage, S = L.S;
  if (!collapse_resident_supported(Q, storage, S, L.NT) || L.cl != 1) return cudaErrorInvalidValue;
  if (L.nbundles == 0 || L.grid == 0) return cudaSuccess;
  LBKS_COLLAPSE_CASES(return (cr_launch_t<Cc, STc, Sc>(L, s)));
  return cudaErrorInvalidValue;
}

}  // namespace lbks
