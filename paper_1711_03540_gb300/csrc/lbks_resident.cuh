// Register-resident, temporally blocked fused step for ensembles of lattices
// (one persistent launch runs ksteps steps of every lattice it is given).
//
// Work unit ("piece"): a whole periodic lattice (ring) or, for lattices larger
// than one work group holds, a stretch of one with c_max * ksteps halo sites on
// each side (segment).  A piece occupies V consecutive threads of a work group;
// thread j holds S or S-1 consecutive sites (all Q planes) in registers, so
// any lattice length n with V (S-1) < n <= V S is held exactly.  Pieces of
// different runs (different N, tau, alpha, beta) are packed into the same
// work group by the host ("bundle").
//
// A work group is one thread block (CL = 1) or a cluster of CL = 2 thread
// blocks (CL = 2) whose threads are numbered g = rank * blockDim.x + t.  This
// holds lattices of up to 2 NT S sites whole, with no halo and no launch-edge
// overhead, where one block would need segments.  At most one piece of a bundle
// spans both blocks; it has exactly two links across the block edge (block 0's
// last thread <-> block 1's first, and its own periodic wrap), so each block has
// one thread that receives right-moving values from the other block and one that
// receives left-moving values.  Those threads push their outgoing values into
// the other block's shared memory with st.async, whose completion counts bytes
// on an mbarrier there; the receiving thread waits on its own block's mbarrier
// (a bounded wait: on time-out it sets an error flag, stops waiting and the
// launch completes).  Each link is used in both directions every step, so a
// push into a double-buffered slot is always ordered after the reads of that
// slot two steps earlier.  The rest of the step uses __syncthreads only.
//
// One step of Eq. LB_equation_ordinary:
//  A. per held site: s_g = sum_i g_i, rho = rhobar + s_g, rho^2;
//  B. per plane i >= 1, the post-collision value of every site is written
//     straight into the register of the site it streams to (c_i > 0: sites
//     visited from the last one down, c_i < 0: from the first one up, so the
//     destination register's old value has already been used); the c_i values
//     that leave the thread go to shared memory;  g_0 = s_g - sum of the others
//     (mass conservation; the same arithmetic, in the same order, as collide());
//  C. one block barrier (and, for the two threads of a cluster block with a link
//     across the block edge, the mbarrier wait), then the values entering from
//     the neighbour thread are read (the neighbour of a piece's last thread is
//     its first: periodic wrap).  The exchange area is double-buffered by step
//     parity, so one barrier per step orders both the reads after the writes
//     and the next overwrite after the reads.
// For a segment the wrap injects unrelated values at its two ends; they travel
// at most c_max sites per step and never reach the stored middle.
//
// Loads and stores at the launch edges go through shared memory so that
// global accesses are coalesced (consecutive threads, consecutive sites); each
// block stages the sites its own threads hold.
//
// Work groups take bundles from a global counter (atomicAdd; in a cluster block 0
// takes it and block 1 reads it from block 0's shared memory), largest first,
// until the queue is empty: a persistent grid with a ragged work queue.  No work
// group waits on another, and every thread of a cluster passes the same sequence
// of cluster barriers (the bundle index, and so the loop trip counts, are the
// same in both blocks).
#pragma once

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
  int* flags;  // bit 2 set when a bounded wait on the other block of a cluster ran out
};

constexpr int kFlagClusterTimeout = 2;
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds before a wait is given up

// Dynamic shared memory (elements): the staging area of the launch edges
// [Q planes][NT threads x S sites], then the exchange area
// [2 parities][2 directions][NX][NT + 2]: a column per thread for the values
// leaving it, and two more (NT: right-moving, NT + 1: left-moving) for the values
// the other block of a cluster pushes in.  The exchange area does not overlap the
// staging area, since a push may land while this block is still staging.
__host__ __device__ constexpr int exchange_rows(int Q) { return 4 * ((Q - 1) / 2) * ((Q - 1) / 2 + 1) / 2; }
__host__ __device__ constexpr size_t smem_elems(int Q, int S, int NT) {
  return (size_t)Q * S * NT + (size_t)exchange_rows(Q) * (NT + 2);
}

// ---- thread block clusters (PTX ISA: barrier.cluster, mapa, ld.shared::cluster)

__device__ __forceinline__ int cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return (int)r;
}

// Every thread of every block of the cluster arrives; shared-memory writes before
// it (in any block) are visible to reads after it (in any block).
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address, in the cluster's shared window, of the object at p in block `rank`.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
               : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ int ld_cluster(uint32_t addr, int) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// ---- mbarriers with transaction counts (PTX ISA: mbarrier, st.async)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

// Makes the initialised mbarriers visible to the other blocks of the cluster
// (complete_tx from there); a cluster barrier follows before any use.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}

// One bounded round of waiting for the completion of phase `parity`; acquire at
// cluster scope, so the bytes that st.async from the other block wrote are visible.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
  return ok != 0;
}

// Store v at addr in another block's shared memory; its completion counts
// sizeof(v) bytes on the mbarrier at mbar (in that block).
__device__ __forceinline__ void st_async(uint32_t addr, float v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];"
               ::"r"(addr), "f"(v), "r"(mbar) : "memory");
}
__device__ __forceinline__ void st_async(uint32_t addr, double v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
               ::"r"(addr), "d"(v), "r"(mbar) : "memory");
}

// Edge values of one thread for the other block of a cluster, from its pre-collision
// populations f (n held sites): the post-collision values that leave the thread to
// the right (c_i > 0: sites n - c_i .. n - 1) or to the left (c_i < 0: sites
// 0 .. |c_i| - 1), with the operations of phase B in the same order, stored into
// the other block's pushed-in column (element stride ntx, row (|c|(|c|-1)/2 + j)).
template <int Q, int n, typename CT, int SF>
__device__ __forceinline__ void push_edge_right(const CT (&f)[Q][SF], const Coef<CT, Q>& k, uint32_t col, int ntx,
                                                uint32_t mbar) {
  constexpr int C = cmax_of(Q);
  CT er[C], er2[C];  // rho and rho^2 of sites n - C .. n - 1
#pragma unroll
  for (int m = 0; m < C; ++m) {
    CT sg = f[0][n - C + m];
#pragma unroll
    for (int i = 1; i < Q; ++i) sg = add_rn(sg, f[i][n - C + m]);
    er[m] = add_rn(k.rhobar, sg);
    er2[m] = mul_rn(er[m], er[m]);
  }
  StaticFor<1, Q>::run([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr int c = speed(i);
    if constexpr (c > 0) {
      constexpr int base = c * (c - 1) / 2;
#pragma unroll
      for (int j = 0; j < c; ++j) {
        const int m = C - c + j;
        const CT v = post_collision(k.r, f[i][n - c + j], er[m], er2[m], k.b[i], mul_rn(er[m], k.a[i]));
        st_async(col + (uint32_t)((base + j) * ntx * sizeof(CT)), v, mbar);
      }
    }
  });
}

template <int Q, typename CT, int SF>
__device__ __forceinline__ void push_edge_left(const CT (&f)[Q][SF], const Coef<CT, Q>& k, uint32_t col, int ntx,
                                               uint32_t mbar) {
  constexpr int C = cmax_of(Q);
  CT er[C], er2[C];  // rho and rho^2 of sites 0 .. C - 1
#pragma unroll
  for (int m = 0; m < C; ++m) {
    CT sg = f[0][m];
#pragma unroll
    for (int i = 1; i < Q; ++i) sg = add_rn(sg, f[i][m]);
    er[m] = add_rn(k.rhobar, sg);
    er2[m] = mul_rn(er[m], er[m]);
  }
  StaticFor<1, Q>::run([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr int c = speed(i);
    if constexpr (c < 0) {
      constexpr int kk = -c;
      constexpr int base = kk * (kk - 1) / 2;
#pragma unroll
      for (int j = 0; j < kk; ++j) {
        // phase B takes rho a_i of the -c plane from the +c plane before it (a_i is even in c)
        const CT v = post_collision(k.r, f[i][j], er[j], er2[j], k.b[i], mul_rn(er[j], k.a[i - 1]));
        st_async(col + (uint32_t)((base + j) * ntx * sizeof(CT)), v, mbar);
      }
    }
  });
}

template <int Q, int ST, int S, int CL>
__global__ void __launch_bounds__(ResidentCfg<ST, S>::kMaxThreads, 1) resident_kernel(const ResidentArgs a) {
  static_assert(CL == 1 || CL == 2, "work groups are one block or a pair of blocks");
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  constexpr int C = cmax_of(Q);
  constexpr int NX = C * (C + 1) / 2;  // values leaving a thread per direction per step
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  const int NTX = NT + 2;                              // exchange-area row length
  CT* const stage = reinterpret_cast<CT*>(smem_raw);   // [Q][NT * S] at the launch edges
  CT* const xbase = stage + Q * S * NT;                // [parity][R|L][NX][NT + 2]
  __shared__ int s_bundle;
  __shared__ __align__(8) uint64_t s_mbar[2];          // CL = 2: counts the pushed bytes, one per parity
  const int t = threadIdx.x;
  const int rank = CL == 1 ? 0 : cluster_rank();
  const int g = rank * NT + t;  // thread index in the work group
  uint32_t peer_x = 0, peer_mbar = 0;  // the other block's exchange area and mbarriers
  uint32_t ph = 0;   // bit p: parity of the next phase of s_mbar[p] to complete
  bool bad = false;  // a wait ran out: stop waiting (the flag tells the host)
  if constexpr (CL == 2) {
    if (t == 0) {
      mbar_init(&s_mbar[0], 1);
      mbar_init(&s_mbar[1], 1);
      fence_mbar_init();
    }
    peer_x = cluster_addr(xbase, rank ^ 1);
    peer_mbar = cluster_addr(s_mbar, rank ^ 1);
  }

  for (;;) {
    int b;
    if constexpr (CL == 1) {
      if (t == 0) s_bundle = atomicAdd(a.queue, 1);
      __syncthreads();
      b = s_bundle;
      __syncthreads();
    } else {
      // (the first of these also publishes the mbarrier initialisation)
      if (rank == 0 && t == 0) s_bundle = atomicAdd(a.queue, 1);
      cluster_barrier();
      b = rank == 0 ? s_bundle : ld_cluster(cluster_addr(&s_bundle, 0), int());
      cluster_barrier();  // block 1 has read s_bundle before block 0 takes the next bundle
    }
    if (b >= a.nbundles) break;
    const int2 bd = a.bundles[b];

    int pidx = -1;
    for (int p = bd.x; p < bd.x + bd.y; ++p) {
      const int t0 = a.pieces[p].t0;
      if (g >= t0 && g < t0 + a.pieces[p].nthr) { pidx = p; break; }
    }
    const bool active = pidx >= 0;

    CT f[Q][S];
    Coef<CT, Q> k;
    bool full = true;
    int j = 0, start = 0;
    int lt = t, rt = t;                    // exchange columns the incoming values are read from
    bool lrem = false, rrem = false;       // left / right neighbour in the other block
    int jlo = 0, Vr = 1, lo_site = 0, hi_site = 0, sbase = 0;
    Piece pc{};
    int64_t N = 1, x_first = 0;
    const T* fs = nullptr;
    T* fd = nullptr;
    if (active) {
      pc = a.pieces[pidx];
      const RunDesc& d = a.runs[pc.run];
      k = load_coef<CT, Q>(d);
      N = d.N;
      const int V = pc.nthr;
      j = g - pc.t0;
      const int mfull = pc.n - V * (S - 1);  // threads holding S sites; the rest hold S-1
      auto site_start = [&](int jj) { return jj < mfull ? jj * S : mfull * S + (jj - mfull) * (S - 1); };
      full = j < mfull;
      start = site_start(j);
      const int lg = pc.t0 + (j == 0 ? V - 1 : j - 1);
      const int rg = pc.t0 + (j == V - 1 ? 0 : j + 1);
      const int lrank = CL == 1 ? 0 : lg / NT;
      const int rrank = CL == 1 ? 0 : rg / NT;
      lrem = lrank != rank;
      rrem = rrank != rank;
      lt = lrem ? NT : lg - lrank * NT;        // pushed-in columns for a neighbour in the other block
      rt = rrem ? NT + 1 : rg - rrank * NT;
      // the piece's threads in this block, and the sites they hold
      jlo = max(0, rank * NT - pc.t0);
      const int jhi = min(V, rank * NT + NT - pc.t0);
      Vr = jhi - jlo;
      lo_site = site_start(jlo);
      hi_site = site_start(jhi);
      sbase = (pc.t0 + jlo - rank * NT) * S - lo_site;  // staged index of piece site li: sbase + li
      x_first = (pc.x0 + lo_site + (j - jlo)) % N;
      fs = static_cast<const T*>(a.src.f) + d.off;
      fd = static_cast<T*>(a.dst.f) + d.off;
    }

    // ---- load: coalesced global reads of all planes into the staging area, then registers
    if (active) {
      int64_t x = x_first;
      for (int li = lo_site + (j - jlo); li < hi_site; li += Vr) {
#pragma unroll
        for (int i = 0; i < Q; ++i) stage[i * NT * S + sbase + li] = to_compute(fs[(int64_t)i * a.src.plane + x], k.scale);
        x += Vr;
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
    // block-uniform: does a piece of this bundle span both blocks (then this block
    // has one thread with lrem and one with rrem, possibly the same thread)
    bool span = false;
    if constexpr (CL == 2) span = __syncthreads_or(lrem || rrem);
    else __syncthreads();

    for (int step = 0; step < a.ksteps; ++step) {
      const int pb = step & 1;
      const int par = pb * 2 * NX * NTX;
      CT* const xr = xbase + par;  // right-moving values leaving threads
      CT* const xl = xr + NX * NTX; // left-moving values leaving threads
      if constexpr (CL == 2) {
        // this step's phase of s_mbar[pb] completes on this arrival and on the
        // 2 NX values the other block pushes (NX per direction)
        if (lrem && !bad) mbar_arrive_expect_tx(&s_mbar[pb], 2 * NX * (uint32_t)sizeof(CT));
        // Push the values this step sends across the block edge first, computed from
        // the pre-collision state with the arithmetic of phase B (which computes them
        // again below), so that the transfer overlaps the step's work.
        if (rrem) {
          if (full) push_edge_right<Q, S>(f, k, peer_x + (uint32_t)((par + NT) * sizeof(CT)), NTX, peer_mbar + 8u * pb);
          else push_edge_right<Q, S - 1>(f, k, peer_x + (uint32_t)((par + NT) * sizeof(CT)), NTX, peer_mbar + 8u * pb);
        }
        if (lrem) push_edge_left<Q>(f, k, peer_x + (uint32_t)((par + NX * NTX + NT + 1) * sizeof(CT)), NTX,
                                    peer_mbar + 8u * pb);
      }
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
                else xr[base * NTX + t] = v;
              } else if (s <= S - 2) {
                xr[(base + (full ? s + kk - S : s + kk - S + 1)) * NTX + t] = v;
              } else if (full) {  // s == S - 1 holds a site only in threads with S sites
                xr[(base + s + kk - S) * NTX + t] = v;
              }
            }
          } else {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const CT v = post_collision(k.r, f[i][s], rho[s], rho2[s], k.b[i], tt[s]);
              acc[s] = add_rn(acc[s], -v);
              if (s >= kk) f[i][s - kk] = v;
              else xl[(base + s) * NTX + t] = v;
            }
          }
        });
#pragma unroll
        for (int s = 0; s < S; ++s) f[0][s] = acc[s];
      }
      __syncthreads();
      if constexpr (CL == 2) {
        if ((lrem || rrem) && !bad) {
          uint32_t it = 0;
          while (!mbar_try_wait(&s_mbar[pb], (ph >> pb) & 1u)) {
            if (++it == kWaitLimit) {
              bad = true;
              if (a.flags) atomicOr(a.flags, kFlagClusterTimeout);
              break;
            }
          }
        }
        if (span) ph ^= 1u << pb;
      }
      if (active) {
        // C. values entering from the neighbours (pushed in by the other block for
        // a piece's threads at a block edge)
        StaticFor<1, Q>::run([&](auto ic) {
          constexpr int i = decltype(ic)::value;
          constexpr int c = speed(i);
          constexpr int kk = c > 0 ? c : -c;
          constexpr int base = kk * (kk - 1) / 2;
          if constexpr (c > 0) {
#pragma unroll
            for (int jj = 0; jj < kk; ++jj)
              f[i][jj] = xr[(base + jj) * NTX + lt];
          } else {
            // threads with S sites fill slots S-kk .. S-1, threads with S-1 sites S-1-kk .. S-2
#pragma unroll
            for (int jj = 0; jj < kk; ++jj) {
              const CT v = xl[(base + jj) * NTX + rt];
              if (full) f[i][S - kk + jj] = v;
              else f[i][S - 1 - kk + jj] = v;
            }
          }
        });
      }
    }
    __syncthreads();

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
      for (int li = lo_site + (j - jlo); li < hi_site; li += Vr) {
        if (li >= pc.st_lo && li < pc.st_hi) {
#pragma unroll
          for (int i = 0; i < Q; ++i)
            from_compute(stage[i * NT * S + sbase + li], k.inv_scale, fd + (int64_t)i * a.dst.plane + x);
        }
        x += Vr;
        while (x >= N) x -= N;
      }
    }
    __syncthreads();
  }
}

template <int Q, int ST, int S>
size_t smem_bytes_t(int NT) {
  using CT = typename StorageType<ST>::compute;
  return sizeof(CT) * smem_elems(Q, S, NT);
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

}  // namespace lbks
