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
// holds lattices of up to 2 NT S sites where one block would need segments
// reloaded at every launch, in one of two forms:
//  * two halves (Piece::halo > 0), one per block from its thread 0, each a segment
//    of the ring with halo sites on both sides; every kx steps the blocks exchange
//    their edge sites through shared memory and one cluster barrier (halo_exchange);
//  * one ring across both blocks: at most one piece of a bundle spans both blocks;
//    it has exactly two links across the block edge (block 0's last thread <->
//    block 1's first, and its own periodic wrap), so each block has one thread that
//    receives right-moving values from the other block and one that receives
//    left-moving values.  The threads that send them store their outgoing values
//    into the other block's shared memory (plain st.shared::cluster) and then arrive
//    on that block's mbarrier with release semantics at cluster scope (two arrivals
//    complete a phase); the receiving threads wait on their own block's mbarrier with
//    acquire semantics (a bounded wait: on time-out it sets an error flag, the block
//    stops waiting for the rest of the launch and the launch completes).  Each link
//    is used in both directions every step, so a store into a double-buffered slot is
//    always ordered after the reads of that slot two steps earlier.  The rest of the
//    step uses block barriers only.  Every remote write is an ordinary store that
//    precedes its thread's next cluster barrier, so none can still be in flight when
//    the blocks pass the cluster barriers between bundles or before they exit, also
//    after a time-out, when the receiving side no longer waits.
// A pair's spare threads hold whole small lattices, and a pair may also run two
// single-block bundles side by side (no piece across the edge); the step loop
// carries link code only for bundles that need it (resident_steps<LINK>).
//
// One step of Eq. LB_equation_ordinary:
//  A. per held site: s_g = sum_i g_i, rho = rhobar + s_g, rho^2; g_0's register takes
//     s_g, from which phase B subtracts each plane's post-collision value (the same
//     arithmetic, in the same order, as collide(): g_0 = s_g - sum_{i>=1} g*_i);
//  B. per plane i >= 1, the post-collision value of every site is written
//     straight into the register of the site it streams to (c_i > 0: sites
//     visited from the last one down, c_i < 0: from the first one up, so the
//     destination register's old value has already been used); the values at the
//     thread's edge go to its column of the exchange area: for speed +k the last k + 1
//     slots, for -k the first k + 1 (one more than leave a thread holding S sites);
//  (a ring across a cluster pair: after A, the two threads at the block edge push
//     the same k + 1 values per plane, computed from A's sums, into the other block;)
//  C. one block barrier (and, for the two threads of a cluster block with a link
//     across the block edge, the mbarrier wait), then the values entering from
//     the neighbour thread are read (the neighbour of a piece's last thread is
//     its first: periodic wrap).  The exchange area is double-buffered by step
//     parity, so one barrier per step orders both the reads after the writes
//     and the next overwrite after the reads.
// Threads holding S - 1 sites (slots 0..S-2; slot S-1 holds a bounded value that no
// site reads) take the same code path: with k + 1 values stored per plane and side,
// a reader finds the k values it needs one row further in or not (per thread, fixed
// for the bundle: its left neighbour holds S sites, or it holds S - 1 itself), so the
// only extra work of an (S - 1)-site thread is one predicated load per -k plane.
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
  // Threads without a piece skip the step's arithmetic (S <= 12), or step zeros in their
  // own exchange column (S > 12: the loop without the two branches schedules better there;
  // measured on uniform lattices, 16 x 256: 8.9e11 -> 9.9e11 site-updates/s, while at
  // 12 x 384, 168 registers, the branches are worth 8 %).
  static constexpr bool kSkipIdle = S <= 12;
  // Upper bound of threads per block; sets the register budget per thread.
  static constexpr int kMaxThreads = (ST == kF64) ? 256 : (S <= 8 ? 512 : (S <= 12 ? 384 : 256));
  // Row length of the exchange area: a column per thread of the largest block and two
  // for the values the other block of a cluster pushes in.  A compile-time stride, so
  // that every exchange access is a base address plus an immediate offset.
  static constexpr int kXS = kMaxThreads + 2;
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
  int kx;      // cluster pairs: steps between the halo exchanges of lattice halves
  uint32_t wait_limit;  // try_wait rounds before a wait on the other block is given up
  int withhold_step;    // testing aid: block 1 of a pair sends nothing across the edge
                        // at this step of every bundle with a ring across both blocks (-1: none)
};

constexpr int kFlagClusterTimeout = 2;

// Dynamic shared memory (elements): the staging area of the launch edges
// [Q planes][NT threads x S sites], then the exchange area
// [2 parities][2 directions][xrows][XS] (XS = ResidentCfg::kXS): a column per thread for
// the values leaving it, and the last two (XS - 2: right-moving, XS - 1: left-moving)
// for the values the other block of a cluster pushes in, then the inbox of a lattice half
// [2 parities][2 sides][Q][c_max kPairStepsMax]: side 0 the other half's last halo
// sites (this half's left halo), side 1 its first ones (the right halo).  Neither
// overlaps the staging area, since the other block may write them while this block
// is still staging.
// Rows of one direction of the exchange area: k + 1 for the plane of speed k = 1..c_max,
// from row xrow(k).
__host__ __device__ constexpr int xrows(int C) { return C * (C + 3) / 2; }
__host__ __device__ constexpr int xrow(int k) { return k * (k + 1) / 2 - 1; }
__host__ __device__ constexpr int exchange_rows(int Q) { return 4 * xrows((Q - 1) / 2); }
__host__ __device__ constexpr int halo_max(int Q) { return ((Q - 1) / 2) * kPairStepsMax; }
__host__ __device__ constexpr size_t smem_elems(int Q, int S, int NT, int XS) {
  return (size_t)Q * S * NT + (size_t)exchange_rows(Q) * XS + (size_t)4 * Q * halo_max(Q);
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

// Plain store into another block's shared memory (made visible by the next cluster barrier).
__device__ __forceinline__ void st_cluster(uint32_t addr, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

// Barrier `id` over the first `count` arrivals (a multiple of 32: whole warps), with the
// memory ordering of __syncthreads among the threads that take part (PTX ISA: bar.sync).
__device__ __forceinline__ void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ---- mbarriers (PTX ISA: mbarrier)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

// Makes the initialised mbarriers visible to the other blocks of the cluster (which
// arrive on them); a cluster barrier follows before any use.
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive on the mbarrier at cluster address `mbar` (in another block of the cluster),
// releasing this thread's earlier stores at cluster scope.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t mbar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// One bounded round of waiting for the completion of phase `parity`; acquire at
// cluster scope, so the values the other block stored before its arrivals are visible.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(smem_u32(m)), "r"(parity) : "memory");
  return ok != 0;
}

// Edge values of one thread for the other block of a cluster: the post-collision
// values of its last k + 1 slots for each speed +k (push_edge_right) or of its first
// k + 1 for each -k (push_edge_left), from the pre-collision populations f and phase
// A's rho and rho^2, with the operations of phase B (which computes the same values
// again below), stored into the other block's pushed-in column (cluster address col,
// element stride ntx, the rows of phase B's own column).
template <int Q, typename CT, int S>
__device__ __forceinline__ void push_edge_right(const CT (&f)[Q][S], const CT (&rho)[S], const CT (&rho2)[S],
                                                const Coef<CT, Q>& k, uint32_t col, int ntx) {
  StaticFor<1, Q>::run([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr int c = speed(i);
    if constexpr (c > 0) {
#pragma unroll
      for (int j = 0; j <= c; ++j) {
        constexpr int s0 = S - 1 - c;
        const CT v = post_collision(k.r, f[i][s0 + j], rho[s0 + j], rho2[s0 + j], k.b[i], mul_rn(rho[s0 + j], k.a[i]));
        st_cluster(col + (uint32_t)((xrow(c) + j) * ntx * sizeof(CT)), v);
      }
    }
  });
}

template <int Q, typename CT, int S>
__device__ __forceinline__ void push_edge_left(const CT (&f)[Q][S], const CT (&rho)[S], const CT (&rho2)[S],
                                               const Coef<CT, Q>& k, uint32_t col, int ntx) {
  StaticFor<1, Q>::run([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    constexpr int c = speed(i);
    if constexpr (c < 0) {
      constexpr int kk = -c;
#pragma unroll
      for (int j = 0; j <= kk; ++j) {
        // phase B takes rho a_i of the -c plane from the +c plane before it (a_i is even in
        // c) and b_i as minus that plane's (b_i is odd in c, exactly)
        const CT v = post_collision(k.r, f[i][j], rho[j], rho2[j], -k.b[i - 1], mul_rn(rho[j], k.a[i - 1]));
        st_cluster(col + (uint32_t)((xrow(kk) + j) * ntx * sizeof(CT)), v);
      }
    }
  });
}

// Link state of a block of a cluster pair whose bundle has a piece across the block
// edge: the thread's links to the other block, this block's mbarriers (one per step
// parity), the other block's exchange area and mbarriers in the cluster window, the
// parities of the next phases to complete, and the time-out state of the waits.
struct ClusterLink {
  uint64_t* mbar = nullptr;
  uint32_t peer_x = 0, peer_mbar = 0;
  uint32_t ph = 0;    // bit p: parity of the next phase of mbar[p] to complete
  bool lrem = false;  // the left neighbour is in the other block
  bool rrem = false;  // the right neighbour is in the other block
  bool bad = false;   // a wait ran out: stop waiting (the flag tells the host)
  int* flags = nullptr;
  uint32_t limit = 0;     // try_wait rounds before a wait is given up
  int withhold = -1;      // testing aid: send nothing across the edge at this step
};

// ksteps steps of the register-resident state f (see the kernel below for phases A-C).
// LINK: the bundle has a piece across the edge of a cluster pair, whose boundary
// values go through the other block's shared memory; without it the loop is that of
// a single block (no link code in the loop, so no registers or instructions spent on it).
// lt, rt: exchange columns of the left and right neighbours; lfull: the left neighbour
// holds S sites; full: this thread does.  SKIP (see ResidentCfg::kSkipIdle): threads
// without a piece skip the arithmetic and every thread takes part in the block barrier.
// Otherwise, without LINK, warps without a piece leave at once (wrun false) and the step
// barrier is the named barrier 1 over the nbar threads of the warps that hold one; with
// LINK every thread steps (those without a piece on zeros), so that every thread keeps
// the link's phase parities.
template <int Q, int S, int XS, bool LINK, bool SKIP, typename CT>
__device__ __forceinline__ void resident_steps(CT (&f)[Q][S], const Coef<CT, Q>& k, const int step0, const int ksteps,
                                               CT* const xbase, const int t, const bool active, const bool full,
                                               const int lt, const int rt, const bool lfull, const bool wrun,
                                               const int nbar, ClusterLink& ln) {
  constexpr bool kLeave = !SKIP && !LINK;
  if (kLeave && !wrun) return;
  constexpr int C = cmax_of(Q);
  constexpr int NR = xrows(C);  // rows per direction
  constexpr int NTX = XS;
  // Where this thread reads: the right-moving values of its left neighbour's column, one
  // row in when that neighbour holds S sites (its row 0 is a value that stays inside it);
  // the left-moving values of its right neighbour's column, one row in when this thread
  // holds S - 1 sites (row 0 then goes to slot S - 1 - k, the others to S - k .. S - 1).
  const int rd_r = (lfull ? NTX : 0) + lt;
  const int rd_l = (NR + (full ? 0 : 1)) * NTX + rt;
  for (int step = step0; step < step0 + ksteps; ++step) {
    const int pb = step & 1;
    CT* const xp = xbase + pb * 2 * NR * NTX;  // this step's exchange area: [R|L][NR][NTX]
    CT* const xw = xp + t;                     // this thread's column
    if (!SKIP || active) {
      // A. per-site sums; g_0's register becomes the accumulator of g*_0
      CT rho[S], rho2[S], tt[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        CT sg = f[0][s];
#pragma unroll
        for (int i = 1; i < Q; ++i) sg = add_rn(sg, f[i][s]);
        rho[s] = add_rn(k.rhobar, sg);
        rho2[s] = mul_rn(rho[s], rho[s]);
        f[0][s] = sg;
      }
      if constexpr (LINK) {
        // Send the values this step sends across the block edge before phase B, from
        // phase A's sums with the arithmetic of phase B (which computes them again
        // below), so that the transfer overlaps the rest of the step; each sending
        // thread then arrives on the other block's mbarrier of this parity, releasing its
        // stores at cluster scope (this step's phase there completes on the two
        // arrivals, one per direction).  Arriving after phase B instead delays the
        // receiver: 7 % slower rings.
        if (step != ln.withhold) {
          if (ln.rrem) {
            push_edge_right<Q>(f, rho, rho2, k, ln.peer_x + (uint32_t)((pb * 2 * NR * NTX + XS - 2) * sizeof(CT)),
                               NTX);
            mbar_arrive_remote(ln.peer_mbar + 8u * pb);
          }
          if (ln.lrem) {
            push_edge_left<Q>(f, rho, rho2, k,
                              ln.peer_x + (uint32_t)(((pb * 2 + 1) * NR * NTX + XS - 1) * sizeof(CT)), NTX);
            mbar_arrive_remote(ln.peer_mbar + 8u * pb);
          }
        }
      }
      // B. plane by plane: collide, write to the destination site's register and/or the
      // exchange column.
      StaticFor<1, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int c = speed(i);
        constexpr int kk = c > 0 ? c : -c;
        constexpr int row0 = xrow(kk);
        if constexpr (c > 0) {
#pragma unroll
          for (int s = S - 1; s >= 0; --s) {
            tt[s] = mul_rn(rho[s], k.a[i]);  // shared with the -c plane that follows
            const CT v = post_collision(k.r, f[i][s], rho[s], rho2[s], k.b[i], tt[s]);
            f[0][s] = add_rn(f[0][s], -v);
            if (s >= S - 1 - kk) xw[(row0 + s - (S - 1 - kk)) * NTX] = v;
            if (s + kk <= S - 1) f[i][s + kk] = v;
          }
        } else {
#pragma unroll
          for (int s = 0; s < S; ++s) {
            // b_i of the -c plane is exactly minus the +c plane's (B_i = J w1_i, w1 odd in
            // c), taken with the FMA's negation so that it needs no register of its own
            const CT v = post_collision(k.r, f[i][s], rho[s], rho2[s], -k.b[i - 1], tt[s]);
            f[0][s] = add_rn(f[0][s], -v);
            if (s <= kk) xw[(NR + row0 + s) * NTX] = v;
            if (s >= kk) f[i][s - kk] = v;
          }
        }
      });
    }
    if constexpr (kLeave) named_barrier(1, nbar);
    else __syncthreads();
    if constexpr (LINK) {
      if ((ln.lrem || ln.rrem) && !ln.bad) {
        uint32_t it = 0;
        while (!mbar_try_wait(&ln.mbar[pb], (ln.ph >> pb) & 1u)) {
          if (++it >= ln.limit) {
            ln.bad = true;
            if (ln.flags) atomicOr(ln.flags, kFlagClusterTimeout);
            break;
          }
        }
      }
      ln.ph ^= 1u << pb;
    }
    if (!SKIP || active) {
      // C. values entering from the neighbours (pushed in by the other block for
      // a piece's threads at a block edge)
      StaticFor<1, Q>::run([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int c = speed(i);
        constexpr int kk = c > 0 ? c : -c;
        constexpr int row0 = xrow(kk);
        if constexpr (c > 0) {
#pragma unroll
          for (int jj = 0; jj < kk; ++jj) f[i][jj] = xp[rd_r + (row0 + jj) * NTX];
        } else {
#pragma unroll
          for (int jj = 0; jj < kk; ++jj) f[i][S - kk + jj] = xp[rd_l + (row0 + jj) * NTX];
          if (!full) f[i][S - 1 - kk] = xp[rd_l + (row0 - 1) * NTX];
        }
      });
    }
  }
}

// Halo exchange of a lattice held as two halves by a cluster pair (Piece::halo = h;
// `half` is this block's half, the bundle's first piece in block 0 and its second in
// block 1, held from thread 0 of the block).  Each half runs kx steps as a segment of
// the ring (its h halo sites on each side absorb the values its thread ring wraps in,
// which travel at most c_max sites per step), then its first and last h own sites go
// to the other block, whose halos they are, and come back as this block's halos.  In
// segment coordinates the own sites are [h, h + own): sites [h, 2h) become the other
// half's right halo, [own, own + h) its left halo; this half's left halo is [0, h) and
// its right halo [h + own, 2h + own) (sites beyond that, when the segment was
// lengthened to split into runs of S and S-1 sites, are farther than h from the own
// sites and are not refreshed).
//  a. threads holding any of those sites put all theirs into the staging area (idle
//     between the launch edges), at their staged index (site index: the half starts
//     at thread 0);
//  b. all threads copy the 2 h Q outgoing values into the other block's inbox;
//  c. after one cluster barrier, all threads copy the inbox into the halo sites of
//     the staging area;
//  d. the threads of a. reload their registers.
// The inbox is double-buffered by exchange parity: a write into it is ordered after
// the other block's reads of that buffer by the cluster barrier of the exchange between.
// (The half's halo, own sites and threads are read from shared memory here, written at
// the start of the bundle, so that the step loop around keeps no registers for them.)
template <int Q, int S, typename CT>
__device__ __forceinline__ void halo_exchange(CT (&f)[Q][S], const int (&half)[3], const bool full,
                                              const int start, const int NT, const int t, CT* const stage,
                                              CT* const inbox, const int par) {
  constexpr int HM = halo_max(Q);
  const int SS = NT * S;  // plane stride of the staging area
  const int h = half[0], own = half[1];
  const int n = full ? S : S - 1;
  const bool mine = t < half[2];  // the half is held from thread 0 of the block
  const bool edge = mine && (start < 2 * h || start + n > own);
  if (edge) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (s < n) stage[i * SS + start + s] = f[i][s];
  }
  __syncthreads();
  const uint32_t peer_inbox = cluster_addr(inbox, cluster_rank() ^ 1);
  for (int tt = t; tt < 2 * h; tt += NT) {
    // tt < h: own site h + tt -> the other half's right halo (side 1); else own site
    // own + tt - h -> its left halo (side 0)
    const int side = tt < h ? 1 : 0;
    const int m = tt < h ? tt : tt - h;
    const int src = tt < h ? h + m : own + m;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      st_cluster(peer_inbox + (uint32_t)((((par * 2 + side) * Q + i) * HM + m) * sizeof(CT)), stage[i * SS + src]);
  }
  cluster_barrier();
  for (int tt = t; tt < 2 * h; tt += NT) {
    const int side = tt < h ? 0 : 1;
    const int m = tt < h ? tt : tt - h;
    const int dst = tt < h ? m : h + own + m;
#pragma unroll
    for (int i = 0; i < Q; ++i) stage[i * SS + dst] = inbox[((par * 2 + side) * Q + i) * HM + m];
  }
  __syncthreads();
  if (edge) {
#pragma unroll
    for (int i = 0; i < Q; ++i)
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (s < n) f[i][s] = stage[i * SS + start + s];
  }
}

// Where a piece's sites sit, for the thread g = rank * NT + t of its work group: the
// thread's index j in the piece and its first site, whether it holds S sites, the
// piece's threads in this block [jlo, jlo + Vr) and their sites [lo_site, hi_site), the
// staged index of piece site li (sbase + li), and the run-local site of this thread's
// first launch-edge access.  Computed before the load and again, from the piece read
// anew, before the store, so that none of it is held in registers through the steps.
struct PieceGeom {
  int64_t N, x_first;
  int j, start, jlo, Vr, lo_site, hi_site, sbase;
  bool full;
};

template <int S>
__device__ __forceinline__ PieceGeom piece_geom(const Piece& pc, const int64_t N, const int g, const int rank,
                                                const int NT) {
  PieceGeom G;
  const int V = pc.nthr;
  const int mfull = pc.n - V * (S - 1);  // threads holding S sites; the rest hold S-1
  auto site_start = [&](int jj) { return jj < mfull ? jj * S : mfull * S + (jj - mfull) * (S - 1); };
  G.N = N;
  G.j = g - pc.t0;
  G.full = G.j < mfull;
  G.start = site_start(G.j);
  G.jlo = max(0, rank * NT - pc.t0);
  const int jhi = min(V, rank * NT + NT - pc.t0);
  G.Vr = jhi - G.jlo;
  G.lo_site = site_start(G.jlo);
  G.hi_site = site_start(jhi);
  G.sbase = (pc.t0 + G.jlo - rank * NT) * S - G.lo_site;
  G.x_first = (pc.x0 + G.lo_site + (G.j - G.jlo)) % N;
  return G;
}

template <int Q, int ST, int S, int CL>
__global__ void __launch_bounds__(ResidentCfg<ST, S>::kMaxThreads, 1) resident_kernel(const ResidentArgs a) {
  static_assert(CL == 1 || CL == 2, "work groups are one block or a pair of blocks");
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NT = blockDim.x;
  constexpr int NTX = ResidentCfg<ST, S>::kXS;        // exchange-area row length
  constexpr bool kSkip = ResidentCfg<ST, S>::kSkipIdle;
  CT* const stage = reinterpret_cast<CT*>(smem_raw);   // [Q][NT * S] at the launch edges
  CT* const xbase = stage + Q * S * NT;                // [parity][R|L][xrows][NTX]
  CT* const inbox = xbase + exchange_rows(Q) * NTX;    // [parity][L|R halo][Q][c_max kPairStepsMax]
  __shared__ int s_bundle;
  __shared__ int s_half[3];                            // CL = 2: halo, own sites, threads of this block's half
  __shared__ __align__(8) uint64_t s_mbar[2];          // CL = 2: the other block's sends, one per parity
  // CL = 2, kept in shared memory between the bundles whose pieces span the block edge
  // (so that no registers are held for them while other bundles run): bit p of s_ph is
  // the parity of the next phase of s_mbar[p] to complete; s_bad: a wait ran out, stop
  // waiting (the flag tells the host)
  __shared__ uint32_t s_ph;
  __shared__ int s_bad;
  const int t = threadIdx.x;
  const int rank = CL == 1 ? 0 : cluster_rank();
  const int g = rank * NT + t;  // thread index in the work group
  if constexpr (CL == 2) {
    if (t == 0) {
      mbar_init(&s_mbar[0], 2);  // one arrival per direction from the other block
      mbar_init(&s_mbar[1], 2);
      fence_mbar_init();
      s_ph = 0;
      s_bad = 0;
    }
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
    if constexpr (CL == 2) {
      // a lattice held as two halves: the first piece of the bundle in block 0, the
      // second in block 1, each from thread 0 (read after the load phase's barriers)
      if (t == 0) {
        const Piece& hp = a.pieces[bd.x + rank];
        const bool hv = bd.y > rank && hp.halo > 0;
        s_half[0] = hv ? hp.halo : 0;
        s_half[1] = hv ? hp.st_hi - hp.st_lo : 0;
        s_half[2] = hv ? hp.nthr : 0;
      }
    }

    CT f[Q][S];
    Coef<CT, Q> k{};
    bool full = true;
    int start = 0;
    int lt = t, rt = t;                    // exchange columns the incoming values are read from
    bool lfull = true;                     // the left neighbour holds S sites
    bool lrem = false, rrem = false;       // left / right neighbour in the other block
    PieceGeom G{};
    const T* fs = nullptr;
    if (active) {
      const Piece pc = a.pieces[pidx];
      const RunDesc& d = a.runs[pc.run];
      k = load_coef<CT, Q>(d);
      G = piece_geom<S>(pc, d.N, g, rank, NT);
      full = G.full;
      start = G.start;
      const int V = pc.nthr, j = G.j;
      const int lg = pc.t0 + (j == 0 ? V - 1 : j - 1);
      const int rg = pc.t0 + (j == V - 1 ? 0 : j + 1);
      const int lrank = CL == 1 ? 0 : lg / NT;
      const int rrank = CL == 1 ? 0 : rg / NT;
      lrem = lrank != rank;
      rrem = rrank != rank;
      lt = lrem ? NTX - 2 : lg - lrank * NT;   // pushed-in columns for a neighbour in the other block
      rt = rrem ? NTX - 1 : rg - rrank * NT;
      lfull = (j == 0 ? V - 1 : j - 1) < pc.n - V * (S - 1);
      fs = static_cast<const T*>(a.src.f) + d.off;
    }

    // ---- load: coalesced global reads of all planes into the staging area, then registers
    if (active) {
      int64_t x = G.x_first;
      for (int li = G.lo_site + (G.j - G.jlo); li < G.hi_site; li += G.Vr) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          stage[i * NT * S + G.sbase + li] = to_compute(fs[(int64_t)i * a.src.plane + x], k.scale);
        x += G.Vr;
        while (x >= G.N) x -= G.N;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s) f[i][s] = (s < S - 1 || full) ? stage[i * NT * S + G.sbase + start + s] : CT(0);
    } else {
      // a thread without a piece steps zeros in its own exchange column
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s) f[i][s] = CT(0);
    }
    // block-uniform: does a piece of this bundle span both blocks (then this block
    // has one thread with lrem and one with rrem, possibly the same thread)
    bool span = false, halves = false;
    if constexpr (CL == 2) {
      span = __syncthreads_or(lrem || rrem);
      // block-uniform: the bundle holds a lattice as two halves (one per block)
      halves = __syncthreads_or(active && a.pieces[pidx].halo > 0);
    }
    // the warps that hold a piece, and their threads (the step barrier's count)
    const bool wrun = __any_sync(0xffffffffu, active);
    const int nbar = 32 * __syncthreads_count(wrun && (t & 31) == 0);

    ClusterLink ln;
    if constexpr (CL == 2) {
      if (span) {
        ln.mbar = s_mbar;
        ln.peer_x = cluster_addr(xbase, rank ^ 1);
        ln.peer_mbar = cluster_addr(s_mbar, rank ^ 1);
        ln.ph = s_ph;
        ln.lrem = lrem;
        ln.rrem = rrem;
        ln.bad = s_bad != 0;
        ln.flags = a.flags;
        ln.limit = a.wait_limit;
        ln.withhold = rank == 1 ? a.withhold_step : -1;
        resident_steps<Q, S, NTX, true, kSkip>(f, k, 0, a.ksteps, xbase, t, active, full, lt, rt, lfull, wrun, nbar, ln);
        // every thread toggled the same parities; the next write follows the barriers
        // of the store phase below
        if (t == 0) s_ph = ln.ph;
        if (ln.bad) s_bad = 1;
      } else if (halves && a.kx > 0) {
        for (int s0 = 0; s0 < a.ksteps; s0 += a.kx) {
          const int kk = min(a.kx, a.ksteps - s0);
          resident_steps<Q, S, NTX, false, kSkip>(f, k, s0, kk, xbase, t, active, full, lt, rt, lfull, wrun, nbar, ln);
          if (s0 + kk < a.ksteps)
            halo_exchange<Q, S>(f, s_half, full, start, NT, t, stage, inbox, (s0 / a.kx) & 1);
        }
      } else {
        resident_steps<Q, S, NTX, false, kSkip>(f, k, 0, a.ksteps, xbase, t, active, full, lt, rt, lfull, wrun, nbar, ln);
      }
    } else {
      resident_steps<Q, S, NTX, false, kSkip>(f, k, 0, a.ksteps, xbase, t, active, full, lt, rt, lfull, wrun, nbar, ln);
    }
    __syncthreads();

    // ---- store: registers into the staging area, then coalesced global writes of all planes
    Piece pc{};
    if (active) {
      pc = a.pieces[pidx];  // read anew (after the barriers of the steps)
      G = piece_geom<S>(pc, a.runs[pc.run].N, g, rank, NT);
#pragma unroll
      for (int i = 0; i < Q; ++i)
#pragma unroll
        for (int s = 0; s < S; ++s)
          if (s < S - 1 || G.full) stage[i * NT * S + G.sbase + G.start + s] = f[i][s];
    }
    __syncthreads();
    if (active) {
      const RunDesc& d = a.runs[pc.run];
      const CT inv_scale = load_coef<CT, Q>(d).inv_scale;
      T* const fd = static_cast<T*>(a.dst.f) + d.off;
      int64_t x = G.x_first;
      for (int li = G.lo_site + (G.j - G.jlo); li < G.hi_site; li += G.Vr) {
        if (li >= pc.st_lo && li < pc.st_hi) {
#pragma unroll
          for (int i = 0; i < Q; ++i)
            from_compute(stage[i * NT * S + G.sbase + li], inv_scale, fd + (int64_t)i * a.dst.plane + x);
        }
        x += G.Vr;
        while (x >= G.N) x -= G.N;
      }
    }
    __syncthreads();
  }
}

template <int Q, int ST, int S>
size_t smem_bytes_t(int NT) {
  using CT = typename StorageType<ST>::compute;
  return sizeof(CT) * smem_elems(Q, S, NT, ResidentCfg<ST, S>::kXS);
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
      case 18: if constexpr (STc != kF64) { constexpr int Sc = 18; OP; } break;       \
      case 20: if constexpr (STc != kF64) { constexpr int Sc = 20; OP; } break;       \
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
