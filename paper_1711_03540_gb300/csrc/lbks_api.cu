// Host side of the C ABI (include/lb_ks.h): handle, validation, memory
// layout, work planning, step scheduling with CUDA-graph replay, guard,
// checkpointing.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lb_ks.h"
#include "lbks_internal.h"
#include "lbks_plan.h"

namespace lbks {
int stream_tile_sites();
cudaError_t stream_prepare(int Q, int storage);
}

using namespace lbks;
using namespace lbks::plan;

namespace {

thread_local std::string g_ctor_error = "no error";

constexpr int kAlign = 32;  // elements: run offsets and the plane stride are multiples of this
constexpr uint32_t kMagic = 0x534b424cu;  // "LBKS"
constexpr uint32_t kVersion = 1;

// Sites of one handle, all runs: 2^34 sites take 320 GB in the smallest storage
// (D1Q5, FP16, two arenas), beyond the device; the bound keeps the host's tile
// lists (int32 indices) and the planning within range before any allocation.
constexpr int64_t kMaxTotalSites = (int64_t)1 << 34;

struct GraphEntry {
  int64_t n, phase;
  int cur_in, cur_out;
  int64_t kernels;
  cudaGraphExec_t exec;
};

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

size_t storage_bytes(int prec) { return prec == kF64 ? 8 : (prec == kF32 ? 4 : 2); }

// Steps between the halo exchanges of a lattice held as two halves by a cluster pair
// (measured on GB300: an exchange costs about two steps of a block; with 32 steps the
// halves ran lattices of 5000-7000 sites 5-8 % faster than one ring across the pair).
constexpr int kPairSteps = 32;
static_assert(kPairSteps >= 1 && kPairSteps <= kPairStepsMax, "halo exchange interval");

// One resident-kernel work list: bundles of pieces, launched k steps at a time on `grid` blocks.
struct Lane {
  bool segmented = false;
  int cl = 1;           // blocks per work group (2: thread block clusters)
  double weight = 1.0;  // cost of a bundle relative to a single-block ring bundle (grid split)
  int k = 0, grid = 0, nbundles = 0;
  int kx = 0;  // cl = 2: steps between the halo exchanges of lattice halves
  bool merged = false;  // cl = 2: single-block bundles run two to a pair work group
  int halves = 0;       // lattices held as two halves
  Piece* d_pieces = nullptr;
  int2* d_bundles = nullptr;
  int* d_queue = nullptr;
};

}  // namespace

// An allocator that default-initialises (leaves untouched) trivially constructible
// elements on resize, so that a large run table is written once, by whoever fills it.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
using RunTable = std::vector<RunDesc, NoInitAlloc<RunDesc>>;

struct lb_ks {
  int Q = 0, prec = 0, kernel = 0, cmax = 0;
  int nplanes = 0;         // stored planes: Q, or 1 for the tau = 1 collapse (rho - rhobar)
  bool collapse_resident = false;  // tau = 1 collapse on its register-resident kernel (lanes below)
  bool reservoir = false;  // lattices with fixed-value ends instead of periodic ones
  lb_ks_opts opts{};
  int32_t nruns = 0;
  std::vector<int64_t> N, rho_off;
  RunTable runs_h;
  std::vector<double> mass0_h;
  // runs_h's device-computed fields (rhobar, FP16 scale) and mass0_h hold the device's
  // values: read back when a checkpoint first needs them
  bool tables_on_host = false;
  int64_t total_sites = 0, plane = 0;
  void* fbuf[2] = {nullptr, nullptr};
  int cur = 0;
  RunDesc* d_runs = nullptr;
  Tile* d_plain_tiles = nullptr;
  int n_plain_tiles = 0;
  int plain_tile = kPlainTileMax;  // sites per plain-family tile, also its launches' block size
  Tile* d_stream_tiles = nullptr;
  int n_stream_tiles = 0;
  int32_t* d_stream_tile_begin = nullptr;
  int64_t* d_rho_off = nullptr;
  double* d_stage = nullptr;
  double* d_partials = nullptr;
  double* d_mass0 = nullptr;
  double* d_mass = nullptr;
  double* d_energy = nullptr;
  double* d_delta = nullptr;
  int* d_flags = nullptr;
  int* d_bad_run = nullptr;  // init: the first run whose rho0 holds a non-finite value (nruns: none)
  // resident kernel: up to three lanes, whole lattices first (one block, then cluster
  // pairs), segmented lattices last
  int S = 0, NT = 0, kmax = 0, kseg = 0, nlanes = 0;
  Lane lanes[3];
  double tuned_weight = 0.0;  // lane split weight chosen by the autotuner (0 = not tuned)
  int tuned_cl = 0;           // ring work-group size chosen by the autotuner (0 = not tuned)
  // scheduling
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t side_stream[2] = {nullptr, nullptr};  // lanes 1 and 2 of the resident kernel
  cudaEvent_t ev_fork = nullptr, ev_join[2] = {nullptr, nullptr};
  // lb_ks_rho into pinned host memory: the streaming tiles in kRhoChunks chunks (first
  // tile, first output site of each; the last entry ends the table), each gathered into
  // the staging buffer and copied out while the next one is gathered
  std::vector<std::pair<int, int64_t>> rho_chunks;
  cudaEvent_t ev_rho = nullptr;
  int64_t steps_done = 0;
  int64_t phase = 0;  // steps since the last guard
  int64_t launches = 0;
  uint32_t link_wait_limit = 1u << 22;  // lb_ks_set_link_test
  int link_withhold_step = -1;
  int sticky = LB_KS_OK;
  std::string err = "no error";
  std::vector<GraphEntry> graphs;
  std::vector<void*> allocations;
};

namespace {

int fail(lb_ks* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_ctor_error = msg;
  return code;
}

int cuda_fail(lb_ks* h, cudaError_t e, const char* what) {
  return fail(h, LB_KS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LBKS_CUDA(h, call, what)                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

// No C++ exception crosses the C ABI: the entry points that allocate host memory catch
// whatever escapes and call this from the handler, which turns the exception being
// handled into a status (host allocation failure: LB_KS_ENOMEM) and a message.
int abi_exception(lb_ks* h) noexcept {
  int code = LB_KS_ECUDA;
  const char* msg = "internal error: unexpected C++ exception";
  try {
    throw;
  } catch (const std::bad_alloc&) {
    code = LB_KS_ENOMEM;
    msg = "host allocation failed";
  } catch (...) {
  }
  try {
    if (h) h->err = msg;
    else g_ctor_error = msg;
  } catch (...) {
  }
  return code;
}

// Device memory of the handles comes from one stream-ordered pool per device, created
// on first use, which keeps up to kPoolKeep bytes reserved once they are freed: a
// program that creates and frees handles repeatedly (one per job) then reuses that
// memory instead of paying cudaMalloc and cudaFree for its arenas every time.
constexpr uint64_t kPoolKeep = 4ull << 30;

cudaError_t handle_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
    uint64_t keep = kPoolKeep;
    if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    pools[dev] = pool;
  }
  *out = pools[dev];
  return cudaSuccess;
}

template <typename T>
int dalloc(lb_ks* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = handle_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), count * sizeof(T), pool, h->stream);
  // usable on every stream of the handle (and by synchronous copies) from here on
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (*p) cudaFreeAsync(*p, h->stream);
    *p = nullptr;
    return fail(h, LB_KS_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  h->allocations.push_back(*p);
  return LB_KS_OK;
}

template <typename T>
void dfree(lb_ks* h, T** p) {
  if (!*p) return;
  for (size_t i = 0; i < h->allocations.size(); ++i)
    if (h->allocations[i] == *p) {
      h->allocations.erase(h->allocations.begin() + i);
      break;
    }
  cudaFreeAsync(*p, h->stream);  // (the handle's streams are idle or joined to h->stream here)
  *p = nullptr;
}

Arena arena(lb_ks* h, int which) { return Arena{h->fbuf[which], h->plane}; }

bool valid_opts(const lb_ks_opts& o, std::string* why) {
  if (o.precision < LB_KS_F64 || o.precision > LB_KS_F16S) { *why = "opts.precision must be 0, 1 or 2"; return false; }
  if (o.dm_variant < 0 || o.dm_variant > (LB_KS_DM_PRINTED | LB_KS_WEIGHTS_FULL_INVERSE)) {
    *why = "opts.dm_variant must be 0..3 (LB_KS_DM_* | LB_KS_WEIGHTS_FULL_INVERSE)"; return false;
  }
  if (o.recentre_every < 0) { *why = "opts.recentre_every must be >= 0"; return false; }
  if (o.kernel < LB_KS_KERNEL_AUTO || o.kernel > LB_KS_KERNEL_COLLAPSE) { *why = "opts.kernel must be 0..4"; return false; }
  if (o.kernel == LB_KS_KERNEL_COLLAPSE && o.precision == LB_KS_F16S) { *why = "the tau = 1 collapse stores F64 or F32"; return false; }
  if (o.steps_per_launch < 0) { *why = "opts.steps_per_launch must be >= 0"; return false; }
  if (o.sites_per_thread != 0 && o.sites_per_thread != 4 && o.sites_per_thread != 6 && o.sites_per_thread != 8 &&
      o.sites_per_thread != 12 && o.sites_per_thread != 16 && o.sites_per_thread != 18 && o.sites_per_thread != 20 &&
      o.sites_per_thread != 32) {
    *why = "opts.sites_per_thread must be 0, 4, 6, 8, 12, 16, 18, 20 or 32"; return false;
  }
  if (o.threads_per_block != 0 && (o.threads_per_block < 32 || o.threads_per_block > 512 || o.threads_per_block % 32)) {
    *why = "opts.threads_per_block must be 0 or a multiple of 32 in [32, 512]"; return false;
  }
  if (o.kernel == LB_KS_KERNEL_PLAIN && o.precision == LB_KS_F16S) { *why = "the plain kernel stores F64 or F32"; return false; }
  if (o.cluster_size < 0 || o.cluster_size > 2) { *why = "opts.cluster_size must be 0, 1 or 2"; return false; }
  return true;
}

// ---------------------------------------------------------------- planning

bool has_pair_lattices(const lb_ks* h, int S, int NT);

int default_threads(int prec, int S) {
  if (prec == kF64) return 256;
  return S <= 8 ? 512 : (S <= 12 ? 384 : 256);
}

int upload_lane(lb_ks* h, Lane* L, const std::vector<Piece>& pieces, const Bins& bins, int cl, int k, bool segmented,
                double weight) {
  std::vector<Piece> ordered;
  std::vector<int2> bundles;
  bins.emit(pieces, &ordered, &bundles);
  L->cl = cl;
  L->segmented = segmented;
  L->weight = weight;
  int rc;
  if ((rc = dalloc(h, &L->d_pieces, ordered.size()))) return rc;
  if ((rc = dalloc(h, &L->d_bundles, bundles.size()))) return rc;
  if ((rc = dalloc(h, &L->d_queue, 1))) return rc;
  LBKS_CUDA(h, cudaMemcpy(L->d_pieces, ordered.data(), ordered.size() * sizeof(Piece), cudaMemcpyHostToDevice), "upload pieces");
  LBKS_CUDA(h, cudaMemcpy(L->d_bundles, bundles.data(), bundles.size() * sizeof(int2), cudaMemcpyHostToDevice), "upload bundles");
  L->k = k;
  L->nbundles = (int)bundles.size();
  return LB_KS_OK;
}

// The kernels' launch preparation (dynamic shared memory opt-in, resident blocks per SM
// or clusters at once), done once per device, kind (0 resident, 1 collapse, 2 cluster
// pairs), scheme, storage and tiling: the attribute set by it stays with the function.
cudaError_t prepared(int kind, int Q, int prec, int S, int NT, int* out) {
  static std::mutex mu;
  static std::map<std::array<int, 6>, int> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::array<int, 6> key{dev, kind, Q, prec, S, NT};
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find(key);
  if (it == done.end()) {
    int v = 0;
    e = kind == 0 ? resident_prepare(Q, prec, S, NT, &v)
                  : (kind == 1 ? collapse_resident_prepare(Q, prec, S, NT, &v) : resident_cluster_prepare(Q, prec, S, NT, &v));
    if (e != cudaSuccess) return e;  // not kept: the caller clears the error and tries another tiling
    it = done.emplace(key, v).first;
  }
  *out = it->second;
  return cudaSuccess;
}

// Resident kernel plan.  Whole lattices (rings) run k_ring steps per launch; lattices
// cut into segments run k_seg-step launches (their halo grows with the steps per
// launch).  Rings of up to NT S sites run in single-block work groups; with cl = 2,
// rings of up to 2 NT S sites run in cluster pairs, as two haloed halves (halo
// exchanged every kx steps) when a half with its halos fits a block, else as one ring
// across both blocks, with smaller rings filling the pairs' spare threads, instead of
// being cut into segments.  The kinds present run as concurrent lanes on disjoint sets
// of blocks, on their own streams, sized so that all finish a chunk of steps at about
// the same time; or (merge = 1, or by default when the pairs hold more threads than the
// single blocks) the single-block bundles go two to a pair on the pair lane's queue.
// S_force / NT_force / cl_force > 0 pin the tiling and kx_force >= 0 the exchange
// interval (0: no halves) for autotuner trials; lane_weight is the cost of a pair or
// segment bundle relative to a single-block ring bundle, used to split the blocks.
int setup_resident(lb_ks* h, bool required, int S_force = 0, int NT_force = 0, double lane_weight = 1.25,
                   int cl_force = 0, int merge = -1, int kx_force = -1) {
  const bool col = h->nplanes == 1;  // the tau = 1 collapse's resident kernel
  auto supported = [&](int S, int NT) {
    return col ? collapse_resident_supported(h->Q, h->prec, S, NT) : resident_supported(h->Q, h->prec, S, NT);
  };
  std::vector<int> cand;
  if (S_force) cand.push_back(S_force);
  else if (h->opts.sites_per_thread) cand.push_back(h->opts.sites_per_thread);
  else if (col) cand = h->prec == kF64 ? std::vector<int>{16, 8} : std::vector<int>{32, 16, 8};
  else if (h->prec == kF64) cand = {8, 6, 4};
  else cand = {20, 18, 12, 8, 16, 6, 4};
  const int R = h->opts.recentre_every;
  for (int S : cand) {
    const int NT = NT_force ? NT_force
                            : (h->opts.threads_per_block ? h->opts.threads_per_block
                                                         : (col ? 256 : default_threads(h->prec, S)));
    if (!supported(S, NT)) continue;
    const int kring = h->opts.steps_per_launch ? h->opts.steps_per_launch : (R > 0 ? std::min(R, 1000) : 1000);
    int kseg = h->opts.steps_per_launch ? h->opts.steps_per_launch
                                        : std::max(1, (int)((int64_t)NT * S / (20 * h->cmax)));
    kseg = std::min(kseg, kring);
    // default: cluster pairs when some lattice needs more than one block and fits two
    int cl = cl_force ? cl_force : h->opts.cluster_size;
    if (cl == 0) cl = has_pair_lattices(h, S, NT) ? 2 : 1;
    if (col) cl = 1;  // no cluster variant of the collapse
    std::vector<Piece> rings, segs;
    const int kx = cl == 2 ? (kx_force >= 0 ? kx_force : kPairSteps) : 0;
    if (!plan_pieces(h->N, h->cmax, S, NT, cl * NT, kseg, kx, &rings, &segs)) continue;
    Bins blocks, pairs, segbins;
    pack_rings(rings, NT, &blocks, &pairs);
    // default: one queue of pair work groups when the pairs hold most of the threads
    int pair_thr = 0, block_thr = 0;
    for (size_t b = 0; b < pairs.used.size(); ++b) pair_thr += pairs.used0[b] + pairs.used[b] - NT;
    for (int u : blocks.used) block_thr += u;
    const bool do_merge = merge >= 0 ? merge != 0 : pair_thr > block_thr;
    bool merged = false;
    if (do_merge && cl == 2 && !pairs.used.empty() && !blocks.used.empty()) {
      merge_blocks_into_pairs(rings, NT, blocks, &pairs);
      blocks = Bins{};
      merged = true;
    }
    int nhalves = 0;
    for (const Piece& p : rings) nhalves += p.halo > 0 ? 1 : 0;
    pack_blocks(segs, NT, &segbins);
    int bps = 0, max_clusters = 0;
    cudaError_t e = prepared(col ? 1 : 0, h->Q, h->prec, S, NT, &bps);
    if (e != cudaSuccess || bps < 1) { cudaGetLastError(); continue; }
    if (!pairs.used.empty()) {
      e = prepared(2, h->Q, h->prec, S, NT, &max_clusters);
      if (e != cudaSuccess || max_clusters < 1) { cudaGetLastError(); continue; }
    }
    int dev = 0, sms = 0;
    LBKS_CUDA(h, cudaGetDevice(&dev), "cudaGetDevice");
    LBKS_CUDA(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    const int slots = bps * sms;  // resident blocks
    int rc;
    h->nlanes = 0;
    if (!blocks.used.empty()) {
      if ((rc = upload_lane(h, &h->lanes[h->nlanes++], rings, blocks, 1, kring, false, 1.0))) return rc;
    }
    if (!pairs.used.empty()) {
      if ((rc = upload_lane(h, &h->lanes[h->nlanes++], rings, pairs, 2, kring, false, lane_weight))) return rc;
      h->lanes[h->nlanes - 1].kx = nhalves ? kx : 0;
      h->lanes[h->nlanes - 1].merged = merged;
      h->lanes[h->nlanes - 1].halves = nhalves / 2;
    }
    if (!segbins.used.empty()) {
      if ((rc = upload_lane(h, &h->lanes[h->nlanes++], segs, segbins, 1, kseg, true, lane_weight))) return rc;
    }
    // Split the resident blocks between the lanes: lane l finishes a chunk of steps in
    // about weight_l ceil(B_l / G_l) rounds of bundles on G_l work groups of cl_l blocks;
    // work groups go one at a time to the lane that would finish last.
    int used = 0;
    for (int l = 0; l < h->nlanes; ++l) {
      h->lanes[l].grid = 1;
      used += h->lanes[l].cl;
    }
    for (;;) {
      int worst = -1;
      double worstT = -1.0;
      for (int l = 0; l < h->nlanes; ++l) {
        const Lane& L = h->lanes[l];
        const double T = L.weight * ((L.nbundles + L.grid - 1) / L.grid);
        if (T > worstT) { worstT = T; worst = l; }
      }
      Lane& W = h->lanes[worst];
      const int cap = W.cl == 2 ? max_clusters : slots;
      if (W.grid >= W.nbundles || W.grid >= cap || used + W.cl > slots) break;
      ++W.grid;
      used += W.cl;
    }
    h->S = S;
    h->NT = NT;
    h->kmax = h->lanes[0].segmented ? kseg : kring;
    h->kseg = kseg;
    return LB_KS_OK;
  }
  if (required) return fail(h, LB_KS_EINVAL, "resident kernel cannot hold these lattices with the requested tiling");
  return 1;  // not possible; caller picks another family
}

// k steps of one lane starting from arena `from`, in launches of at most lane.k steps,
// alternating arenas.  Returns the arena holding the result; a single launch may write
// in place (to == from) when `in_place` is set.
int issue_lane(lb_ks* h, const Lane& L, int64_t k, int from, bool in_place, cudaStream_t s, int64_t* nk, int* to) {
  int cur = from;
  while (k > 0) {
    const int64_t kk = std::min<int64_t>(k, L.k);
    const int dst = (in_place && kk == k && cur == from) ? cur : 1 - cur;
    LBKS_CUDA(h, cudaMemsetAsync(L.d_queue, 0, sizeof(int), s), "queue reset");
    ResidentLaunch RL{h->Q, h->prec, h->S, h->NT, arena(h, cur), arena(h, dst), h->d_runs,
                      L.d_pieces, L.d_bundles, L.nbundles, L.d_queue, (int)kk, L.grid, L.cl, h->d_flags,
                      h->nplanes == 1, L.kx, h->link_wait_limit, h->link_withhold_step};
    LBKS_CUDA(h, launch_resident(RL, s), "resident step");
    *nk += 1;
    cur = dst;
    k -= kk;
  }
  *to = cur;
  return LB_KS_OK;
}

// ---------------------------------------------------------------- step scheduling

int issue_guard(lb_ks* h, cudaStream_t s, bool recentre, int64_t* nk) {
  LBKS_CUDA(h, launch_mass_partials(h->nplanes, h->prec, arena(h, h->cur), h->d_runs, h->d_stream_tiles,
                                    h->n_stream_tiles, h->d_partials, s), "mass partials");
  LBKS_CUDA(h, launch_mass_finalize(h->nruns, h->d_stream_tile_begin, h->d_partials, h->d_runs, h->d_mass0, h->d_mass,
                                    h->d_energy, recentre ? h->d_delta : nullptr, h->d_flags, s), "mass finalize");
  *nk += 2;
  if (recentre) {
    LBKS_CUDA(h, launch_recentre(h->prec, arena(h, h->cur), h->d_runs, h->d_stream_tiles, h->n_stream_tiles,
                                 h->d_delta, s), "recentre");
    *nk += 1;
  }
  return LB_KS_OK;
}

// Issue n steps on stream s, updating cur / phase / steps_done as the work will.
int issue_steps(lb_ks* h, int64_t n, cudaStream_t s, int64_t* nk) {
  const int64_t R = h->opts.recentre_every;
  while (n > 0) {
    int64_t k = 1;
    if (h->kernel == LB_KS_KERNEL_RESIDENT || h->collapse_resident) {
      k = std::min<int64_t>(n, h->kmax);
      if (R > 0) k = std::min<int64_t>(k, R - h->phase);
      int to = h->cur, rc;
      if (h->nlanes == 1) {
        if ((rc = issue_lane(h, h->lanes[0], k, h->cur, false, s, nk, &to))) return rc;
      } else {
        // lane 0 on s, the others on their side streams.  Whole-lattice lanes make one
        // launch, in place when the segment lane (if any) makes an even number of
        // launches, so that all lanes end in the same arena.
        int64_t mseg = 1;
        for (int l = 0; l < h->nlanes; ++l)
          if (h->lanes[l].segmented) mseg = (k + h->lanes[l].k - 1) / h->lanes[l].k;
        const bool has_seg = h->lanes[h->nlanes - 1].segmented;
        LBKS_CUDA(h, cudaEventRecord(h->ev_fork, s), "fork");
        int to_l[3] = {h->cur, h->cur, h->cur};
        for (int l = 0; l < h->nlanes; ++l) {
          cudaStream_t sl = l == 0 ? s : h->side_stream[l - 1];
          if (l > 0) LBKS_CUDA(h, cudaStreamWaitEvent(sl, h->ev_fork, 0), "fork wait");
          Lane L = h->lanes[l];
          if (!L.segmented) L.k = (int)k;
          if ((rc = issue_lane(h, L, k, h->cur, !L.segmented && has_seg && (mseg % 2) == 0, sl, nk, &to_l[l]))) return rc;
          if (l > 0) LBKS_CUDA(h, cudaEventRecord(h->ev_join[l - 1], sl), "join");
        }
        for (int l = 1; l < h->nlanes; ++l) {
          LBKS_CUDA(h, cudaStreamWaitEvent(s, h->ev_join[l - 1], 0), "join wait");
          if (to_l[l] != to_l[0]) return fail(h, LB_KS_ECUDA, "internal: lanes ended in different arenas");
        }
        to = to_l[0];
      }
      h->cur = to;
    } else {
      if (h->kernel == LB_KS_KERNEL_COLLAPSE) {
        LBKS_CUDA(h, launch_collapse_step(h->Q, h->prec, arena(h, h->cur), arena(h, 1 - h->cur), h->d_runs,
                                          h->d_stream_tiles, h->n_stream_tiles, s), "collapse step");
      } else if (h->reservoir) {
        LBKS_CUDA(h, launch_reservoir_step(h->Q, h->prec, arena(h, h->cur), arena(h, 1 - h->cur), h->d_runs,
                                           h->d_plain_tiles, h->n_plain_tiles, h->plain_tile, 0, s), "reservoir step");
      } else if (h->kernel == LB_KS_KERNEL_STREAM) {
        LBKS_CUDA(h, launch_stream_step(h->Q, h->prec, arena(h, h->cur), arena(h, 1 - h->cur), h->d_runs,
                                        h->d_stream_tiles, h->n_stream_tiles, s), "stream step");
      } else {
        LBKS_CUDA(h, launch_plain_step(h->Q, h->prec, arena(h, h->cur), arena(h, 1 - h->cur), h->d_runs,
                                       h->d_plain_tiles, h->n_plain_tiles, h->plain_tile, s), "plain step");
      }
      *nk += 1;
      h->cur = 1 - h->cur;
    }
    n -= k;
    h->steps_done += k;
    if (R > 0) {
      h->phase += k;
      if (h->phase == R) {
        h->phase = 0;
        int rc = issue_guard(h, s, true, nk);
        if (rc) return rc;
      }
    }
  }
  return LB_KS_OK;
}

int run_chunk_graph(lb_ks* h, int64_t n) {
  for (auto& g : h->graphs) {
    if (g.n == n && g.phase == h->phase && g.cur_in == h->cur) {
      LBKS_CUDA(h, cudaGraphLaunch(g.exec, h->stream), "graph launch");
      h->cur = g.cur_out;
      h->steps_done += n;
      const int64_t R = h->opts.recentre_every;
      if (R > 0) h->phase = (h->phase + n) % R;
      h->launches += g.kernels;
      return LB_KS_OK;
    }
  }
  GraphEntry ge{};
  ge.n = n;
  ge.phase = h->phase;
  ge.cur_in = h->cur;
  LBKS_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int64_t nk = 0;
  const int rc = issue_steps(h, n, h->cap_stream, &nk);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &graph);
  if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
  if (ee != cudaSuccess) return cuda_fail(h, ee, "end capture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return cuda_fail(h, ie, "graph instantiate");
  ge.cur_out = h->cur;
  ge.kernels = nk;
  ge.exec = exec;
  if (h->graphs.size() >= 8) {
    cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  h->graphs.push_back(ge);
  LBKS_CUDA(h, cudaGraphLaunch(exec, h->stream), "graph launch");
  h->launches += nk;
  return LB_KS_OK;
}

void release_lanes(lb_ks* h) {
  for (Lane& L : h->lanes) {
    dfree(h, &L.d_pieces);
    dfree(h, &L.d_bundles);
    dfree(h, &L.d_queue);
    L = Lane{};
  }
  h->nlanes = 0;
}

// True if some lattice is longer than one block of NT threads x S sites holds but
// fits a cluster pair.
bool has_pair_lattices(const lb_ks* h, int S, int NT) {
  for (int64_t N : h->N)
    if (N > (int64_t)NT * S && N <= 2LL * NT * S) return true;
  return false;
}

// Autotuner of the resident kernel: times a few tilings (sites per thread, threads per
// block), ring work-group sizes (one block or a cluster pair) and lane splits on this
// handle's own lattices for a short run, and keeps the fastest.  Runs before the state
// is initialised, on the zeroed arenas (the kernel's work does not depend on the values).
int autotune_resident(lb_ks* h) {
  struct Cand { int S, NT; double w; int cl; int merge; int kx; };
  std::vector<Cand> cands;
  std::vector<std::pair<int, int>> tilings;
  const bool col = h->nplanes == 1;  // the tau = 1 collapse's resident kernel
  if (h->opts.sites_per_thread) {
    tilings.push_back({h->opts.sites_per_thread, h->opts.threads_per_block});
  } else if (col) {
    if (h->prec == kF64) tilings = {{16, 256}, {16, 512}, {8, 512}};
    else tilings = {{32, 256}, {32, 512}, {16, 512}};
  } else if (h->prec == kF64) {
    tilings = {{8, 256}, {6, 256}, {4, 256}};
  } else {
    tilings = {{20, 256}, {18, 256}, {12, 384}, {16, 256}, {8, 512}};
  }
  for (auto& tl : tilings) {
    const int NT = tl.second ? tl.second : (col ? 256 : default_threads(h->prec, tl.first));
    for (int cl : {2, 1}) {
      if (col && cl == 2) continue;
      if (h->opts.cluster_size && cl != h->opts.cluster_size) continue;
      if (cl == 2 && !has_pair_lattices(h, tl.first, NT)) continue;  // same plan as cl = 1
      for (int kx : {kPairSteps, 0}) {
        if (cl == 1 && kx != 0) continue;
        for (double w : {1.0, 1.25, 1.6}) cands.push_back({tl.first, tl.second, w, cl, 0, kx});
        if (cl == 2) cands.push_back({tl.first, tl.second, 1.0, cl, 1, kx});
      }
    }
  }
  if (cands.empty()) return LB_KS_OK;  // keep the plan made before tuning
  // one full whole-lattice launch per trial (500 steps, or fewer when the guard
  // interval or steps_per_launch is shorter), so the launch edges weigh as in a run
  const int64_t trial = std::max<int64_t>(2 * h->kseg, std::min<int64_t>(h->kmax, 500));
  cudaEvent_t e0, e1;
  LBKS_CUDA(h, cudaEventCreate(&e0), "tuner event");
  LBKS_CUDA(h, cudaEventCreate(&e1), "tuner event");
  double best_ms = 1e300;
  Cand best = cands.front();
  int rc = LB_KS_OK;
  for (const Cand& c : cands) {
    release_lanes(h);
    if (setup_resident(h, false, c.S, c.NT, c.w, c.cl, c.merge, c.kx) != LB_KS_OK) { cudaGetLastError(); continue; }
    if (h->nlanes < 2 && c.w != 1.0) continue;  // the split weight only matters with more than one lane
    int64_t nk = 0;
    for (int rep = 0; rep < 2 && rc == LB_KS_OK; ++rep) {  // first repetition warms up
      cudaEventRecord(e0, h->stream);
      rc = issue_steps(h, trial, h->stream, &nk);
      cudaEventRecord(e1, h->stream);
    }
    if (rc != LB_KS_OK) break;
    cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce != cudaSuccess) { rc = cuda_fail(h, ce, "tuner timing"); break; }
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != LB_KS_OK) return rc;
  release_lanes(h);
  if (best_ms < 1e300) {
    if ((rc = setup_resident(h, true, best.S, best.NT, best.w, best.cl, best.merge, best.kx)) != LB_KS_OK) return rc;
    h->tuned_weight = best.w;
    h->tuned_cl = best.cl;
  } else if ((rc = setup_resident(h, true)) != LB_KS_OK) {
    return rc;
  }
  // the trials advanced the (zero) state: start the real run from the first arena
  h->cur = 0;
  h->steps_done = 0;
  h->phase = 0;
  h->launches = 0;
  LBKS_CUDA(h, cudaMemsetAsync(h->d_flags, 0, sizeof(int), h->stream), "clear flags");
  return LB_KS_OK;
}

int check_flags(lb_ks* h) {
  int flag = 0;
  LBKS_CUDA(h, cudaMemcpy(&flag, h->d_flags, sizeof(int), cudaMemcpyDeviceToHost), "read flags");
  if (flag & 2) {
    h->sticky = LB_KS_ETIMEOUT;
    return fail(h, LB_KS_ETIMEOUT, "a bounded wait between the two blocks of a resident cluster ran out");
  }
  if (flag) {
    h->sticky = LB_KS_EUNSTABLE;
    return fail(h, LB_KS_EUNSTABLE, "non-finite FP64 mass at a guard step (the run went unstable)");
  }
  return LB_KS_OK;
}

// Linear stability check (lb_ks_max_growth, nk = 128, about rho = 0) of every distinct
// (dx, dt, tau) when a batch has at most 64 of them; a run whose growth rate exceeds
// 1.05 x 1/4 leaves a warning in last_error (the handle is still created).
void warn_if_linearly_unstable(lb_ks* h, const double* L, const double* dt, const double* tau) {
  std::vector<std::array<double, 3>> seen;
  for (int32_t r = 0; r < h->nruns; ++r) {
    const double dx = L[r] / (double)(h->reservoir ? h->N[r] - 1 : h->N[r]);
    const std::array<double, 3> key{dx, dt[r], tau[r]};
    if (std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
    seen.push_back(key);
    if (seen.size() > 64) return;
  }
  int bad = 0, first = -1;
  double worst = 0.0;
  for (int32_t r = 0; r < h->nruns; ++r) {
    const double dx = L[r] / (double)(h->reservoir ? h->N[r] - 1 : h->N[r]);
    double g = 0.0;
    if (lb_ks_max_growth(h->Q, dx, dt[r], tau[r], h->opts.dm_variant, 0.0, 128, &g) != LB_KS_OK) continue;
    if (g > 1.05 * 0.25) {
      if (bad++ == 0) { first = r; worst = g; }
    }
  }
  if (bad)
    h->err = "warning: " + std::to_string(bad) + " run(s) linearly unstable (run " + std::to_string(first) +
             ": growth rate " + std::to_string(worst) + " per unit time > 1.05 x 1/4)";
}

// The constructor.  h holds the handle while it is being built, so that the caller can
// release it if an exception escapes; bail() releases it on a failed status.
int create_body(lb_ks*& h, lb_ks_t** out, int scheme, int32_t nruns, const int64_t* N, const double* L,
                const double* dt, const double* tau, const double* rho0, const lb_ks_opts* opts,
                const double* rho_left, const double* rho_right) {
  if (!out) return fail(nullptr, LB_KS_EINVAL, "h must not be NULL");
  *out = nullptr;
  const bool reservoir = rho_left != nullptr;
  if (reservoir) {
    if (!rho_right) return fail(nullptr, LB_KS_EINVAL, "rho_left and rho_right must both be given");
    for (int32_t r = 0; r < nruns; ++r)
      if (!std::isfinite(rho_left[r]) || !std::isfinite(rho_right[r]))
        return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": reservoir values must be finite");
    if (opts && (opts->kernel == LB_KS_KERNEL_STREAM || opts->kernel == LB_KS_KERNEL_RESIDENT))
      return fail(nullptr, LB_KS_EINVAL, "reservoir ends run on the plain kernel family only");
    if (opts && opts->recentre_every != 0)
      return fail(nullptr, LB_KS_EINVAL, "reservoir ends exchange mass: recentre_every must be 0");
  }
  if (scheme != LB_KS_D1Q5 && scheme != LB_KS_D1Q7) return fail(nullptr, LB_KS_EINVAL, "scheme must be 5 or 7");
  if (nruns < 1) return fail(nullptr, LB_KS_EINVAL, "nruns must be >= 1");
  if (!N || !L || !dt || !tau || !rho0) return fail(nullptr, LB_KS_EINVAL, "NULL argument");
  lb_ks_opts o;
  lb_ks_default_opts(&o);
  if (opts) o = *opts;
  std::string why;
  if (!valid_opts(o, &why)) return fail(nullptr, LB_KS_EINVAL, why);
  const int cmax = (scheme - 1) / 2;
  int64_t total = 0;
  for (int32_t r = 0; r < nruns; ++r) {
    if (N[r] < 2 * cmax + 1 || N[r] > (int64_t)1 << 30)
      return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": N must be in [2 c_max + 1, 2^30]");
    if (!(L[r] > 0.0) || !std::isfinite(L[r])) return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": L must be > 0");
    if (!(dt[r] > 0.0) || !std::isfinite(dt[r])) return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": dt must be > 0");
    if (!(tau[r] >= 1.0) || !std::isfinite(tau[r])) return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": tau must be >= 1");
    if (o.kernel == LB_KS_KERNEL_COLLAPSE && tau[r] != 1.0)
      return fail(nullptr, LB_KS_EINVAL, "run " + std::to_string(r) + ": the collapse kernel needs tau = 1");
    total += N[r];
    if (total > kMaxTotalSites)
      return fail(nullptr, LB_KS_EINVAL, "the runs hold more than 2^34 sites in all (more than device memory holds)");
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(nullptr, LB_KS_ECUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(ce));
  }

  h = new (std::nothrow) lb_ks();
  if (!h) return fail(nullptr, LB_KS_ENOMEM, "host allocation failed");
  auto bail = [&](int rc) {
    g_ctor_error = h->err;
    lb_ks* dead = h;
    h = nullptr;
    lb_ks_free(dead);
    return rc;
  };
  h->Q = scheme;
  h->cmax = cmax;
  h->nplanes = o.kernel == LB_KS_KERNEL_COLLAPSE ? 1 : scheme;
  h->prec = o.precision;
  h->opts = o;
  h->nruns = nruns;
  h->stream = static_cast<cudaStream_t>(o.stream);
  h->N.assign(N, N + nruns);
  h->total_sites = total;

  // rho0 goes up first, on the capture stream (idle until the first graph capture), so
  // that the copy runs while the host computes the run table and plans below; the
  // populations' clearing and rho0's statistics follow it there.  The handle's stream
  // waits for them (stats.ev) before its first kernel that uses the populations or the
  // run table, so that the stream synchronisations of planning's allocations do not.
  // create() waits for the copy before it returns, so the caller's buffer is free again
  // when it does.
  int rc;
  struct CopyWait {
    cudaEvent_t ev = nullptr;
    ~CopyWait() {
      if (ev) {
        cudaEventSynchronize(ev);
        cudaEventDestroy(ev);
      }
    }
  } staged;
  if ((rc = dalloc(h, &h->d_stage, (size_t)total))) return bail(rc);
  if ((ce = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(h, ce, "create capture stream"));
  cudaStream_t const is = h->cap_stream;
  if ((ce = cudaMemcpyAsync(h->d_stage, rho0, sizeof(double) * (size_t)total, cudaMemcpyDefault, is)) !=
          cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&staged.ev, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventRecord(staged.ev, is)) != cudaSuccess)
    return bail(cuda_fail(h, ce, "upload rho0"));

  // Per run on the host: the coefficients and the arena layout.  The statistics of rho0
  // (finiteness, mass M0, mean rhobar, FP16 scale) are computed on the device after its
  // upload above, while the host plans.
  h->rho_off.resize(nruns + 1);
  h->rho_off[0] = 0;
  for (int32_t r = 0; r < nruns; ++r) h->rho_off[r + 1] = h->rho_off[r] + N[r];
  h->mass0_h.assign(nruns, 0.0);
  // Each descriptor is written once, in place (the table's allocator does not zero it).
  // One thread: spreading the runs over a few host threads saved ~0.1 ms on 4096 runs,
  // but a new thread sometimes started milliseconds late.
  h->runs_h.resize(nruns);
  int64_t off = 0;
  for (int32_t r = 0; r < nruns; ++r) {
    RunDesc& d = h->runs_h[r];
    std::memset(&d, 0, sizeof(d));
    double A[7], B[7];
    // periodic: N sites on [0, L); reservoir ends: N nodes on [0, L] including both ends
    const double dx = L[r] / (double)(reservoir ? N[r] - 1 : N[r]);
    if (lb_ks_params(scheme, dx, dt[r], tau[r], o.dm_variant, A, B, nullptr) != LB_KS_OK)
      return bail(fail(h, LB_KS_EINVAL, "run " + std::to_string(r) + ": coefficients are not finite"));
    const double w = 1.0 / tau[r];
    d.N = N[r];
    d.reservoir = reservoir ? 1 : 0;
    d.rho_left = reservoir ? rho_left[r] : 0.0;
    d.rho_right = reservoir ? rho_right[r] : 0.0;
    for (int i = 0; i < scheme; ++i) {
      d.A[i] = A[i];
      d.B[i] = B[i];
      d.a[i] = A[i] * w;
      d.b[i] = B[i] * w;
      d.af[i] = (float)d.a[i];
      d.bf[i] = (float)d.b[i];
    }
    d.r = 1.0 - w;
    d.rf = (float)d.r;
    d.rhobar = 0.0;  // rhobar and the FP16 scale: set on the device
    d.scale = d.inv_scale = 1.0;
    d.scalef = d.inv_scalef = 1.0f;
    const int64_t ghost = reservoir ? cmax : 0;  // ghost nodes stored before node 0 and after node N-1
    d.off = off + ghost;
    off += align_up(N[r] + 2 * ghost, kAlign);
  }
  h->plane = std::max<int64_t>(off, kAlign);

  // Tiles.  The streaming tiles (also those of the guard, the statistics of rho0 and the
  // gathers) always; the plain family's only when a kernel that uses them runs (the
  // plain and reservoir steps, the collapse's initialisation).
  std::vector<Tile> st;
  std::vector<int32_t> st_begin(nruns + 1);
  const int TS = stream_tile_sites();
  for (int32_t r = 0; r < nruns; ++r) {
    st_begin[r] = (int32_t)st.size();
    for (int64_t x = 0; x < N[r]; x += TS) st.push_back(Tile{r, (int32_t)x, (int32_t)std::min<int64_t>(TS, N[r] - x), 0});
  }
  st_begin[nruns] = (int32_t)st.size();
  h->n_stream_tiles = (int)st.size();
  {
    constexpr int kRhoChunks = 8;
    const int nt = (int)st.size();
    for (int c = 0; c <= kRhoChunks; ++c) {
      const int t = (int)((int64_t)nt * c / kRhoChunks);
      const int64_t o0 = t < nt ? h->rho_off[st[t].run] + st[t].x0 : total;
      if (h->rho_chunks.empty() || h->rho_chunks.back().first != t) h->rho_chunks.emplace_back(t, o0);
    }
  }
  auto plain_tiles = [&]() -> int {
    if (h->d_plain_tiles) return LB_KS_OK;
    int dev = 0, sms = 0;
    cudaError_t e1 = cudaGetDevice(&dev);
    if (e1 == cudaSuccess) e1 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e1 != cudaSuccess) return cuda_fail(h, e1, "cudaDeviceGetAttribute");
    int tile = 0;
    const std::vector<Tile> pt = lbks::plan::plain_tiles(h->N, reservoir, cmax, sms, &tile);
    int rc2;
    if ((rc2 = dalloc(h, &h->d_plain_tiles, pt.size()))) return rc2;
    cudaError_t e2 = cudaMemcpy(h->d_plain_tiles, pt.data(), sizeof(Tile) * pt.size(), cudaMemcpyHostToDevice);
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "upload plain tiles");
    h->n_plain_tiles = (int)pt.size();
    h->plain_tile = tile;
    return LB_KS_OK;
  };

  const size_t fbytes = storage_bytes(h->prec) * (size_t)h->nplanes * (size_t)h->plane;
  for (int b = 0; b < 2; ++b) {
    unsigned char* p = nullptr;
    if ((rc = dalloc(h, &p, fbytes))) return bail(rc);
    h->fbuf[b] = p;
  }
  if ((rc = dalloc(h, &h->d_runs, nruns))) return bail(rc);
  if ((rc = dalloc(h, &h->d_stream_tiles, st.size()))) return bail(rc);
  if ((rc = dalloc(h, &h->d_stream_tile_begin, st_begin.size()))) return bail(rc);
  if ((rc = dalloc(h, &h->d_rho_off, h->rho_off.size()))) return bail(rc);
  if ((rc = dalloc(h, &h->d_partials, 2 * st.size()))) return bail(rc);
  if ((rc = dalloc(h, &h->d_mass0, nruns))) return bail(rc);
  if ((rc = dalloc(h, &h->d_mass, nruns))) return bail(rc);
  if ((rc = dalloc(h, &h->d_energy, nruns))) return bail(rc);
  if ((rc = dalloc(h, &h->d_delta, nruns))) return bail(rc);
  if ((rc = dalloc(h, &h->d_flags, 1))) return bail(rc);
  if ((rc = dalloc(h, &h->d_bad_run, 1))) return bail(rc);
  auto up = [&](void* dst, const void* src, size_t bytes) { return cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice); };
  if ((ce = up(h->d_runs, h->runs_h.data(), sizeof(RunDesc) * nruns)) != cudaSuccess ||
      (ce = up(h->d_stream_tiles, st.data(), sizeof(Tile) * st.size())) != cudaSuccess ||
      (ce = up(h->d_stream_tile_begin, st_begin.data(), sizeof(int32_t) * st_begin.size())) != cudaSuccess ||
      (ce = up(h->d_rho_off, h->rho_off.data(), sizeof(int64_t) * h->rho_off.size())) != cudaSuccess ||
      (ce = cudaMemset(h->d_flags, 0, sizeof(int))) != cudaSuccess)
    return bail(cuda_fail(h, ce, "upload"));
  for (int b = 0; b < 2; ++b)
    if ((ce = cudaMemsetAsync(h->fbuf[b], 0, fbytes, is)) != cudaSuccess)
      return bail(cuda_fail(h, ce, "clear populations"));
  // rho0's statistics on the device, read back after planning (once the event after
  // them has completed)
  CopyWait stats;
  const int no_bad = nruns;
  if ((ce = cudaMemcpyAsync(h->d_bad_run, &no_bad, sizeof(int), cudaMemcpyHostToDevice, is)) != cudaSuccess ||
      (ce = launch_init_stats(scheme, h->prec, nruns, h->d_stage, h->d_rho_off, h->d_runs, h->d_stream_tiles,
                              h->n_stream_tiles, h->d_stream_tile_begin, h->d_partials, h->d_mass0, h->d_bad_run,
                              is)) != cudaSuccess ||
      (ce = cudaEventCreateWithFlags(&stats.ev, cudaEventDisableTiming)) != cudaSuccess ||
      (ce = cudaEventRecord(stats.ev, is)) != cudaSuccess)
    return bail(cuda_fail(h, ce, "rho0 statistics"));
  bool init_joined = false;
  auto join_init = [&]() -> cudaError_t {  // the handle's stream after the capture stream's init work
    if (init_joined) return cudaSuccess;
    init_joined = true;
    return cudaStreamWaitEvent(h->stream, stats.ev, 0);
  };

  // Kernel family.
  int kern = o.kernel;
  h->reservoir = reservoir;
  if (kern == LB_KS_KERNEL_COLLAPSE) {
    if (collapse_tile_sites() != TS) return bail(fail(h, LB_KS_ECUDA, "internal: collapse and streaming tiles differ"));
    // periodic lattices: the register-resident collapse (many steps per launch), unless
    // one step per launch is asked for; reservoir ends: the streaming collapse
    if (!reservoir && o.steps_per_launch != 1) {
      rc = setup_resident(h, false);
      if (rc < 0) return bail(rc);
      h->collapse_resident = rc == 0;
    }
  } else if (reservoir) {
    kern = LB_KS_KERNEL_PLAIN;
  } else if (kern == LB_KS_KERNEL_AUTO || kern == LB_KS_KERNEL_RESIDENT) {
    rc = setup_resident(h, kern == LB_KS_KERNEL_RESIDENT);
    if (rc < 0) return bail(rc);
    kern = rc == 0 ? LB_KS_KERNEL_RESIDENT : (h->prec == kF64 ? LB_KS_KERNEL_PLAIN : LB_KS_KERNEL_STREAM);
  }
  h->kernel = kern;
  if (kern == LB_KS_KERNEL_STREAM && (ce = stream_prepare(scheme, h->prec)) != cudaSuccess)
    return bail(cuda_fail(h, ce, "stream kernel setup"));
  // streams and events for concurrent lanes, when the plan has several (or the tuner
  // may choose one that does)
  if ((kern == LB_KS_KERNEL_RESIDENT || h->collapse_resident) && (o.autotune || h->nlanes > 1)) {
    for (int l = 0; l < 2 && ce == cudaSuccess; ++l)
      if ((ce = cudaStreamCreateWithFlags(&h->side_stream[l], cudaStreamNonBlocking)) == cudaSuccess)
        ce = cudaEventCreateWithFlags(&h->ev_join[l], cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(cuda_fail(h, ce, "create lane stream"));
    if (o.autotune && (ce = join_init()) != cudaSuccess) return bail(cuda_fail(h, ce, "join init"));
    if (o.autotune && (rc = autotune_resident(h)) != LB_KS_OK) return bail(rc);
  }
  if (h->nlanes > 1 && !h->ev_fork) return bail(fail(h, LB_KS_ECUDA, "internal: lanes without their streams"));

  if ((kern == LB_KS_KERNEL_COLLAPSE || kern == LB_KS_KERNEL_PLAIN || reservoir) && (rc = plain_tiles()) != LB_KS_OK)
    return bail(rc);
  if ((ce = join_init()) != cudaSuccess) return bail(cuda_fail(h, ce, "join init"));
  if (kern == LB_KS_KERNEL_COLLAPSE) {
    // rho - rhobar in both arenas (reservoir ends and ghosts keep their values in both)
    for (int b = 0; b < 2; ++b)
      if ((ce = launch_collapse_init(h->prec, arena(h, b), h->d_runs, h->d_plain_tiles, h->n_plain_tiles, h->d_stage,
                                     h->d_rho_off, h->stream)) != cudaSuccess)
        return bail(cuda_fail(h, ce, "init"));
    h->launches += 2;
  } else {
    // f = f^eq(rho0)
    if ((ce = launch_init_eq(scheme, h->prec, arena(h, 0), h->d_runs, h->d_stream_tiles, h->n_stream_tiles, h->d_stage,
                             h->d_rho_off, h->stream)) != cudaSuccess)
      return bail(cuda_fail(h, ce, "init"));
    h->launches += 1;
    if (reservoir) {  // end nodes and ghosts at f^eq(rho_bc)
      for (int b = 0; b < 2; ++b)
        if ((ce = launch_reservoir_step(scheme, h->prec, arena(h, b), arena(h, b), h->d_runs, h->d_plain_tiles,
                                        h->n_plain_tiles, h->plain_tile, 1, h->stream)) != cudaSuccess)
          return bail(cuda_fail(h, ce, "reservoir init"));
      h->launches += 2;
    }
  }
  if ((ce = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(h, ce, "init sync"));
  // rho0's statistics, computed on the device while the host planned
  int bad_run = nruns;
  if ((ce = cudaEventSynchronize(stats.ev)) != cudaSuccess ||
      (ce = cudaMemcpy(&bad_run, h->d_bad_run, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bail(cuda_fail(h, ce, "read rho0 statistics"));
  if (bad_run < nruns) return bail(fail(h, LB_KS_EINVAL, "run " + std::to_string(bad_run) + ": rho0 is not finite"));
  warn_if_linearly_unstable(h, L, dt, tau);
  *out = h;
  return LB_KS_OK;
}

int create(lb_ks_t** out, int scheme, int32_t nruns, const int64_t* N, const double* L, const double* dt,
           const double* tau, const double* rho0, const lb_ks_opts* opts, const double* rho_left = nullptr,
           const double* rho_right = nullptr) {
  lb_ks* h = nullptr;
  try {
    return create_body(h, out, scheme, nruns, N, L, dt, tau, rho0, opts, rho_left, rho_right);
  } catch (...) {
    const int rc = abi_exception(nullptr);
    if (h) lb_ks_free(h);
    if (out) *out = nullptr;
    return rc;
  }
}

}  // namespace

extern "C" {

void lb_ks_default_opts(lb_ks_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = LB_KS_F64;
  o->dm_variant = LB_KS_DM_DERIVED;
  o->recentre_every = 0;
  o->kernel = LB_KS_KERNEL_AUTO;
  o->use_graph = 1;
  o->stream = nullptr;
  o->cluster_size = 0;
}

int lb_ks_init(lb_ks_t** h, int scheme, int64_t N, double L, double dt, double tau, const double* rho0,
               const lb_ks_opts* opts) {
  return create(h, scheme, 1, &N, &L, &dt, &tau, rho0, opts);
}

int lb_ks_batch_init(lb_ks_t** h, int scheme, int32_t nruns, const int64_t* N, const double* L, const double* dt,
                     const double* tau, const double* rho0, const lb_ks_opts* opts) {
  return create(h, scheme, nruns, N, L, dt, tau, rho0, opts);
}

int lb_ks_batch_init_reservoir(lb_ks_t** h, int scheme, int32_t nruns, const int64_t* N, const double* L,
                               const double* dt, const double* tau, const double* rho0, const double* rho_left,
                               const double* rho_right, const lb_ks_opts* opts) try {
  if (!rho_left || !rho_right) {
    if (h) *h = nullptr;
    return fail(nullptr, LB_KS_EINVAL, "rho_left and rho_right must not be NULL");
  }
  return create(h, scheme, nruns, N, L, dt, tau, rho0, opts, rho_left, rho_right);
} catch (...) {
  if (h) *h = nullptr;
  return abi_exception(nullptr);
}

int lb_ks_step(lb_ks_t* h, int64_t n) try {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  if (h->sticky) return h->sticky;
  if (n < 0) return fail(h, LB_KS_EINVAL, "n must be >= 0");
  const int64_t R = h->opts.recentre_every;
  const int64_t chunk_max = (h->kernel == LB_KS_KERNEL_RESIDENT || h->collapse_resident) ? 64LL * h->kmax : 512;
  while (n > 0) {
    int64_t c = std::min(n, chunk_max);
    if (R > 0) c = std::min<int64_t>(c, R - h->phase);
    int rc;
    if (h->opts.use_graph) {
      rc = run_chunk_graph(h, c);
    } else {
      int64_t nk = 0;
      rc = issue_steps(h, c, h->stream, &nk);
      h->launches += nk;
    }
    if (rc) return rc;
    n -= c;
  }
  return LB_KS_OK;
} catch (...) {
  // the host's step counters may be ahead of what was issued: the handle is unusable
  const int rc = abi_exception(h);
  if (h) {
    h->sticky = rc;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (h->cap_stream && cudaStreamIsCapturing(h->cap_stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(h->cap_stream, &g);
      if (g) cudaGraphDestroy(g);
    }
    cudaGetLastError();
  }
  return rc;
}

int lb_ks_rho(lb_ks_t* h, double* out) try {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  if (h->sticky) return h->sticky;
  if (!out) return fail(h, LB_KS_EINVAL, "out must not be NULL");
  // The gather writes straight into out when it is memory of this device.  Pinned host
  // memory gets the gather in chunks into the staging buffer, each chunk copied out by
  // the copy engine (on the capture stream, idle outside lb_ks_step) while the next one is
  // gathered: the copy engine moves more over the host link than the gather's own stores
  // to mapped host memory.  Other host memory gets one staged copy.
  double* dst = h->d_stage;
  bool pinned = false;
  {
    int dev = 0;
    cudaPointerAttributes pa{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaPointerGetAttributes(&pa, out) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeDevice && pa.device == dev) dst = static_cast<double*>(pa.devicePointer);
      else if (pa.type == cudaMemoryTypeHost) pinned = true;
    } else {
      cudaGetLastError();
    }
  }
  if (pinned && h->rho_chunks.size() > 1) {
    if (!h->ev_rho) LBKS_CUDA(h, cudaEventCreateWithFlags(&h->ev_rho, cudaEventDisableTiming), "create event");
    for (size_t c = 0; c + 1 < h->rho_chunks.size(); ++c) {
      const int t0 = h->rho_chunks[c].first, t1 = h->rho_chunks[c + 1].first;
      const int64_t o0 = h->rho_chunks[c].second, o1 = h->rho_chunks[c + 1].second;
      LBKS_CUDA(h, launch_gather_rho(h->nplanes, h->prec, arena(h, h->cur), h->d_runs, h->d_stream_tiles + t0, t1 - t0,
                                     h->d_stage, h->d_rho_off, h->stream), "gather rho");
      h->launches += 1;
      LBKS_CUDA(h, cudaEventRecord(h->ev_rho, h->stream), "record");
      LBKS_CUDA(h, cudaStreamWaitEvent(h->cap_stream, h->ev_rho, 0), "wait");
      LBKS_CUDA(h, cudaMemcpyAsync(out + o0, h->d_stage + o0, sizeof(double) * (size_t)(o1 - o0),
                                   cudaMemcpyDeviceToHost, h->cap_stream), "copy rho");
    }
    LBKS_CUDA(h, cudaStreamSynchronize(h->cap_stream), "sync");
    LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
    return check_flags(h);
  }
  LBKS_CUDA(h, launch_gather_rho(h->nplanes, h->prec, arena(h, h->cur), h->d_runs, h->d_stream_tiles, h->n_stream_tiles,
                                 dst, h->d_rho_off, h->stream), "gather rho");
  h->launches += 1;
  if (dst == h->d_stage)
    LBKS_CUDA(h, cudaMemcpyAsync(out, h->d_stage, sizeof(double) * (size_t)h->total_sites, cudaMemcpyDefault, h->stream),
              "copy rho");
  LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  return check_flags(h);
} catch (...) {
  return abi_exception(h);
}

int lb_ks_mass_energy(lb_ks_t* h, double* mass, double* energy) try {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  if (h->sticky) return h->sticky;
  int64_t nk = 0;
  int rc = issue_guard(h, h->stream, false, &nk);
  if (rc) return rc;
  h->launches += nk;
  std::vector<double> m(h->nruns), e(h->nruns);
  LBKS_CUDA(h, cudaMemcpyAsync(m.data(), h->d_mass, sizeof(double) * h->nruns, cudaMemcpyDeviceToHost, h->stream), "copy mass");
  LBKS_CUDA(h, cudaMemcpyAsync(e.data(), h->d_energy, sizeof(double) * h->nruns, cudaMemcpyDeviceToHost, h->stream), "copy energy");
  LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  if (mass) std::memcpy(mass, m.data(), sizeof(double) * h->nruns);
  if (energy) std::memcpy(energy, e.data(), sizeof(double) * h->nruns);
  return check_flags(h);
} catch (...) {
  return abi_exception(h);
}

int lb_ks_state_bytes(const lb_ks_t* h, size_t* bytes) {
  if (!h || !bytes) return LB_KS_EINVAL;
  *bytes = 64 + sizeof(int64_t) * h->nruns + sizeof(RunDesc) * h->nruns + sizeof(double) * h->nruns +
           storage_bytes(h->prec) * (size_t)h->nplanes * (size_t)h->plane;
  return LB_KS_OK;
}

int lb_ks_save(lb_ks_t* h, void* buf, size_t bytes) try {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  if (h->sticky) return h->sticky;
  size_t need = 0;
  lb_ks_state_bytes(h, &need);
  if (!buf || bytes < need) return fail(h, LB_KS_EINVAL, "buffer too small for the checkpoint");
  unsigned char* p = static_cast<unsigned char*>(buf);
  std::memset(p, 0, 64);
  uint32_t hdr[6] = {kMagic, kVersion, (uint32_t)h->Q, (uint32_t)h->prec, (uint32_t)h->nruns,
                     h->nplanes == 1 ? 1u : 0u};
  std::memcpy(p, hdr, sizeof(hdr));
  int64_t hdr2[3] = {h->plane, h->steps_done, h->phase};
  std::memcpy(p + 24, hdr2, sizeof(hdr2));
  p += 64;
  std::memcpy(p, h->N.data(), sizeof(int64_t) * h->nruns);
  p += sizeof(int64_t) * h->nruns;
  if (!h->tables_on_host) {  // the run constants and initial masses rho0's statistics set
    LBKS_CUDA(h, cudaMemcpyAsync(h->runs_h.data(), h->d_runs, sizeof(RunDesc) * h->nruns, cudaMemcpyDeviceToHost,
                                 h->stream), "read run table");
    LBKS_CUDA(h, cudaMemcpyAsync(h->mass0_h.data(), h->d_mass0, sizeof(double) * h->nruns, cudaMemcpyDeviceToHost,
                                 h->stream), "read initial masses");
    LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
    h->tables_on_host = true;
  }
  std::memcpy(p, h->runs_h.data(), sizeof(RunDesc) * h->nruns);
  p += sizeof(RunDesc) * h->nruns;
  std::memcpy(p, h->mass0_h.data(), sizeof(double) * h->nruns);
  p += sizeof(double) * h->nruns;
  LBKS_CUDA(h, cudaMemcpyAsync(p, h->fbuf[h->cur], storage_bytes(h->prec) * (size_t)h->nplanes * (size_t)h->plane,
                               cudaMemcpyDeviceToHost, h->stream), "save");
  LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  return check_flags(h);
} catch (...) {
  return abi_exception(h);
}

int lb_ks_load(lb_ks_t* h, const void* buf, size_t bytes) try {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  size_t need = 0;
  lb_ks_state_bytes(h, &need);
  if (!buf || bytes < need) return fail(h, LB_KS_EINVAL, "checkpoint buffer too small");
  const unsigned char* p = static_cast<const unsigned char*>(buf);
  uint32_t hdr[6];
  int64_t hdr2[3];
  std::memcpy(hdr, p, sizeof(hdr));
  std::memcpy(hdr2, p + 24, sizeof(hdr2));
  if (hdr[0] != kMagic || hdr[1] != kVersion || hdr[2] != (uint32_t)h->Q || hdr[3] != (uint32_t)h->prec ||
      hdr[4] != (uint32_t)h->nruns || hdr[5] != (h->nplanes == 1 ? 1u : 0u) || hdr2[0] != h->plane)
    return fail(h, LB_KS_EINVAL, "checkpoint does not match this handle (scheme, precision or runs)");
  p += 64;
  if (std::memcmp(p, h->N.data(), sizeof(int64_t) * h->nruns) != 0)
    return fail(h, LB_KS_EINVAL, "checkpoint lattice sizes differ from this handle's");
  p += sizeof(int64_t) * h->nruns;
  if (hdr2[1] < 0 || hdr2[2] < 0) return fail(h, LB_KS_EINVAL, "checkpoint step counters are negative");
  std::vector<RunDesc> runs(h->nruns);
  std::memcpy(runs.data(), p, sizeof(RunDesc) * h->nruns);
  p += sizeof(RunDesc) * h->nruns;
  // the constants (coefficients, rhobar, storage scale) come from the checkpoint; where
  // each run lies in the arenas, and its ends, must be this handle's (the kernels index by them)
  for (int32_t r = 0; r < h->nruns; ++r) {
    const RunDesc &c = runs[r], &own = h->runs_h[r];
    if (c.off != own.off || c.N != own.N || c.reservoir != own.reservoir)
      return fail(h, LB_KS_EINVAL, "checkpoint run " + std::to_string(r) + ": layout differs from this handle's");
    bool finite = std::isfinite(c.r) && std::isfinite(c.rhobar) && std::isfinite(c.scale) && c.scale > 0.0;
    for (int i = 0; i < h->Q; ++i) finite = finite && std::isfinite(c.a[i]) && std::isfinite(c.b[i]);
    if (!finite) return fail(h, LB_KS_EINVAL, "checkpoint run " + std::to_string(r) + ": constants are not finite");
  }
  std::vector<double> m0(h->nruns);
  std::memcpy(m0.data(), p, sizeof(double) * h->nruns);
  p += sizeof(double) * h->nruns;
  LBKS_CUDA(h, cudaStreamSynchronize(h->stream), "sync");
  h->runs_h.assign(runs.begin(), runs.end());
  h->mass0_h = m0;
  h->tables_on_host = true;
  LBKS_CUDA(h, cudaMemcpy(h->d_runs, runs.data(), sizeof(RunDesc) * h->nruns, cudaMemcpyHostToDevice), "load runs");
  LBKS_CUDA(h, cudaMemcpy(h->d_mass0, m0.data(), sizeof(double) * h->nruns, cudaMemcpyHostToDevice), "load mass0");
  LBKS_CUDA(h, cudaMemcpy(h->fbuf[h->cur], p, storage_bytes(h->prec) * (size_t)h->nplanes * (size_t)h->plane,
                          cudaMemcpyHostToDevice), "load populations");
  h->steps_done = hdr2[1];
  // steps since the last guard, on this handle's guard interval (which may differ from
  // the saving handle's): a phase at or past it would never meet it again
  const int64_t R = h->opts.recentre_every;
  h->phase = R > 0 ? hdr2[2] % R : 0;
  h->sticky = LB_KS_OK;
  LBKS_CUDA(h, cudaMemset(h->d_flags, 0, sizeof(int)), "clear flags");
  return LB_KS_OK;
} catch (...) {
  return abi_exception(h);
}

int64_t lb_ks_steps_done(const lb_ks_t* h) { return h ? h->steps_done : -1; }

int lb_ks_set_link_test(lb_ks_t* h, int32_t withhold_step, uint32_t wait_rounds) {
  if (!h) return fail(nullptr, LB_KS_EINVAL, "NULL handle");
  if (withhold_step < -1) return fail(h, LB_KS_EINVAL, "withhold_step must be >= -1");
  if (h->steps_done != 0 || !h->graphs.empty())
    return fail(h, LB_KS_EINVAL, "lb_ks_set_link_test must be called before the first lb_ks_step");
  h->link_withhold_step = withhold_step;
  h->link_wait_limit = wait_rounds ? wait_rounds : (1u << 22);
  return LB_KS_OK;
}

int lb_ks_describe(const lb_ks_t* h, int* kernel, int* spt, int* tpb, int* spl, int* cl, int32_t* nruns,
                   int64_t* total) {
  if (!h) return LB_KS_EINVAL;
  const bool res = h->kernel == LB_KS_KERNEL_RESIDENT || h->collapse_resident;
  if (kernel) *kernel = h->kernel;
  if (spt) *spt = res ? h->S : 0;
  if (tpb) *tpb = res ? h->NT : 0;
  if (spl) *spl = res ? h->kmax : 0;
  if (cl) {
    *cl = res ? 1 : 0;
    for (int l = 0; res && l < h->nlanes; ++l) *cl = std::max(*cl, h->lanes[l].cl);
  }
  if (nruns) *nruns = h->nruns;
  if (total) *total = h->total_sites;
  return LB_KS_OK;
}

int lb_ks_describe_lanes(const lb_ks_t* h, int32_t* lanes, int max_lanes) {
  if (!h || max_lanes < 0 || (max_lanes > 0 && !lanes)) return LB_KS_EINVAL;
  if (!(h->kernel == LB_KS_KERNEL_RESIDENT || h->collapse_resident)) return 0;
  for (int l = 0; l < h->nlanes && l < max_lanes; ++l) {
    const Lane& L = h->lanes[l];
    int32_t* r = lanes + LB_KS_LANE_FIELDS * l;
    r[0] = L.cl;
    r[1] = L.grid;
    r[2] = L.nbundles;
    r[3] = L.segmented ? L.k : h->kmax;
    r[4] = L.segmented ? 1 : 0;
    r[5] = L.kx;
    r[6] = L.merged ? 1 : 0;
    r[7] = L.halves;
  }
  return h->nlanes;
}

int64_t lb_ks_launches(const lb_ks_t* h) { return h ? h->launches : -1; }

void lb_ks_free(lb_ks_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  for (cudaStream_t ss : h->side_stream)
    if (ss) cudaStreamSynchronize(ss);
  if (h->cap_stream) cudaStreamSynchronize(h->cap_stream);  // init work, when create() bails out
  for (void* p : h->allocations) cudaFreeAsync(p, h->stream);  // back to the pool, in stream order
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int l = 0; l < 2; ++l) {
    if (h->side_stream[l]) cudaStreamDestroy(h->side_stream[l]);
    if (h->ev_join[l]) cudaEventDestroy(h->ev_join[l]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_rho) cudaEventDestroy(h->ev_rho);
  cudaGetLastError();
  delete h;
}

const char* lb_ks_last_error(const lb_ks_t* h) { return h ? h->err.c_str() : g_ctor_error.c_str(); }

int lb_ks_fma_peak(int fp64, double* flops_per_s) try {
  if (!flops_per_s) return LB_KS_EINVAL;
  cudaError_t e = fma_peak(fp64, flops_per_s, nullptr);
  if (e != cudaSuccess) {
    g_ctor_error = std::string("fma peak: ") + cudaGetErrorString(e);
    return LB_KS_ECUDA;
  }
  return LB_KS_OK;
} catch (...) {
  return abi_exception(nullptr);
}

}  // extern "C"
