// Internal declarations shared by the host API and the kernel translation units.
// Not part of the public ABI (that is include/lb_ks.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbks {

constexpr int kMaxQ = 7;

// Storage precisions (same values as LB_KS_F64 / LB_KS_F32 / LB_KS_F16S).
enum Storage : int { kF64 = 0, kF32 = 1, kF16S = 2 };

// Per-run constants, computed in FP64 on the host (lbks_params.cpp) and uploaded
// once; rhobar and the FP16 scale, which depend on rho0, are filled in on the device
// (launch_init_stats).  The step of Eq. LB_equation_ordinary is evaluated as
//     rho  = rhobar + sum_i g_i                 (g_i = f_i - w0_i rhobar, the stored deviation)
//     g*_i = r g_i + rho a_i + rho^2 b_i        (i >= 1)
//     g*_0 = sum_i g_i - sum_{i>=1} g*_i        (mass conservation of the collision)
// with r = 1 - 1/tau, a_i = A_i / tau, b_i = B_i / tau, where f^eq_i = A_i rho + B_i rho^2.
// For rhobar = 0 this is f*_i = f_i - (f_i - f^eq_i)/tau.
struct RunDesc {
  int64_t off;  // arena offset (elements) of site 0 of this run in every plane
  int64_t N;    // sites
  double a[8], b[8];  // A_i / tau, B_i / tau
  double A[8], B[8];  // equilibrium coefficients
  double r, rhobar, scale, inv_scale;  // scale: F16S stored value = g / scale
  float af[8], bf[8];
  float rf, rhobarf, scalef, inv_scalef;
  // Fixed-value ends (front test of Table 5): nodes j <= 0 and j >= N-1, and c_max ghost
  // nodes beyond each end (stored at j = -c_max..-1 and N..N-1+c_max), are reservoirs
  // held at f^eq(rho_left) / f^eq(rho_right).  reservoir = 0: periodic lattice.
  int32_t reservoir, pad_;
  double rho_left, rho_right;
};

// One unit of work of the resident kernel: a lattice (ring) or a stretch of
// one (segment) held by a range of threads of one thread block.
struct Piece {
  int32_t run;
  int32_t t0;     // first thread of the block
  int32_t nthr;   // threads V; thread j holds S or S-1 consecutive sites
  int32_t n;      // sites loaded (ring: N)
  int64_t x0;     // run-local site of loaded index 0, in [0, N)
  int32_t st_lo;  // loaded indices [st_lo, st_hi) are written back
  int32_t st_hi;
  // > 0: one half of a lattice held by a cluster pair (the other half in the other
  // block), with halo = c_max * kx sites on each side of its own sites [st_lo, st_hi)
  // (st_lo = halo), refreshed from the other block every kx steps
  int32_t halo;
  int32_t pad_;
};

// Steps between the halo exchanges of a lattice held as two halves by a cluster pair
// (the exchange area is sized for at most kPairStepsMax).
constexpr int kPairStepsMax = 32;

// Tile of the one-thread-per-site and streaming kernels: sites [x0, x0 + len) of one run.
struct Tile {
  int32_t run;
  int32_t x0;
  int32_t len;
  int32_t pad;
};

struct Arena {
  void* f;        // plane i of run r at element i * plane + runs[r].off
  int64_t plane;  // plane stride (elements)
};

// ---- launchers (each returns the CUDA error of the launch) ----
cudaError_t launch_init_eq(int Q, int storage, Arena dst, const RunDesc* runs, const Tile* tiles,
                           int ntiles, const double* rho0, const int64_t* rho_off, cudaStream_t s);
cudaError_t launch_gather_rho(int Q, int storage, Arena src, const RunDesc* runs, const Tile* tiles,
                              int ntiles, double* out, const int64_t* out_off, cudaStream_t s);
// threads: the block size, 32..256 (a multiple of 32), at least every tile's length.
cudaError_t launch_plain_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs,
                              const Tile* tiles, int ntiles, int threads, cudaStream_t s);
cudaError_t launch_stream_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs,
                               const Tile* tiles, int ntiles, cudaStream_t s);
// Lattices with reservoir ends: tiles cover nodes -c_max .. N-1+c_max.  reset_only = 1
// writes f^eq(rho_bc) into the reservoir nodes of dst and nothing else (initial state).
// threads: as for launch_plain_step.
cudaError_t launch_reservoir_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs,
                                  const Tile* tiles, int ntiles, int threads, int reset_only, cudaStream_t s);
// Initial statistics of rho0 (FP64, staged on the device; tiles cover [0, N) of each run):
// mass0 per run, rhobar (and for F16S the storage scale) written into runs, and the first
// run holding a non-finite value atomically min-ed into bad_run (scratch: 2 doubles per tile).
cudaError_t launch_init_stats(int Q, int storage, int nruns, const double* rho0, const int64_t* rho_off,
                              RunDesc* runs, const Tile* tiles, int ntiles, const int32_t* tile_begin,
                              double* partials, double* mass0, int* bad_run, cudaStream_t s);
// Guard: per-tile FP64 partial sums of rho and rho^2 (scratch: 2 doubles per tile),
// then per-run totals, non-finite flag, and (if recentre) g_0 += (M0 - M)/N.
cudaError_t launch_mass_partials(int Q, int storage, Arena src, const RunDesc* runs, const Tile* tiles,
                                 int ntiles, double* partials, cudaStream_t s);
cudaError_t launch_mass_finalize(int nruns, const int32_t* tile_begin, const double* partials,
                                 const RunDesc* runs, const double* mass0, double* mass, double* energy,
                                 double* delta, int* flags, cudaStream_t s);
cudaError_t launch_recentre(int storage, Arena f, const RunDesc* runs, const Tile* tiles, int ntiles,
                            const double* delta, cudaStream_t s);

struct ResidentLaunch {
  int Q, storage, S, NT;
  Arena src, dst;
  const RunDesc* runs;
  const Piece* pieces;
  const int2* bundles;  // (first piece, piece count) per bundle
  int nbundles;
  int* queue;           // work counter, zeroed before each launch
  int ksteps;
  int grid;    // work groups (blocks, or clusters of cl blocks)
  int cl = 1;  // blocks per work group: 1, or 2 (a thread block cluster)
  int* flags = nullptr;  // error flags (bit 2: a bounded wait between the blocks of a cluster ran out)
  bool collapse = false;  // the tau = 1 collapse (one stored plane) instead of the LB populations
  int kx = 0;             // cl = 2: steps between the halo exchanges of lattice halves (Piece::halo)
  uint32_t wait_limit = 1u << 22;  // cl = 2: try_wait rounds before a wait on the other block gives up
  int withhold_step = -1;          // cl = 2, testing aid: block 1 sends nothing across the edge at this step
};
bool resident_supported(int Q, int storage, int S, int NT);
cudaError_t resident_prepare(int Q, int storage, int S, int NT, int* blocks_per_sm);
// The tau = 1 collapse (one stored plane).
int collapse_tile_sites();
cudaError_t launch_collapse_init(int storage, Arena dst, const RunDesc* runs, const Tile* tiles, int ntiles,
                                 const double* rho0, const int64_t* rho_off, cudaStream_t s);
cudaError_t launch_collapse_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs, const Tile* tiles,
                                 int ntiles, cudaStream_t s);
bool collapse_resident_supported(int Q, int storage, int S, int NT);
cudaError_t collapse_resident_prepare(int Q, int storage, int S, int NT, int* blocks_per_sm);
cudaError_t launch_collapse_resident(const ResidentLaunch& L, cudaStream_t s);

// Clusters of two blocks: the largest number of clusters resident at once.
cudaError_t resident_cluster_prepare(int Q, int storage, int S, int NT, int* max_clusters);
cudaError_t launch_resident_cluster(const ResidentLaunch& L, cudaStream_t s);
cudaError_t launch_resident(const ResidentLaunch& L, cudaStream_t s);

// Diagnostic micro-benchmark of the FMA pipes (flop/s), used by the benchmark
// to state measured ALU peaks beside the derived ones.
cudaError_t fma_peak(int fp64, double* flops_per_s, cudaStream_t s);

}  // namespace lbks
