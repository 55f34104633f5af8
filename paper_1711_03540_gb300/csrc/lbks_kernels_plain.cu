// One-thread-per-site kernels: initialisation at equilibrium, the plain
// fused step (the FP64 baseline), the rho gather and the FP64 mass guard.
#include "lbks_device.cuh"

namespace lbks {

namespace {

constexpr int kPlainThreads = 256;

// Error-free sum: s + e == a + b exactly (Knuth's TwoSum, six rounded operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// An unevaluated sum h + l of two floats (|l| <= ulp(h) / 2 after renormalisation):
// ~48 bits carried on GB300's wide FP32 pipe instead of its narrow FP64 pipe.
struct F2 {
  float h, l;
};

// (a.h + a.l) + (b.h + b.l): the high parts added error-free, the error and the low
// parts added to it, the result renormalised (both steps TwoSum).
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  F2 r;
  two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ F2 f2_shfl_xor(F2 a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

// x as a pair: its float rounding and the float rounding of the rest (exact to ~48 bits).
__device__ __forceinline__ F2 f2_of(double x) {
  const float h = (float)x;
  return {h, (float)__dsub_rn(x, (double)h)};
}

// a b as a pair: the high product's rounding error exact by FMA, the cross terms
// added to it, then renormalised (|error| << |product|, so Fast2Sum suffices).
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}


// f_i = f^eq_i(rho0) = A_i rho0 + B_i rho0^2 (Sec. 2, Eq. feq and its D1Q7 form),
// stored as the deviation g_i = f_i - w0_i rhobar.  FP64 storage: evaluated in FP64.
// FP32/FP16 storage: evaluated in float pairs (f2_mul, f2_add: ~48 bits, more than
// the stored float keeps) and rounded once to the compute float; the coefficients'
// pairs are formed once per tile.  GB300's FP64 pipe would otherwise bound the pass
// (about 20 FP64 operations per site).
template <int Q, int ST>
__global__ void __launch_bounds__(kPlainThreads) init_eq_kernel(Arena dst, const RunDesc* __restrict__ runs,
                                                                const Tile* __restrict__ tiles,
                                                                const double* __restrict__ rho0,
                                                                const int64_t* __restrict__ rho_off) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  if constexpr (ST == kF64) {
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
      const int64_t x = tl.x0 + k;
      const double rho = rho0[rho_off[tl.run] + x];
      T* f = static_cast<T*>(dst.f) + d.off + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        double v = __fma_rn(d.B[i], __dmul_rn(rho, rho), __dmul_rn(d.A[i], rho));
        if (i == 0) v = __dsub_rn(v, d.rhobar);
        from_compute(static_cast<CT>(v), static_cast<CT>(d.inv_scale), f + (int64_t)i * dst.plane);
      }
    }
  } else {
    __shared__ F2 s_c[2 * Q + 1];  // A_i, B_i, -rhobar
    if ((int)threadIdx.x < 2 * Q + 1) {
      const int c = threadIdx.x;
      s_c[c] = f2_of(c < Q ? d.A[c] : (c < 2 * Q ? d.B[c - Q] : -d.rhobar));
    }
    __syncthreads();
    const float inv = d.inv_scalef;
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
      const int64_t x = tl.x0 + k;
      const F2 r = f2_of(rho0[rho_off[tl.run] + x]);
      const F2 r2 = f2_mul(r, r);
      T* f = static_cast<T*>(dst.f) + d.off + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        F2 v = f2_add(f2_mul(s_c[Q + i], r2), f2_mul(s_c[i], r));
        if (i == 0) v = f2_add(v, s_c[2 * Q]);
        from_compute(__fadd_rn(v.h, v.l), inv, f + (int64_t)i * dst.plane);
      }
    }
  }
}

// rho = rhobar + sum_i g_i.  FP64 storage: accumulated in FP64.  FP32/FP16 storage: as
// a float pair (TwoSum per plane), converted to FP64 exactly once per site.
template <int Q, int ST>
__global__ void __launch_bounds__(kPlainThreads) gather_rho_kernel(Arena src, const RunDesc* __restrict__ runs,
                                                                   const Tile* __restrict__ tiles,
                                                                   double* __restrict__ out,
                                                                   const int64_t* __restrict__ out_off) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  if constexpr (ST == kF64) {
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
      const int64_t x = tl.x0 + k;
      const T* f = static_cast<const T*>(src.f) + d.off + x;
      double rho = d.rhobar;
#pragma unroll
      for (int i = 0; i < Q; ++i) rho += static_cast<double>(to_compute(f[(int64_t)i * src.plane], static_cast<CT>(d.scale)));
      out[out_off[tl.run] + x] = rho;
    }
  } else {
    __shared__ F2 s_rb;
    if (threadIdx.x == 0) s_rb = f2_of(d.rhobar);
    __syncthreads();
    const F2 rb = s_rb;
    const float scale = d.scalef;
    for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
      const int64_t x = tl.x0 + k;
      const T* f = static_cast<const T*>(src.f) + d.off + x;
      float hi = rb.h, lo = rb.l, t, te;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        two_sum(hi, to_compute(f[(int64_t)i * src.plane], scale), t, te);
        hi = t;
        lo = __fadd_rn(lo, te);
      }
      out[out_off[tl.run] + x] = (double)hi + (double)lo;
    }
  }
}

// The plain fused step: one thread per site reads its Q populations, collides
// (Eq. LB_equation_ordinary) and pushes f*_i to site x + c_i (mod N).
template <int Q, int ST>
__global__ void __launch_bounds__(kPlainThreads) plain_step_kernel(Arena src, Arena dst,
                                                                   const RunDesc* __restrict__ runs,
                                                                   const Tile* __restrict__ tiles) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  wait_prior_grid();
  const Tile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.len) return;
  const RunDesc& d = runs[tl.run];
  const Coef<CT, Q> k = load_coef<CT, Q>(d);
  const int64_t x = tl.x0 + threadIdx.x;
  const T* fs = static_cast<const T*>(src.f) + d.off;
  T* fd = static_cast<T*>(dst.f) + d.off;
  CT g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) g[i] = to_compute(fs[(int64_t)i * src.plane + x], k.scale);
  collide<Q, CT>(g, k);
#pragma unroll
  for (int i = 0; i < Q; ++i)
    from_compute(g[i], k.inv_scale, fd + (int64_t)i * dst.plane + wrap_site(x + speed(i), d.N));
}

// Lattices with reservoir ends (the fixed end values of the front test, Table 5).
// One thread per node j in [-c_max, N + c_max).  Reservoir nodes (j <= 0, j >= N-1,
// ghosts included) rewrite their own populations as f^eq(rho_bc) in the
// destination; every node collides its source populations once (a reservoir node
// the f^eq(rho_bc) it holds) with the same collide() as every other kernel and
// pushes plane i to j + c_i when that node is interior (pushes into reservoir
// nodes are dropped), so each interior node receives exactly one value per plane.
template <int Q, int ST>
__global__ void __launch_bounds__(kPlainThreads) reservoir_step_kernel(Arena src, Arena dst,
                                                                       const RunDesc* __restrict__ runs,
                                                                       const Tile* __restrict__ tiles, int reset_only) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  wait_prior_grid();
  const Tile tl = tiles[blockIdx.x];
  if ((int)threadIdx.x >= tl.len) return;
  const RunDesc& d = runs[tl.run];
  const int64_t j = (int64_t)tl.x0 + threadIdx.x;
  T* fd = static_cast<T*>(dst.f) + d.off;
  if (j <= 0 || j >= d.N - 1) {
    const double rb = j <= 0 ? d.rho_left : d.rho_right;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double v = __fma_rn(d.B[i], __dmul_rn(rb, rb), __dmul_rn(d.A[i], rb));
      if (i == 0) v = __dsub_rn(v, d.rhobar);
      from_compute(static_cast<CT>(v), static_cast<CT>(d.inv_scale), fd + (int64_t)i * dst.plane + j);
    }
  }
  if (reset_only) return;
  const T* fs = static_cast<const T*>(src.f) + d.off;
  const Coef<CT, Q> k = load_coef<CT, Q>(d);
  CT g[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) g[q] = to_compute(fs[(int64_t)q * src.plane + j], k.scale);
  collide<Q, CT>(g, k);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int64_t y = j + speed(i);
    if (y > 0 && y < d.N - 1) from_compute(g[i], k.inv_scale, fd + (int64_t)i * dst.plane + y);
  }
}

// One site of FP32/FP16 storage into the thread's sums: rho = rhobar + sum_i g_i as a
// pair (TwoSum per plane, then renormalised), then m += rho and e += rho^2 (the low part
// of hi^2 exact by FMA, 2 hi lo added to it).
template <int Q>
__device__ __forceinline__ void site_pair(const float (&g)[Q], const F2 rb, F2& m, F2& e) {
  float hi = rb.h, lo = rb.l, t, te;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    two_sum(hi, g[i], t, te);
    hi = t;
    lo = __fadd_rn(lo, te);
  }
  two_sum(hi, lo, hi, lo);  // renormalise
  two_sum(m.h, hi, t, te);
  m.h = t;
  m.l = __fadd_rn(m.l, __fadd_rn(te, lo));
  const float p = __fmul_rn(hi, hi);
  const float pe = __fmaf_rn(hi, hi, -p);  // exact low part of hi^2
  two_sum(e.h, p, t, te);
  e.h = t;
  e.l = __fadd_rn(e.l, __fadd_rn(te, __fmaf_rn(2.f * hi, lo, pe)));
}

// FP64 storage: FP64 rho and rho^2 sums of the sites k0, k0 + stride, ... < len of one tile.
template <int Q>
__device__ __forceinline__ void site_sums_f64(const double* f, int64_t plane, const RunDesc& d, int k0, int len,
                                              int stride, double& m, double& e) {
  m = 0.0;
  e = 0.0;
  for (int k = k0; k < len; k += stride) {
    double rho = d.rhobar;
#pragma unroll
    for (int i = 0; i < Q; ++i) rho += f[(int64_t)i * plane + k];
    m += rho;
    e = __fma_rn(rho, rho, e);
  }
}

// FP32/FP16 storage: the same sums as pairs (site_pair), sites k0, k0 + stride, ...
template <int Q, int ST>
__device__ __forceinline__ void site_sums_pair(const typename StorageType<ST>::type* f, int64_t plane,
                                               const RunDesc& d, const F2 rb, int k0, int len, int stride, F2& m,
                                               F2& e) {
  m = {0.f, 0.f};
  e = {0.f, 0.f};
  for (int k = k0; k < len; k += stride) {
    float g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = to_compute(f[(int64_t)i * plane + k], d.scalef);
    site_pair<Q>(g, rb, m, e);
  }
}

// FP32 storage, tile start 16-byte aligned: thread k sums sites 4k .. 4k+3 of the tile,
// one 16-byte load per plane (site_pair per site, sites in order).
template <int Q>
__device__ __forceinline__ void site_sums_vec4(const float* f, int64_t plane, const F2 rb, int k, int len, F2& m,
                                               F2& e) {
  m = {0.f, 0.f};
  e = {0.f, 0.f};
  const int x = 4 * k;
  if (x >= len) return;
  float v[4][Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float* p = f + (int64_t)i * plane + x;
    if (x + 4 <= len) {
      const float4 q = *reinterpret_cast<const float4*>(p);
      v[0][i] = q.x; v[1][i] = q.y; v[2][i] = q.z; v[3][i] = q.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u][i] = x + u < len ? p[u] : 0.f;
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (x + u >= len) break;
    site_pair<Q>(v[u], rb, m, e);
  }
}

// Guard, pass 1: sums of rho and rho^2 over one tile (fixed-order tree), stored as FP64.
// FP64 storage sums in FP64.  FP32/FP16 storage keeps the sums as float pairs through
// the warp tree and the warps' sum (thread 0), converted to FP64 once per tile: the
// narrow FP64 pipe (about 1/40 of the FP32 rate on this part) would otherwise
// take most of the pass.
template <int Q, int ST>
__global__ void __launch_bounds__(kPlainThreads) mass_partials_kernel(Arena src, const RunDesc* __restrict__ runs,
                                                                      const Tile* __restrict__ tiles,
                                                                      double* __restrict__ partials) {
  using T = typename StorageType<ST>::type;
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  const T* const base = static_cast<const T*>(src.f) + d.off + tl.x0;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if constexpr (ST == kF64) {
    double m, e;
    site_sums_f64<Q>(base, src.plane, d, threadIdx.x, tl.len, blockDim.x, m, e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_xor_sync(0xffffffffu, m, o);
      e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    __shared__ double sm[2][kPlainThreads / 32];
    if (lane == 0) { sm[0][w] = m; sm[1][w] = e; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double mm = 0.0, ee = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { mm += sm[0][i]; ee += sm[1][i]; }
      partials[2 * blockIdx.x] = mm;
      partials[2 * blockIdx.x + 1] = ee;
    }
  } else {
    // rhobar as a float pair, formed once per tile
    __shared__ float s_rb[2];
    if (threadIdx.x == 0) {
      const float hi = (float)d.rhobar;
      s_rb[0] = hi;
      s_rb[1] = (float)(d.rhobar - (double)hi);
    }
    __syncthreads();
    const F2 rb{s_rb[0], s_rb[1]};
    F2 m, e;
    if (ST == kF32 && Q > 1 && ((d.off + tl.x0) & 3) == 0 && (src.plane & 3) == 0 && tl.len <= 4 * (int)blockDim.x)
      site_sums_vec4<Q>(reinterpret_cast<const float*>(base), src.plane, rb, threadIdx.x, tl.len, m, e);
    else
      site_sums_pair<Q, ST>(base, src.plane, d, rb, threadIdx.x, tl.len, blockDim.x, m, e);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = f2_add(m, f2_shfl_xor(m, o));
      e = f2_add(e, f2_shfl_xor(e, o));
    }
    __shared__ F2 sm[2][kPlainThreads / 32];
    if (lane == 0) { sm[0][w] = m; sm[1][w] = e; }
    __syncthreads();
    if (threadIdx.x == 0) {
      F2 mm = sm[0][0], ee = sm[1][0];
      for (int i = 1; i < (int)(blockDim.x >> 5); ++i) { mm = f2_add(mm, sm[0][i]); ee = f2_add(ee, sm[1][i]); }
      partials[2 * blockIdx.x] = (double)mm.h + (double)mm.l;
      partials[2 * blockIdx.x + 1] = (double)ee.h + (double)ee.l;
    }
  }
}

// Guard, pass 2: one warp per run sums that run's tile partials in a fixed
// order, flags a non-finite mass, and computes the re-centring increment
// (M0 - M)/N for g_0 (the mass invariant: sum_i f^eq_i = rho, Eq. cond_weight).
__global__ void mass_finalize_kernel(int nruns, const int32_t* __restrict__ tile_begin,
                                     const double* __restrict__ partials, const RunDesc* __restrict__ runs,
                                     const double* __restrict__ mass0, double* __restrict__ mass,
                                     double* __restrict__ energy, double* __restrict__ delta, int* __restrict__ flags) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nruns) return;
  double m = 0.0, e = 0.0;
  for (int t = tile_begin[warp] + lane; t < tile_begin[warp + 1]; t += 32) {
    m += partials[2 * t];
    e += partials[2 * t + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    e += __shfl_xor_sync(0xffffffffu, e, o);
  }
  if (lane == 0) {
    if (mass) mass[warp] = m;
    if (energy) energy[warp] = e;
    const bool ok = isfinite(m) && isfinite(e);
    if (!ok) atomicOr(flags, 1);
    if (delta) delta[warp] = ok ? (mass0[warp] - m) / static_cast<double>(runs[warp].N) : 0.0;
  }
}

// Guard, pass 3: g_0 += (M0 - M)/N at every site of a tile.  The increment is
// usually far below half an ulp of the stored g_0 (FP32 or FP16), where plain
// rounding would discard it every time.  One warp per tile: each lane walks a
// contiguous chunk and carries the exact rounding residual (TwoSum) to its next
// site; the lanes' leftover residuals are then summed and added to the tile's
// first site, so the tile as a whole receives its share of the correction to
// within half an ulp.  Arithmetic in the compute type (FP32 for FP32/FP16).
constexpr int kRecentreThreads = 32;
template <int ST>
__device__ __forceinline__ typename StorageType<ST>::compute add_carry(typename StorageType<ST>::type* p,
                                                                        typename StorageType<ST>::compute inc,
                                                                        typename StorageType<ST>::compute scale,
                                                                        typename StorageType<ST>::compute inv) {
  using CT = typename StorageType<ST>::compute;
  using T = typename StorageType<ST>::type;
  const CT v = to_compute(*p, scale);
  CT t, te;
  two_sum(v, inc, t, te);  // t + te == v + inc exactly
  T q;
  from_compute(t, inv, &q);
  *p = q;
  return add_rn(add_rn(t, -to_compute(q, scale)), te);  // (v + inc) - stored value
}

template <int ST>
__global__ void __launch_bounds__(kRecentreThreads) recentre_kernel(Arena f, const RunDesc* __restrict__ runs,
                                                                    const Tile* __restrict__ tiles,
                                                                    const double* __restrict__ delta) {
  using T = typename StorageType<ST>::type;
  using CT = typename StorageType<ST>::compute;
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  const CT dl = static_cast<CT>(delta[tl.run]);
  if (dl == CT(0)) return;
  T* base = static_cast<T*>(f.f) + d.off + tl.x0;
  const CT scale = static_cast<CT>(d.scale), inv = static_cast<CT>(d.inv_scale);
  const int chunk = (tl.len + 31) / 32;
  const int k0 = threadIdx.x * chunk, k1 = min(tl.len, k0 + chunk);
  CT carry = CT(0);
  if (chunk <= 32) {
    // the tile through shared memory: coalesced global loads and stores; lane L's chunk
    // at padded rows (stride 33) so that the lanes' walks hit distinct banks
    __shared__ T tile[32 * 33];
    for (int k = threadIdx.x; k < tl.len; k += 32) tile[(k / chunk) * 33 + k % chunk] = base[k];
    __syncwarp();
    for (int k = k0; k < k1; ++k) carry = add_carry<ST>(tile + threadIdx.x * 33 + (k - k0), add_rn(dl, carry), scale, inv);
    __syncwarp();
    for (int k = threadIdx.x; k < tl.len; k += 32) base[k] = tile[(k / chunk) * 33 + k % chunk];
  } else {
    for (int k = k0; k < k1; ++k) carry = add_carry<ST>(base + k, add_rn(dl, carry), scale, inv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) carry = add_rn(carry, __shfl_xor_sync(0xffffffffu, carry, o));
  __syncwarp();
  if (threadIdx.x == 0) add_carry<ST>(base, carry, scale, inv);
}

// Initial statistics of rho0 (staged in FP64 on the device), pass 1: per tile the FP64
// sum of rho0 and the number of non-finite values, in the fixed order of the guard's
// partial sums (thread-strided, warp tree, warps in order).
__global__ void __launch_bounds__(kPlainThreads) init_stats_partials_kernel(const double* __restrict__ rho0,
                                                                           const int64_t* __restrict__ rho_off,
                                                                           const Tile* __restrict__ tiles,
                                                                           double* __restrict__ partials) {
  const Tile tl = tiles[blockIdx.x];
  const double* r = rho0 + rho_off[tl.run] + tl.x0;
  double m = 0.0, bad = 0.0;
  for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
    const double v = r[k];
    if (isfinite(v)) m += v;
    else bad += 1.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  __shared__ double sm[2][kPlainThreads / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sm[0][w] = m; sm[1][w] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0, bb = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { mm += sm[0][i]; bb += sm[1][i]; }
    partials[2 * blockIdx.x] = mm;
    partials[2 * blockIdx.x + 1] = bb;
  }
}

// Pass 2: one warp per run sums its tiles' partials in a fixed order: the initial mass
// M0 (the guard's re-centring target), the mean rhobar = M0 / N that the deviation
// form stores g_0 against (0 for FP64 storage), and the first run with a non-finite
// value (atomicMin into bad_run).
__global__ void init_stats_finalize_kernel(int nruns, int storage, const int32_t* __restrict__ tile_begin,
                                           const double* __restrict__ partials, RunDesc* __restrict__ runs,
                                           double* __restrict__ mass0, int* __restrict__ bad_run) {
  const int run = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (run >= nruns) return;
  double m = 0.0, bad = 0.0;
  for (int t = tile_begin[run] + lane; t < tile_begin[run + 1]; t += 32) {
    m += partials[2 * t];
    bad += partials[2 * t + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m += __shfl_xor_sync(0xffffffffu, m, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) {
    mass0[run] = m;
    if (bad > 0.0) atomicMin(bad_run, run);
    const double rhobar = storage == kF64 ? 0.0 : m / static_cast<double>(runs[run].N);
    runs[run].rhobar = rhobar;
    runs[run].rhobarf = (float)rhobar;
  }
}

// Scaled FP16 storage, pass 3: per tile the largest |g_i| of the initial state,
// g_i = A_i rho + B_i rho^2 (minus rhobar for i = 0), over sites and planes.
template <int Q>
__global__ void __launch_bounds__(kPlainThreads) init_scale_partials_kernel(const double* __restrict__ rho0,
                                                                           const int64_t* __restrict__ rho_off,
                                                                           const RunDesc* __restrict__ runs,
                                                                           const Tile* __restrict__ tiles,
                                                                           double* __restrict__ partials) {
  const Tile tl = tiles[blockIdx.x];
  const RunDesc& d = runs[tl.run];
  const double* r = rho0 + rho_off[tl.run] + tl.x0;
  double g = 0.0;
  for (int k = threadIdx.x; k < tl.len; k += blockDim.x) {
    const double v = r[k], v2 = __dmul_rn(v, v);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      double gi = __fma_rn(d.B[i], v2, __dmul_rn(d.A[i], v));
      if (i == 0) gi = __dsub_rn(gi, d.rhobar);
      g = fmax(g, fabs(gi));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  __shared__ double sm[kPlainThreads / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = g;
  __syncthreads();
  if (threadIdx.x == 0) {
    double gg = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) gg = fmax(gg, sm[i]);
    partials[blockIdx.x] = gg;
  }
}

// Pass 4: per run, the FP16 storage scale (the largest |g_i|, or 1 for a zero state).
__global__ void init_scale_finalize_kernel(int nruns, const int32_t* __restrict__ tile_begin,
                                           const double* __restrict__ partials, RunDesc* __restrict__ runs) {
  const int run = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (run >= nruns) return;
  double g = 0.0;
  for (int t = tile_begin[run] + lane; t < tile_begin[run + 1]; t += 32) g = fmax(g, partials[t]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  if (lane == 0) {
    const double scale = g > 0.0 ? g : 1.0;
    runs[run].scale = scale;
    runs[run].inv_scale = 1.0 / scale;
    runs[run].scalef = (float)scale;
    runs[run].inv_scalef = (float)(1.0 / scale);
  }
}

// FMA-pipe micro-benchmark: independent chains of fused multiply-adds.
template <typename T>
__global__ void fma_peak_kernel(T* out, int iters, T seed) {
  T a0 = seed + threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  const T m = (T)0.999999, c = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      a0 = fma_rn(a0, m, c); a1 = fma_rn(a1, m, c); a2 = fma_rn(a2, m, c); a3 = fma_rn(a3, m, c);
      a4 = fma_rn(a4, m, c); a5 = fma_rn(a5, m, c); a6 = fma_rn(a6, m, c); a7 = fma_rn(a7, m, c);
    }
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == (T)-1.2345) out[threadIdx.x] = s;  // keeps the chains alive
}

}  // namespace

#define LBKS_DISPATCH_Q_ST(Q, ST, CALL)                                     \
  do {                                                                      \
    if ((Q) == 5 && (ST) == kF64) { constexpr int Qc = 5, STc = kF64; CALL; } \
    else if ((Q) == 5 && (ST) == kF32) { constexpr int Qc = 5, STc = kF32; CALL; } \
    else if ((Q) == 5 && (ST) == kF16S) { constexpr int Qc = 5, STc = kF16S; CALL; } \
    else if ((Q) == 7 && (ST) == kF64) { constexpr int Qc = 7, STc = kF64; CALL; } \
    else if ((Q) == 7 && (ST) == kF32) { constexpr int Qc = 7, STc = kF32; CALL; } \
    else if ((Q) == 7 && (ST) == kF16S) { constexpr int Qc = 7, STc = kF16S; CALL; } \
    else return cudaErrorInvalidValue;                                      \
  } while (0)

cudaError_t launch_init_eq(int Q, int storage, Arena dst, const RunDesc* runs, const Tile* tiles, int ntiles,
                           const double* rho0, const int64_t* rho_off, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  LBKS_DISPATCH_Q_ST(Q, storage, (init_eq_kernel<Qc, STc><<<ntiles, kPlainThreads, 0, s>>>(dst, runs, tiles, rho0, rho_off)));
  return cudaGetLastError();
}

// Q = 1: the single stored plane of the tau = 1 collapse (rho = rhobar + delta).
cudaError_t launch_gather_rho(int Q, int storage, Arena src, const RunDesc* runs, const Tile* tiles, int ntiles,
                              double* out, const int64_t* out_off, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (Q == 1) {
    if (storage == kF64) gather_rho_kernel<1, kF64><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, out, out_off);
    else if (storage == kF32) gather_rho_kernel<1, kF32><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, out, out_off);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }
  LBKS_DISPATCH_Q_ST(Q, storage, (gather_rho_kernel<Qc, STc><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, out, out_off)));
  return cudaGetLastError();
}

cudaError_t launch_plain_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs, const Tile* tiles,
                              int ntiles, int threads, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (storage == kF16S || threads < 32 || threads > kPlainThreads || threads % 32) return cudaErrorInvalidValue;
  LBKS_DISPATCH_Q_ST(Q, storage, return launch_early(plain_step_kernel<Qc, STc>, ntiles, threads, 0, s, src, dst, runs, tiles));
}

cudaError_t launch_reservoir_step(int Q, int storage, Arena src, Arena dst, const RunDesc* runs, const Tile* tiles,
                                  int ntiles, int threads, int reset_only, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (threads < 32 || threads > kPlainThreads || threads % 32) return cudaErrorInvalidValue;
  LBKS_DISPATCH_Q_ST(Q, storage, return launch_early(reservoir_step_kernel<Qc, STc>, ntiles, threads, 0, s, src, dst,
                                                     runs, tiles, reset_only));
}

cudaError_t launch_mass_partials(int Q, int storage, Arena src, const RunDesc* runs, const Tile* tiles, int ntiles,
                                 double* partials, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (Q == 1) {
    if (storage == kF64) mass_partials_kernel<1, kF64><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, partials);
    else if (storage == kF32) mass_partials_kernel<1, kF32><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, partials);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }
  LBKS_DISPATCH_Q_ST(Q, storage, (mass_partials_kernel<Qc, STc><<<ntiles, kPlainThreads, 0, s>>>(src, runs, tiles, partials)));
  return cudaGetLastError();
}

cudaError_t launch_init_stats(int Q, int storage, int nruns, const double* rho0, const int64_t* rho_off,
                              RunDesc* runs, const Tile* tiles, int ntiles, const int32_t* tile_begin,
                              double* partials, double* mass0, int* bad_run, cudaStream_t s) {
  if (ntiles == 0 || nruns == 0) return cudaSuccess;
  const int fin_blocks = (nruns * 32 + 127) / 128;
  init_stats_partials_kernel<<<ntiles, kPlainThreads, 0, s>>>(rho0, rho_off, tiles, partials);
  init_stats_finalize_kernel<<<fin_blocks, 128, 0, s>>>(nruns, storage, tile_begin, partials, runs, mass0, bad_run);
  if (storage == kF16S) {
    if (Q == 5) init_scale_partials_kernel<5><<<ntiles, kPlainThreads, 0, s>>>(rho0, rho_off, runs, tiles, partials);
    else if (Q == 7) init_scale_partials_kernel<7><<<ntiles, kPlainThreads, 0, s>>>(rho0, rho_off, runs, tiles, partials);
    else return cudaErrorInvalidValue;
    init_scale_finalize_kernel<<<fin_blocks, 128, 0, s>>>(nruns, tile_begin, partials, runs);
  }
  return cudaGetLastError();
}

cudaError_t launch_mass_finalize(int nruns, const int32_t* tile_begin, const double* partials, const RunDesc* runs,
                                 const double* mass0, double* mass, double* energy, double* delta, int* flags,
                                 cudaStream_t s) {
  if (nruns == 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (nruns * 32 + threads - 1) / threads;
  mass_finalize_kernel<<<blocks, threads, 0, s>>>(nruns, tile_begin, partials, runs, mass0, mass, energy, delta, flags);
  return cudaGetLastError();
}

cudaError_t launch_recentre(int storage, Arena f, const RunDesc* runs, const Tile* tiles, int ntiles,
                            const double* delta, cudaStream_t s) {
  if (ntiles == 0) return cudaSuccess;
  if (storage == kF64) recentre_kernel<kF64><<<ntiles, kRecentreThreads, 0, s>>>(f, runs, tiles, delta);
  else if (storage == kF32) recentre_kernel<kF32><<<ntiles, kRecentreThreads, 0, s>>>(f, runs, tiles, delta);
  else if (storage == kF16S) recentre_kernel<kF16S><<<ntiles, kRecentreThreads, 0, s>>>(f, runs, tiles, delta);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t fma_peak(int fp64, double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  void* out = nullptr;
  e = cudaMalloc(&out, 1024 * sizeof(double));
  if (e != cudaSuccess) return e;
  const int threads = 1024, blocks = sms * 2;
  const int iters = fp64 ? 256 : 8192;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  for (int rep = 0; rep < 2; ++rep) {  // first pass warms up
    cudaEventRecord(t0, s);
    if (fp64) fma_peak_kernel<double><<<blocks, threads, 0, s>>>((double*)out, iters, 0.5);
    else fma_peak_kernel<float><<<blocks, threads, 0, s>>>((float*)out, iters, 0.5f);
    cudaEventRecord(t1, s);
  }
  e = cudaEventSynchronize(t1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  if (e == cudaSuccess) *flops_per_s = 2.0 * 8.0 * 8.0 * iters * (double)threads * blocks / (ms * 1e-3);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaFree(out);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace lbks
