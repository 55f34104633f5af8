// Device-side building blocks shared by every kernel: lattice speeds,
// storage conversion, and the fused collision of one site.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "lbks_internal.h"

namespace lbks {

// Lattice speeds c_i in the order 0, +1, -1, +2, -2, +3, -3 (Appendix A of the paper).
__host__ __device__ constexpr int speed(int i) { return i == 0 ? 0 : ((i & 1) ? (i + 1) / 2 : -(i / 2)); }
__host__ __device__ constexpr int cmax_of(int Q) { return (Q - 1) / 2; }

template <int ST> struct StorageType;
template <> struct StorageType<kF64> { using type = double; using compute = double; };
template <> struct StorageType<kF32> { using type = float; using compute = float; };
template <> struct StorageType<kF16S> { using type = __half; using compute = float; };

// Per-run constants in the compute type.
template <typename CT, int Q> struct Coef {
  CT a[Q], b[Q];
  CT r, rhobar, scale, inv_scale;
};

template <typename CT, int Q>
__device__ __forceinline__ Coef<CT, Q> load_coef(const RunDesc& d) {
  Coef<CT, Q> c;
  if constexpr (sizeof(CT) == 8) {
#pragma unroll
    for (int i = 0; i < Q; ++i) { c.a[i] = d.a[i]; c.b[i] = d.b[i]; }
    c.r = d.r; c.rhobar = d.rhobar; c.scale = d.scale; c.inv_scale = d.inv_scale;
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) { c.a[i] = d.af[i]; c.b[i] = d.bf[i]; }
    c.r = d.rf; c.rhobar = d.rhobarf; c.scale = d.scalef; c.inv_scale = d.inv_scalef;
  }
  return c;
}

// Explicitly rounded arithmetic: no contraction choices are left to the compiler.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ double to_compute(double v, double) { return v; }
__device__ __forceinline__ float to_compute(float v, float) { return v; }
__device__ __forceinline__ float to_compute(__half v, float scale) { return __fmul_rn(__half2float(v), scale); }

__device__ __forceinline__ void from_compute(double v, double, double* p) { *p = v; }
__device__ __forceinline__ void from_compute(float v, float, float* p) { *p = v; }
__device__ __forceinline__ void from_compute(float v, float inv_scale, __half* p) {
  *p = __float2half_rn(__fmul_rn(v, inv_scale));
}

// One site of Eq. LB_equation_ordinary in deviation form (see RunDesc):
//   rho = rhobar + sum_i g_i;  g_i <- r g_i + rho a_i + rho^2 b_i   (i >= 1),
//   g_0 <- sum_i g_i - sum_{i>=1} g_i   (the collision conserves mass: sum_i f^eq_i = rho
//                                        by the zeroth moments of the weights, Eq. cond_weight).
// Evaluating f*_0 from the conservation identity instead of r g_0 + rho a_0 keeps the
// rounded arithmetic exactly mass-conserving at every site: with r and a_i rounded,
// r + sum_i a_i = 1 holds only to ~1 ulp and the direct form scales every mode of rho
// by (1 + O(ulp)) per step (in FP32 a 1e-5 relative error after ~2000 steps).
// rho a_i is shared by the pair +-c; rho^2 b_i enters through an fma, so the small
// advection term is rounded relative to rho a_i (whose low bits change every step).
// Summation order and fma forms are fixed here (g_0 = sum_i g_i minus g*_{+1}, g*_{-1},
// g*_{+2}, ... in that order): every kernel family, including the resident kernel's
// plane-by-plane form of the same arithmetic, produces bitwise the same values.
template <typename CT>
__device__ __forceinline__ CT post_collision(CT r, CT g, CT rho, CT rho2, CT b, CT t) {
  return fma_rn(r, g, fma_rn(rho2, b, t));
}

template <int Q, typename CT>
__device__ __forceinline__ void collide(CT (&g)[Q], const Coef<CT, Q>& k) {
  CT sg = g[0];
#pragma unroll
  for (int i = 1; i < Q; ++i) sg = add_rn(sg, g[i]);
  const CT rho = add_rn(k.rhobar, sg);
  const CT rho2 = mul_rn(rho, rho);
  CT acc = sg;
#pragma unroll
  for (int p = 1; 2 * p < Q; ++p) {  // speeds +p (index 2p-1) and -p (index 2p)
    const CT t = mul_rn(rho, k.a[2 * p - 1]);  // a_{+p} = a_{-p}
    g[2 * p - 1] = post_collision(k.r, g[2 * p - 1], rho, rho2, k.b[2 * p - 1], t);
    acc = add_rn(acc, -g[2 * p - 1]);
    g[2 * p] = post_collision(k.r, g[2 * p], rho, rho2, k.b[2 * p], t);
    acc = add_rn(acc, -g[2 * p]);
  }
  g[0] = acc;
}

__device__ __forceinline__ int64_t wrap_site(int64_t x, int64_t N) {
  return x < 0 ? x + N : (x >= N ? x - N : x);
}

// Programmatic dependent launch (PTX ISA: griddepcontrol), for the kernels that run one
// step per launch (plain, reservoir, streaming, tau = 1 streaming).  They are launched
// with programmatic stream serialisation (launch_early), so that the next step's grid is
// scheduled while this one runs instead of after it.  Every thread first waits until
// the grid before it in the stream (the previous step, which reads this step's
// destination and writes its source) has completed and its writes are visible; only
// then does it touch global memory and let the next grid be scheduled.  In a grid
// launched without the attribute both instructions return at once.
__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with programmatic stream serialisation allowed (for kernels that start with
// wait_prior_grid): the grid may be scheduled before the kernel ahead of it in the
// stream has finished.  Other work in the stream (copies, event waits) orders it fully.
template <typename... KArgs, typename... Args>
cudaError_t launch_early(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lbks
