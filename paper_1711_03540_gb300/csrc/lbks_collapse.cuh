// The tau = 1 collapse of the LB scheme (one stored value per site).
//
// At tau = 1 the BGK collision of Eq. LB_equation_ordinary sets f*_i = f^eq_i(rho)
// (Eq. feq), so after streaming rho'(x) = sum_i f^eq_i(rho(x - c_i)): the state is
// rho alone.  f^eq_i = A_i rho + B_i rho^2 with A_i even and B_i odd in c_i, and
// sum_i A_i = 1, sum_i B_i = 0 (the moment conditions of Sec. 2), so the +c and -c
// planes pair into a symmetric stencil of half-width c_max:
//
//   rho'(x) = rho(x) + sum_{c=1}^{c_max} { A_c [rho(x-c) + rho(x+c) - 2 rho(x)]
//                                         + B_c [rho(x-c) - rho(x+c)] [rho(x-c) + rho(x+c)] }.
//
// Stored as the deviation delta = rho - rhobar (rhobar = 0 for FP64 storage, the
// run's initial mean for FP32); the products use rho(x-c) + rho(x+c) = 2 rhobar +
// delta(x-c) + delta(x+c).  A constant field stays exactly constant in floating
// point (every bracket is an exact zero), so the rounding has no bias from rhobar.
#pragma once

#include "lbks_device.cuh"

namespace lbks {

// Per-run constants of the collapsed step in the compute type.
template <typename CT, int C> struct CollapseCoef {
  CT A[C + 1], B[C + 1];  // index c = 1..C: A_{+c}, B_{+c}
  CT two_rhobar;
};

template <typename CT, int C>
__device__ __forceinline__ CollapseCoef<CT, C> load_collapse_coef(const RunDesc& d) {
  CollapseCoef<CT, C> k;
#pragma unroll
  for (int c = 1; c <= C; ++c) {
    k.A[c] = static_cast<CT>(d.A[2 * c - 1]);
    k.B[c] = static_cast<CT>(d.B[2 * c - 1]);
  }
  k.A[0] = k.B[0] = CT(0);
  k.two_rhobar = static_cast<CT>(2.0 * d.rhobar);
  return k;
}

// New deviation of one site from its own value d0 and its neighbours' dl[c] =
// delta(x - c), dr[c] = delta(x + c).  The 2 c_max terms are summed into a
// separate increment (their roundings are at the increment's scale, ~1e-3 of
// rho) and added to d0 once: one rounding at the scale of rho per step instead
// of 2 c_max, which in FP32 would bias the slow long-wave modes.  Every kernel of
// the collapse family calls this with the same operands, so their results agree
// bitwise.
template <typename CT, int C>
__device__ __forceinline__ CT collapse_site(CT d0, const CT (&dl)[C + 1], const CT (&dr)[C + 1],
                                            const CollapseCoef<CT, C>& k) {
  CT inc = CT(0);
#pragma unroll
  for (int c = 1; c <= C; ++c) {
    const CT s = add_rn(dl[c], dr[c]);
    const CT df = add_rn(dl[c], -dr[c]);
    const CT lap = fma_rn(CT(-2), d0, s);                  // rho(x-c) + rho(x+c) - 2 rho(x)
    const CT q = mul_rn(df, add_rn(k.two_rhobar, s));      // rho(x-c)^2 - rho(x+c)^2
    inc = fma_rn(k.A[c], lap, inc);
    inc = fma_rn(k.B[c], q, inc);
  }
  return add_rn(d0, inc);
}

}  // namespace lbks
