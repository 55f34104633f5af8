// Host precompute of the scheme's constants (FP64): lb_ks_params and lb_ks_tau_fit.
#include <cmath>
#include <cstring>

#include "../../include/lb_ks.h"

namespace {

// Velocity order 0, +1, -1, +2, -2, +3, -3 (Appendix A).  Weights of
// Eq. weight_D1Q5 (w0, w1, w2, w4); D1Q7 uses the same sets with zeros at
// c = +-3 and adds w6 of Eq. weight_D1Q7 (Sec. 2.3 refers to both equations).
constexpr double kW0[7] = {1.0, 0, 0, 0, 0, 0, 0};
constexpr double kW1[7] = {0.0, 2.0 / 3.0, -2.0 / 3.0, -1.0 / 12.0, 1.0 / 12.0, 0, 0};
constexpr double kW2[7] = {-5.0 / 4.0, 2.0 / 3.0, 2.0 / 3.0, -1.0 / 24.0, -1.0 / 24.0, 0, 0};
constexpr double kW4[7] = {1.0 / 4.0, -1.0 / 6.0, -1.0 / 6.0, 1.0 / 24.0, 1.0 / 24.0, 0, 0};
constexpr double kW6[7] = {-1.0 / 36.0, 1.0 / 48.0, 1.0 / 48.0, -1.0 / 120.0, -1.0 / 120.0, 1.0 / 720.0, 1.0 / 720.0};

}  // namespace

extern "C" int lb_ks_params(int scheme, double dx, double dt, double tau, int dm_variant, double* A, double* B,
                            double* coef) {
  if (scheme != LB_KS_D1Q5 && scheme != LB_KS_D1Q7) return LB_KS_EINVAL;
  if (!(dx > 0.0) || !(dt > 0.0) || !(tau > 0.5) || !std::isfinite(dx) || !std::isfinite(dt) || !std::isfinite(tau))
    return LB_KS_EINVAL;
  if (dm_variant != LB_KS_DM_DERIVED && dm_variant != LB_KS_DM_PRINTED) return LB_KS_EINVAL;
  if (!A || !B) return LB_KS_EINVAL;
  const double alpha = dx, beta = dt;
  // Eq. T_form, as T_i + 1.
  const double t1 = tau;                                    // T1 + 1
  const double t2 = 2.0 * tau * tau - tau;                  // T2 + 1
  const double t3 = 6.0 * tau * tau * tau - 6.0 * tau * tau + tau;   // T3 + 1
  const double t4 = (tau - 1.0) * (24.0 * tau * tau * tau - 12.0 * tau * tau + 2.0 * tau + 1.0) + 1.0;  // T4 + 1
  const double a2 = alpha * alpha, a4 = a2 * a2;
  // Table 2.
  const double J = beta / (2.0 * alpha);
  const double K = -2.0 * beta * t1 / (a2 * t2);
  const double M = -24.0 * beta * t1 / (a4 * t4);
  double dM = 0.0, E = 0.0;
  if (scheme == LB_KS_D1Q7) {
    // Eq. delta_M; the bracket's second term is (T3+1)/(T2+1) in the derived
    // reading (the one that cancels the beta d4 term of Eq. KS_trunc2).
    const double second = dm_variant == LB_KS_DM_PRINTED ? t3 / t4 : t3 / t2;
    dM = -24.0 * beta * beta * t1 / (a4 * t4) * (t2 / (2.0 * t1) - second);
    // delta f^eq of Sec. 2.2: coefficient of rho w6.
    E = 120.0 * t1 * beta / (t4 * a4);
  }
  const double Mp = M + dM;
  for (int i = 0; i < scheme; ++i) {
    A[i] = kW0[i] + K * kW2[i] + Mp * kW4[i] + E * kW6[i];
    B[i] = J * kW1[i];
    if (!std::isfinite(A[i]) || !std::isfinite(B[i])) return LB_KS_EINVAL;
  }
  if (coef) {
    const double c[9] = {t1 - 1.0, t2 - 1.0, t3 - 1.0, t4 - 1.0, J, K, M, dM, E};
    std::memcpy(coef, c, sizeof(c));
  }
  return LB_KS_OK;
}

extern "C" double lb_ks_tau_fit(int scheme, double dX, double dT) {
  if ((scheme != LB_KS_D1Q5 && scheme != LB_KS_D1Q7) || !(dX > 0.0) || !(dT > 0.0)) return std::nan("");
  // Eq. A_B_fit_D1Q5 / Eq. A_B_fit_D1Q7, then Eq. general_tau_formula.
  const double A = scheme == LB_KS_D1Q5 ? 0.103 * std::pow(dX, -0.381) : 0.0886 * std::pow(dX, -0.472);
  const double Bc = scheme == LB_KS_D1Q5 ? -13.2 * dX + 6.56 : -12.5 * dX + 6.64;
  const double lg = std::log10(dT);
  return lg >= -Bc ? A * (lg + Bc) * (lg + Bc) + 1.0 : 1.0;
}
