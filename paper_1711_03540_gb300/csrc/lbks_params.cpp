// Host precompute of the scheme's constants (FP64): lb_ks_params and lb_ks_tau_fit.
#include <algorithm>
#include <cmath>
#include <complex>
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
// Ablation (LB_KS_WEIGHTS_FULL_INVERSE): w1, w2, w4 of the full 7-speed inverse of
// Appendix A's D1Q7 moment matrix (the rule of Eq. cond_weight for p = 0..6; the
// appendix prints only w5 and w6 of that inverse).
constexpr double kF1[7] = {0.0, 3.0 / 4.0, -3.0 / 4.0, -3.0 / 20.0, 3.0 / 20.0, 1.0 / 60.0, -1.0 / 60.0};
constexpr double kF2[7] = {-49.0 / 36.0, 3.0 / 4.0, 3.0 / 4.0, -3.0 / 40.0, -3.0 / 40.0, 1.0 / 180.0, 1.0 / 180.0};
constexpr double kF4[7] = {7.0 / 18.0, -13.0 / 48.0, -13.0 / 48.0, 1.0 / 12.0, 1.0 / 12.0, -1.0 / 144.0, -1.0 / 144.0};

}  // namespace

extern "C" int lb_ks_params(int scheme, double dx, double dt, double tau, int dm_variant, double* A, double* B,
                            double* coef) {
  if (scheme != LB_KS_D1Q5 && scheme != LB_KS_D1Q7) return LB_KS_EINVAL;
  if (!(dx > 0.0) || !(dt > 0.0) || !(tau > 0.5) || !std::isfinite(dx) || !std::isfinite(dt) || !std::isfinite(tau))
    return LB_KS_EINVAL;
  if (dm_variant < 0 || dm_variant > (LB_KS_DM_PRINTED | LB_KS_WEIGHTS_FULL_INVERSE)) return LB_KS_EINVAL;
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
    const double second = (dm_variant & LB_KS_DM_PRINTED) ? t3 / t4 : t3 / t2;
    dM = -24.0 * beta * beta * t1 / (a4 * t4) * (t2 / (2.0 * t1) - second);
    // delta f^eq of Sec. 2.2: coefficient of rho w6.
    E = 120.0 * t1 * beta / (t4 * a4);
  }
  const double Mp = M + dM;
  const bool full = scheme == LB_KS_D1Q7 && (dm_variant & LB_KS_WEIGHTS_FULL_INVERSE);
  const double* w1 = full ? kF1 : kW1;
  const double* w2 = full ? kF2 : kW2;
  const double* w4 = full ? kF4 : kW4;
  for (int i = 0; i < scheme; ++i) {
    A[i] = kW0[i] + K * w2[i] + Mp * w4[i] + E * kW6[i];
    B[i] = J * w1[i];
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

// ---------------------------------------------------------------- linear stability

namespace {

// Largest |lambda| of the linearised step's amplification matrix at phase kappa:
// G = D (r I + w a 1^T), D = diag(exp(-i kappa c_j)), r = 1 - 1/tau, w = 1/tau,
// a_j = d f^eq_j / d rho at the background state.  G is a diagonal matrix plus a
// rank-one term, so its characteristic polynomial is
//   p(lambda) = prod_j (lambda - r d_j) - sum_j u_j prod_{k != j} (lambda - r d_k),
// u = w D a; its roots are found by the Weierstrass (Durand-Kerner) iteration.
double max_abs_eigenvalue(int Q, const double* a, double tau, double kappa) {
  using cd = std::complex<double>;
  const double r = 1.0 - 1.0 / tau, w = 1.0 / tau;
  cd d[7], u[7];
  for (int j = 0; j < Q; ++j) {
    const int c = j == 0 ? 0 : ((j & 1) ? (j + 1) / 2 : -(j / 2));
    d[j] = std::polar(1.0, -kappa * c);
    u[j] = w * d[j] * a[j];
  }
  // coefficients of p, highest power first: p = sum_k coef[k] lambda^(Q - k)
  cd coef[8] = {};
  cd prod_all[8] = {};
  prod_all[0] = 1.0;
  int deg = 0;
  for (int j = 0; j < Q; ++j) {  // prod_j (lambda - r d_j)
    for (int k = deg + 1; k >= 1; --k) prod_all[k] -= r * d[j] * prod_all[k - 1];
    ++deg;
  }
  for (int k = 0; k <= Q; ++k) coef[k] = prod_all[k];
  for (int j = 0; j < Q; ++j) {  // - u_j prod_{k != j} (lambda - r d_k), degree Q - 1
    cd q[8] = {};
    q[0] = 1.0;
    int dg = 0;
    for (int k = 0; k < Q; ++k) {
      if (k == j) continue;
      for (int m = dg + 1; m >= 1; --m) q[m] -= r * d[k] * q[m - 1];
      ++dg;
    }
    for (int m = 0; m < Q; ++m) coef[m + 1] -= u[j] * q[m];
  }
  auto eval = [&](cd z) {
    cd v = coef[0];
    for (int k = 1; k <= Q; ++k) v = v * z + coef[k];
    return v;
  };
  cd z[7];
  const cd seed(0.4, 0.9);
  for (int k = 0; k < Q; ++k) z[k] = std::pow(seed, k) * 1.2;
  for (int it = 0; it < 500; ++it) {
    double change = 0.0;
    for (int k = 0; k < Q; ++k) {
      cd den = 1.0;
      for (int m = 0; m < Q; ++m)
        if (m != k) den *= z[k] - z[m];
      if (std::abs(den) == 0.0) den = 1e-300;
      const cd step = eval(z[k]) / den;
      z[k] -= step;
      change = std::max(change, std::abs(step));
    }
    if (change < 1e-15) break;
  }
  double best = 0.0;
  for (int k = 0; k < Q; ++k) best = std::max(best, std::abs(z[k]));
  return best;
}

}  // namespace

extern "C" int lb_ks_max_growth(int scheme, double dx, double dt, double tau, int dm_variant, double rho_bar, int nk,
                                double* growth) {
  if (!growth || nk < 1) return LB_KS_EINVAL;
  double A[7], B[7];
  const int rc = lb_ks_params(scheme, dx, dt, tau, dm_variant, A, B, nullptr);
  if (rc != LB_KS_OK) return rc;
  double a[7];
  for (int j = 0; j < scheme; ++j) a[j] = A[j] + 2.0 * B[j] * rho_bar;
  double best = -HUGE_VAL;
  for (int k = 1; k <= nk; ++k) {
    const double kappa = M_PI * k / nk;
    best = std::max(best, std::log(max_abs_eigenvalue(scheme, a, tau, kappa)) / dt);
  }
  *growth = best;
  return LB_KS_OK;
}
