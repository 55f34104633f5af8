/*
 * lbks_oracle.c -- plain FP64 CPU oracle for the lattice Boltzmann (LB) scheme
 * for the Kuramoto-Sivashinsky (KS) equation of Otomo, Boghosian & Dubois,
 * "Efficient lattice Boltzmann models for the Kuramoto-Sivashinsky equation"
 * (arXiv:1711.03540).
 *
 * TEST INFRASTRUCTURE. This file is the independent checker of the CUDA
 * library: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, table or header with the CUDA path.
 * Every constant below is typed in from the paper.
 *
 * It is deliberately slow and literal: the equilibrium is evaluated every
 * step in the paper's own form (weights times coefficients), the collision
 * is the BGK rule as printed, and streaming is a push with modular indices.
 *
 * Readings where the paper is ambiguous (each one pinned by a test):
 *  - delta M (Eq. delta_M): the bracket's second denominator is taken as
 *    (T2+1), the value the truncation-error expression Eq. KS_trunc2 needs;
 *    dm_variant = 1 selects the printed (T4+1).
 *  - D1Q7 uses the D1Q5 weights w0, w1, w2, w4 padded with zeros at c = +-3,
 *    plus the 7-speed w6 of Eq. weight_D1Q7 (Sec. 2.3 points to both sets).
 *    The dm_variant bit 2 (value 2) selects the other reading, w1, w2, w4 of the
 *    full 7-speed inverse of Appendix A, as an ablation.
 *  - Velocity order is that of the Vandermonde columns of Appendix A:
 *    0, +1, -1, +2, -2, +3, -3.
 *  - "+-" in Eq. weight_D1Q5 is the value at +c, "-+" its negative.
 *  - The state is initialised at equilibrium, f_i = f_i^eq(rho0).
 *  - The front test's fixed end values (Table 5) are imposed with reservoir
 *    nodes: the boundary node and c_max ghost nodes beyond it are reset to
 *    f^eq(rho_boundary) every step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LBO_OK 0
#define LBO_EINVAL -1
#define LBO_ENOMEM -2

/* Lattice speeds, Appendix A (Vandermonde column order). */
static const int C_Q5[5] = {0, 1, -1, 2, -2};
static const int C_Q7[7] = {0, 1, -1, 2, -2, 3, -3};

/* Eq. weight_D1Q5, padded with zeros at c = +-3 for D1Q7 (Sec. 2.3). */
static const double W0[7] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
static const double W1[7] = {0.0, 2.0 / 3.0, -2.0 / 3.0, -1.0 / 12.0, 1.0 / 12.0, 0.0, 0.0};
static const double W2[7] = {-5.0 / 4.0, 2.0 / 3.0, 2.0 / 3.0, -1.0 / 24.0, -1.0 / 24.0, 0.0, 0.0};
static const double W3[7] = {0.0, -1.0 / 6.0, 1.0 / 6.0, 1.0 / 12.0, -1.0 / 12.0, 0.0, 0.0};
static const double W4[7] = {1.0 / 4.0, -1.0 / 6.0, -1.0 / 6.0, 1.0 / 24.0, 1.0 / 24.0, 0.0, 0.0};
/* Eq. weight_D1Q7 (7-speed set only). */
static const double W5[7] = {0.0, 1.0 / 48.0, -1.0 / 48.0, -1.0 / 60.0, 1.0 / 60.0, 1.0 / 240.0, -1.0 / 240.0};
static const double W6[7] = {-1.0 / 36.0, 1.0 / 48.0, 1.0 / 48.0, -1.0 / 120.0, -1.0 / 120.0, 1.0 / 720.0, 1.0 / 720.0};
/* The other rows of the full inverse of Appendix A's 7x7 moment matrix (Eq.
 * cond_weight for p = 0..6; the appendix prints only w5 and w6 of it), used only by
 * the weight ablation (variant bit 2): the alternative reading of Sec. 2.3. */
static const double WF1[7] = {0.0, 3.0 / 4.0, -3.0 / 4.0, -3.0 / 20.0, 3.0 / 20.0, 1.0 / 60.0, -1.0 / 60.0};
static const double WF2[7] = {-49.0 / 36.0, 3.0 / 4.0, 3.0 / 4.0, -3.0 / 40.0, -3.0 / 40.0, 1.0 / 180.0, 1.0 / 180.0};
static const double WF3[7] = {0.0, -13.0 / 48.0, 13.0 / 48.0, 1.0 / 6.0, -1.0 / 6.0, -1.0 / 48.0, 1.0 / 48.0};
static const double WF4[7] = {7.0 / 18.0, -13.0 / 48.0, -13.0 / 48.0, 1.0 / 12.0, 1.0 / 12.0, -1.0 / 144.0, -1.0 / 144.0};

/* Deliberate mistakes that the tests plant to show that the pins catch them.
 * 0 = none (the only value used outside those tests). */
static int g_mutation = 0;
void lbo_set_mutation(int m) { g_mutation = m; }

static const int *speeds(int Q) { return Q == 5 ? C_Q5 : C_Q7; }

int lbo_speed(int Q, int i) {
    if ((Q != 5 && Q != 7) || i < 0 || i >= Q) return 0;
    return speeds(Q)[i];
}

/* w^(l)_i for l = 0..6 as used by the scheme with Q speeds (w5, w6 only for Q = 7). */
int lbo_weight(int Q, int l, int i, double *w) {
    if ((Q != 5 && Q != 7) || i < 0 || i >= Q || l < 0 || l > 6) return LBO_EINVAL;
    if (Q == 5 && l > 4) return LBO_EINVAL;
    const double *tab[7] = {W0, W1, W2, W3, W4, W5, W6};
    *w = tab[l][i];
    return LBO_OK;
}

/* w^(l)_i of the full 7-speed inverse (l = 0..6), for the weight ablation and its pins. */
int lbo_weight_full(int l, int i, double *w) {
    if (i < 0 || i >= 7 || l < 0 || l > 6) return LBO_EINVAL;
    const double *tab[7] = {W0, WF1, WF2, WF3, WF4, W5, W6};
    *w = tab[l][i];
    return LBO_OK;
}

/* Eq. T_form: closed forms of T_i = sum_{n>=1} (1-1/tau)^n [(n+1)^i - n^i], tau > 1/2. */
static void t_closed_forms(double tau, double T[5]) {
    T[0] = 0.0;
    T[1] = tau - 1.0;
    T[2] = 2.0 * tau * tau - tau - 1.0;
    T[3] = 6.0 * tau * tau * tau - 6.0 * tau * tau + tau - 1.0;
    T[4] = (tau - 1.0) * (24.0 * tau * tau * tau - 12.0 * tau * tau + 2.0 * tau + 1.0);
}

/*
 * Coefficients of the equilibrium.
 * out[0..3] = T1..T4 (Eq. T_form)
 * out[4] = J, out[5] = K, out[6] = M        (Table 2; X = alpha x, T = beta t, Eq. scaling)
 * out[7] = delta M (Eq. delta_M; D1Q7 only, 0 for D1Q5)
 * out[8] = E, the coefficient of rho w6 in the D1Q7 equilibrium (delta f^eq, Sec. 2.2)
 */
int lbo_coefficients(int Q, double alpha, double beta, double tau, int dm_variant, double out[9]) {
    if ((Q != 5 && Q != 7) || !(alpha > 0.0) || !(beta > 0.0) || !(tau > 0.5)) return LBO_EINVAL;
    if (dm_variant < 0 || dm_variant > 3) return LBO_EINVAL;
    double T[5];
    t_closed_forms(tau, T);
    double J = beta / (2.0 * alpha);
    double K = -2.0 * beta * (T[1] + 1.0) / (alpha * alpha * (T[2] + 1.0));
    double M = -24.0 * beta * (T[1] + 1.0) / (pow(alpha, 4) * (T[4] + 1.0));
    double dM = 0.0, E = 0.0;
    if (Q == 7) {
        double second = (dm_variant & 1) ? (T[3] + 1.0) / (T[4] + 1.0) : (T[3] + 1.0) / (T[2] + 1.0);
        dM = -24.0 * beta * beta * (T[1] + 1.0) / (pow(alpha, 4) * (T[4] + 1.0)) *
             ((T[2] + 1.0) / (2.0 * (T[1] + 1.0)) - second);
        E = 120.0 * (T[1] + 1.0) * beta / ((T[4] + 1.0) * pow(alpha, 4));
    }
    out[0] = T[1];
    out[1] = T[2];
    out[2] = T[3];
    out[3] = T[4];
    out[4] = J;
    out[5] = K;
    out[6] = M;
    out[7] = dM;
    out[8] = E;
    return LBO_OK;
}

/* Scheme constants held by one run. */
typedef struct {
    int Q;
    int full_weights; /* D1Q7 weight ablation: the full 7-speed inverse for w1, w2, w4 */
    double tau, J, K, M, dM, E;
} scheme_t;

static int make_scheme(int Q, double alpha, double beta, double tau, int dm_variant, int advection,
                       scheme_t *s) {
    double c[9];
    int rc = lbo_coefficients(Q, alpha, beta, tau, dm_variant, c);
    if (rc) return rc;
    s->Q = Q;
    s->full_weights = Q == 7 && (dm_variant & 2);
    s->tau = tau;
    s->J = advection ? c[4] : 0.0;
    s->K = c[5];
    s->M = c[6];
    s->dM = c[7];
    s->E = c[8];
    if (g_mutation == 3) s->K = 0.0;  /* planted: drop the K w2 term */
    if (g_mutation == 4) s->J = -s->J; /* planted: wrong sign of the advection term */
    if (g_mutation == 5) s->E = 0.0;  /* planted: drop delta f^eq */
    if (g_mutation == 6) s->M = 0.0;  /* planted: drop the M w4 term */
    if (g_mutation == 7) s->dM = 0.0; /* planted: drop delta M */
    return LBO_OK;
}

/* f^eq_i(rho): Eq. feq for D1Q5 (Sec. 2.3), and the D1Q7 form of Sec. 2.3
 * rho {w0 + K w2 + (M + dM) w4 + E w6} + rho^2 J w1. */
static void equilibrium(const scheme_t *s, double rho, double *feq) {
    for (int i = 0; i < s->Q; ++i) {
        double lin;
        const double *w1 = s->full_weights ? WF1 : W1;
        double w1_swapped[7];
        if (g_mutation == 9) { /* planted: the w1 entries of c = +2 and c = -2 exchanged */
            for (int j = 0; j < s->Q; ++j) w1_swapped[j] = w1[j];
            w1_swapped[3] = w1[4];
            w1_swapped[4] = w1[3];
            w1 = w1_swapped;
        }
        const double *w2 = s->full_weights ? WF2 : W2;
        const double *w4 = s->full_weights ? WF4 : W4;
        if (s->Q == 5)
            lin = W0[i] + s->K * w2[i] + s->M * w4[i];
        else
            lin = W0[i] + s->K * w2[i] + (s->M + s->dM) * w4[i] + s->E * W6[i];
        feq[i] = rho * lin + rho * rho * s->J * w1[i];
        if (g_mutation == 10) feq[i] = rho * lin + rho * s->J * w1[i]; /* planted: linear advection term */
    }
}

int lbo_feq(int Q, double alpha, double beta, double tau, int dm_variant, int advection, double rho,
            double *feq) {
    scheme_t s;
    int rc = make_scheme(Q, alpha, beta, tau, dm_variant, advection, &s);
    if (rc) return rc;
    equilibrium(&s, rho, feq);
    return LBO_OK;
}

static int64_t wrap(int64_t x, int64_t N) {
    int64_t r = x % N;
    return r < 0 ? r + N : r;
}

/* One periodic step of Eq. LB_equation_ordinary on populations f[i*N + x]:
 * rho = sum_i f_i, f*_i = f_i - (f_i - f^eq_i)/tau, f_i(x + c_i) <- f*_i(x). */
static void step_periodic(const scheme_t *s, int64_t N, const double *f, double *fn) {
    const int *c = speeds(s->Q);
    double feq[7];
    for (int64_t x = 0; x < N; ++x) {
        double rho = 0.0;
        for (int i = 0; i < s->Q; ++i) rho += f[(int64_t)i * N + x];
        equilibrium(s, rho, feq);
        for (int i = 0; i < s->Q; ++i) {
            double fi = f[(int64_t)i * N + x];
            double fstar = fi - (fi - feq[i]) / s->tau;
            if (g_mutation == 8) fstar = fi - (fi - feq[i]) * s->tau; /* planted: relaxed by tau, not 1/tau */
            int ci = g_mutation == 1 ? -c[i] : c[i]; /* planted: streaming direction flipped */
            fn[(int64_t)i * N + wrap(x + ci, N)] = fstar;
        }
    }
}

/* Front-test boundary (Table 5): the array holds nodes j = -cmax .. Nn-1+cmax
 * at index j + cmax.  Nodes j <= 0 and j >= Nn-1 are reservoirs. */
static void reset_reservoirs(const scheme_t *s, int64_t Nn, int cmax, double rho_l, double rho_r,
                             double *f) {
    int64_t Ne = Nn + 2 * cmax;
    double fl[7], fr[7];
    equilibrium(s, rho_l, fl);
    equilibrium(s, rho_r, fr);
    for (int64_t g = 0; g <= cmax; ++g)
        for (int i = 0; i < s->Q; ++i) f[(int64_t)i * Ne + g] = fl[i];
    for (int64_t g = Nn - 1 + cmax; g < Ne; ++g)
        for (int i = 0; i < s->Q; ++i) f[(int64_t)i * Ne + g] = fr[i];
}

static void step_reservoir(const scheme_t *s, int64_t Ne, const double *f, double *fn) {
    const int *c = speeds(s->Q);
    double feq[7];
    for (int64_t x = 0; x < Ne; ++x) {
        double rho = 0.0;
        for (int i = 0; i < s->Q; ++i) rho += f[(int64_t)i * Ne + x];
        equilibrium(s, rho, feq);
        for (int i = 0; i < s->Q; ++i) {
            double fi = f[(int64_t)i * Ne + x];
            double fstar = fi - (fi - feq[i]) / s->tau;
            if (g_mutation == 8) fstar = fi - (fi - feq[i]) * s->tau; /* planted: relaxed by tau, not 1/tau */
            int64_t y = x + (g_mutation == 1 ? -c[i] : c[i]);
            if (y >= 0 && y < Ne) fn[(int64_t)i * Ne + y] = fstar;
        }
    }
}

/*
 * Run nsteps steps from f = f^eq(rho0) and return rho = sum_i f_i at T = nsteps*beta.
 *   boundary 0: periodic lattice of N sites, X_j = j alpha.
 *   boundary 1: front test, N nodes X_j = X_m + j alpha with fixed rho_left / rho_right
 *               at j = 0 and j = N-1 (and reservoir nodes beyond them).
 *   advection 0 sets J = 0 (linear test switch).
 * f_out (optional) receives the final populations, layout f[i*N + x] over the N nodes.
 */
int lbo_run(int Q, int64_t N, double alpha, double beta, double tau, int dm_variant, int advection,
            int boundary, double rho_left, double rho_right, const double *rho0, int64_t nsteps,
            double *rho_out, double *f_out) {
    scheme_t s;
    int rc = make_scheme(Q, alpha, beta, tau, dm_variant, advection, &s);
    if (rc) return rc;
    int cmax = Q == 5 ? 2 : 3;
    if (N < 1 || nsteps < 0 || (boundary != 0 && boundary != 1)) return LBO_EINVAL;
    int64_t pad = boundary == 1 ? cmax : 0;
    int64_t Ne = N + 2 * pad;
    double *f = (double *)malloc(sizeof(double) * (size_t)Q * (size_t)Ne);
    double *fn = (double *)malloc(sizeof(double) * (size_t)Q * (size_t)Ne);
    if (!f || !fn) {
        free(f);
        free(fn);
        return LBO_ENOMEM;
    }
    double feq[7];
    for (int64_t g = 0; g < Ne; ++g) {
        int64_t j = g - pad;
        double r = j < 0 ? rho_left : (j >= N ? rho_right : rho0[j]);
        equilibrium(&s, r, feq);
        for (int i = 0; i < Q; ++i) f[(int64_t)i * Ne + g] = feq[i];
    }
    if (boundary == 1) {
        reset_reservoirs(&s, N, cmax, rho_left, rho_right, f);
        memcpy(fn, f, sizeof(double) * (size_t)Q * (size_t)Ne);
    }
    for (int64_t n = 0; n < nsteps; ++n) {
        if (boundary == 0) {
            step_periodic(&s, N, f, fn);
        } else {
            step_reservoir(&s, Ne, f, fn);
            reset_reservoirs(&s, N, cmax, rho_left, rho_right, fn);
        }
        double *t = f;
        f = fn;
        fn = t;
    }
    for (int64_t j = 0; j < N; ++j) {
        double rho = 0.0;
        for (int i = 0; i < Q; ++i) rho += f[(int64_t)i * Ne + j + pad];
        rho_out[j] = rho;
        if (f_out)
            for (int i = 0; i < Q; ++i) f_out[(int64_t)i * N + j] = f[(int64_t)i * Ne + j + pad];
    }
    free(f);
    free(fn);
    return LBO_OK;
}

/*
 * Independent periodic runs (an ensemble), rho0 and rho_out concatenated in run
 * order.  Runs are spread over nthreads OpenMP threads (each run is the same
 * serial loop as lbo_run).  Returns the number of threads used through *used.
 */
int lbo_run_batch(int Q, int32_t nruns, const int64_t *N, const double *alpha, const double *beta,
                  const double *tau, int dm_variant, const double *rho0, int64_t nsteps,
                  double *rho_out, int nthreads, int *used) {
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nruns + 1));
    if (!off) return LBO_ENOMEM;
    off[0] = 0;
    for (int32_t r = 0; r < nruns; ++r) off[r + 1] = off[r] + N[r];
    int rc_all = LBO_OK;
    int nt = nthreads > 0 ? nthreads : 1;
#ifdef _OPENMP
    *used = nt;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(min : rc_all)
#else
    *used = 1;
#endif
    for (int32_t r = 0; r < nruns; ++r) {
        int rc = lbo_run(Q, N[r], alpha[r], beta[r], tau[r], dm_variant, 1, 0, 0.0, 0.0,
                         rho0 + off[r], nsteps, rho_out + off[r], NULL);
        if (rc < rc_all) rc_all = rc;
    }
    free(off);
    return rc_all;
}
