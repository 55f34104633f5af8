/* A plain C11 caller of the library, built by tests/test_abi_c.py with
 * gcc -std=c11 -pedantic -Werror against include/lb_ks.h: the header is valid C
 * and the entry points are callable from C.  Prints one "OK ..." line per check,
 * or "FAIL ..." and exits 1.  Without a usable device the constructors must
 * return LB_KS_ECUDA (no CPU fallback); with one, a short run is made.
 * "abi_check layout" instead prints, as "name value" lines, the size and field
 * offsets of lb_ks_opts and the header's constants, for comparison with the
 * Python binding. */
#include <math.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "lb_ks.h"

static int failures = 0;

static void check(int ok, const char *what) {
    printf("%s %s\n", ok ? "OK" : "FAIL", what);
    if (!ok) failures++;
}

static int print_layout(void) {
#define FIELD(f) printf("offset_%s %zu\n", #f, offsetof(lb_ks_opts, f))
    printf("sizeof_opts %zu\n", sizeof(lb_ks_opts));
    FIELD(precision);
    FIELD(dm_variant);
    FIELD(recentre_every);
    FIELD(kernel);
    FIELD(steps_per_launch);
    FIELD(sites_per_thread);
    FIELD(threads_per_block);
    FIELD(use_graph);
    FIELD(autotune);
    FIELD(stream);
    FIELD(cluster_size);
#undef FIELD
#define CONST(c) printf("%s %d\n", #c, (int)(c))
    CONST(LB_KS_OK);
    CONST(LB_KS_EINVAL);
    CONST(LB_KS_ENOMEM);
    CONST(LB_KS_ECUDA);
    CONST(LB_KS_EUNSTABLE);
    CONST(LB_KS_ETIMEOUT);
    CONST(LB_KS_D1Q5);
    CONST(LB_KS_D1Q7);
    CONST(LB_KS_F64);
    CONST(LB_KS_F32);
    CONST(LB_KS_F16S);
    CONST(LB_KS_KERNEL_AUTO);
    CONST(LB_KS_KERNEL_PLAIN);
    CONST(LB_KS_KERNEL_STREAM);
    CONST(LB_KS_KERNEL_RESIDENT);
    CONST(LB_KS_KERNEL_COLLAPSE);
    CONST(LB_KS_DM_DERIVED);
    CONST(LB_KS_DM_PRINTED);
    CONST(LB_KS_WEIGHTS_FULL_INVERSE);
    CONST(LB_KS_LANE_FIELDS);
#undef CONST
    return 0;
}

int main(int argc, char **argv) {
    if (argc > 1 && strcmp(argv[1], "layout") == 0) return print_layout();
    lb_ks_opts o;
    memset(&o, 0xff, sizeof o);
    lb_ks_default_opts(&o);
    check(o.precision == LB_KS_F64 && o.dm_variant == LB_KS_DM_DERIVED && o.recentre_every == 0 &&
              o.kernel == LB_KS_KERNEL_AUTO && o.use_graph == 1 && o.autotune == 0 && o.stream == NULL &&
              o.cluster_size == 0,
          "default options");

    /* Host precompute (Sec. 2): sum_i A_i = 1 and sum_i B_i = 0 (w0 sums to 1; w1, w2,
     * w4, w6 to 0), J = dt / (2 dx). */
    double A[7], B[7], coef[9];
    int rc = lb_ks_params(LB_KS_D1Q7, 0.1, 1e-4, 1.5, LB_KS_DM_DERIVED, A, B, coef);
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < 7; ++i) {
        sa += A[i];
        sb += B[i];
    }
    check(rc == LB_KS_OK && fabs(sa - 1.0) < 1e-13 && sb == 0.0 && fabs(coef[4] - 5e-4) < 1e-18,
          "lb_ks_params: D1Q7 moments and J");
    check(lb_ks_params(6, 0.1, 1e-4, 1.5, 0, A, B, NULL) == LB_KS_EINVAL, "lb_ks_params: unknown scheme");

    const double tf = lb_ks_tau_fit(LB_KS_D1Q7, 0.1, 1e-4);
    check(isfinite(tf) && tf >= 1.0 && isnan(lb_ks_tau_fit(6, 0.1, 1e-4)), "lb_ks_tau_fit");

    double g = -1.0;
    rc = lb_ks_max_growth(LB_KS_D1Q7, 0.1, 1e-4, 1.5, 0, 0.0, 128, &g);
    check(rc == LB_KS_OK && isfinite(g) && g <= 1.05 * 0.25, "lb_ks_max_growth: a stable setting");
    check(lb_ks_max_growth(LB_KS_D1Q7, 0.1, 1e-4, 1.5, 0, 0.0, 0, &g) == LB_KS_EINVAL, "lb_ks_max_growth: nk < 1");

    /* Handles. */
    double rho0[64], rho[64];
    double m0 = 0.0;
    for (int x = 0; x < 64; ++x) {
        rho0[x] = 0.01 * cos(2.0 * 3.14159265358979323846 * 3.0 * x / 64.0) + 0.001 * x / 64.0;
        m0 += rho0[x];
    }
    lb_ks_t *h = (lb_ks_t *)&o; /* any non-NULL value: a failed constructor must clear it */
    check(lb_ks_init(&h, LB_KS_D1Q7, 6, 0.6, 1e-4, 1.5, rho0, NULL) == LB_KS_EINVAL && h == NULL &&
              strlen(lb_ks_last_error(NULL)) > 0,
          "lb_ks_init: N below 2 c_max + 1");
    h = (lb_ks_t *)&o;
    rc = lb_ks_init(&h, LB_KS_D1Q7, 64, 6.4, 1e-4, 1.5, rho0, NULL);
    if (rc == LB_KS_ECUDA) {
        check(h == NULL && strlen(lb_ks_last_error(NULL)) > 0, "lb_ks_init: no usable device is LB_KS_ECUDA");
    } else {
        double mass = 0.0, energy = 0.0;
        check(rc == LB_KS_OK && h != NULL, "lb_ks_init on a device");
        check(lb_ks_step(h, 100) == LB_KS_OK && lb_ks_rho(h, rho) == LB_KS_OK &&
                  lb_ks_mass_energy(h, &mass, &energy) == LB_KS_OK && lb_ks_steps_done(h) == 100,
              "100 steps, rho, mass");
        check(fabs(mass - m0) < 1e-12 && energy > 0.0 && isfinite(rho[0]), "mass conserved");
        lb_ks_free(h);
    }

    lb_ks_free(NULL);
    size_t bytes = 0;
    check(lb_ks_steps_done(NULL) == -1 && lb_ks_launches(NULL) == -1 && lb_ks_state_bytes(NULL, &bytes) == LB_KS_EINVAL &&
              lb_ks_step(NULL, 1) == LB_KS_EINVAL && lb_ks_rho(NULL, rho) == LB_KS_EINVAL &&
              lb_ks_set_link_test(NULL, 0, 16u) == LB_KS_EINVAL,
          "NULL handles");
    return failures ? 1 : 0;
}
