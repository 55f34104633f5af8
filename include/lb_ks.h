/*
 * lb_ks.h -- C ABI of the GB300 (sm_103a) library for the lattice Boltzmann
 * scheme for the Kuramoto-Sivashinsky equation of Otomo, Boghosian & Dubois,
 * "Efficient lattice Boltzmann models for the Kuramoto-Sivashinsky equation"
 * (arXiv:1711.03540).
 *
 * The library advances periodic lattices with the BGK lattice Boltzmann
 * equation (Sec. 2, Eq. LB_equation_ordinary)
 *     f_i(x + c_i, t + 1) - f_i(x, t) = -(f_i - f^eq_i) / tau,
 *     f^eq_i = rho (w0_i + K w2_i + M' w4_i + E w6_i) + rho^2 J w1_i,  rho = sum_i f_i,
 * on D1Q5 (c = 0, +-1, +-2; M' = M, E = 0; Eq. feq) or D1Q7
 * (c = 0, +-1, +-2, +-3; M' = M + delta M, E = 120 beta (T1+1)/((T4+1) alpha^4);
 * Sec. 2.3), with J, K, M from Table 2, T_i from Eq. T_form and the scaling
 * X = alpha x, T = beta t (Eq. scaling): alpha = L / N, beta = dt.
 *
 * Conventions shared by every entry point:
 *  - Every function returns a status code (LB_KS_OK or a negative LB_KS_E*);
 *    no C++ exception crosses this boundary: a host allocation that fails
 *    inside a call returns LB_KS_ENOMEM (inside lb_ks_step it is also sticky,
 *    since the handle's step count may then be ahead of the work issued).
 *    lb_ks_last_error() gives a one-line reason for the last failure on a handle.
 *  - A handle owns its device memory (allocated in lb_ks_init /
 *    lb_ks_batch_init, released by lb_ks_free).  It never keeps or frees a
 *    pointer the caller passes in.  Input and output pointers may be host or
 *    device memory of the current device; the library tells them apart with
 *    cudaPointerGetAttributes.
 *  - Work is issued on the stream given in lb_ks_opts (NULL = the legacy
 *    default stream).  lb_ks_step returns without waiting; lb_ks_rho,
 *    lb_ks_mass_energy and lb_ks_save wait for the stream.  The stream must
 *    outlive the handle: lb_ks_free waits for it and returns the handle's
 *    device memory to the pool in its order.
 *  - Errors detected on the device (a non-finite FP64 mass at a guard step)
 *    are sticky: they are reported by the next call that waits, and every
 *    later call on the handle returns the same code.
 *  - One handle must not be used from two host threads at once.
 *  - There is no CPU fallback.  Without a usable CUDA device the
 *    constructors return LB_KS_ECUDA.
 */
#ifndef LB_KS_H
#define LB_KS_H

#include <stddef.h>
#include <stdint.h>

/* Symbols of the C ABI stay visible when the library is built with hidden default visibility. */
#if defined(__GNUC__)
#define LB_KS_API __attribute__((visibility("default")))
#else
#define LB_KS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define LB_KS_OK 0
#define LB_KS_EINVAL (-1)    /* invalid argument; nothing was done */
#define LB_KS_ENOMEM (-2)    /* device or host allocation failed */
#define LB_KS_ECUDA (-3)     /* CUDA runtime error, or no usable device */
#define LB_KS_EUNSTABLE (-4) /* non-finite FP64 mass found at a guard step (sticky) */
#define LB_KS_ETIMEOUT (-5)  /* a bounded device wait ran out (sticky): the two blocks of a
                                resident cluster stopped exchanging values (an internal error) */

/* Lattice schemes (Sec. 2.3): the number of speeds. */
#define LB_KS_D1Q5 5
#define LB_KS_D1Q7 7

/* Storage precision of the populations.
 * F64: FP64 storage and arithmetic.
 * F32: FP32 storage of f_i - w0_i rho_bar (rho_bar = the run's initial mean;
 *      w0 = (1, 0, ...), so only f_0 is offset), FP32 arithmetic.
 * F16S: the same deviations stored as FP16 times a per-run scale, FP32 arithmetic.
 * In F32 and F16S the FP64 mass guard (recentre_every) restores the run's
 * initial mass. */
#define LB_KS_F64 0
#define LB_KS_F32 1
#define LB_KS_F16S 2

/* Kernel family. */
#define LB_KS_KERNEL_AUTO 0     /* resident when every run fits its constraints, else plain (F64) / stream */
#define LB_KS_KERNEL_PLAIN 1    /* one thread per site, one launch per step (F64, F32) */
#define LB_KS_KERNEL_STREAM 2   /* HBM-streaming tiles, one launch per step (F32, F16S) */
#define LB_KS_KERNEL_RESIDENT 3 /* register-resident, many steps per launch (F64, F32, F16S) */
/* tau = 1 only (every run): at tau = 1 the BGK collision of Eq. LB_equation_ordinary
 * sets f* = f^eq(rho), so rho alone is the state and the step is the stencil
 * rho'(x) = sum_i f^eq_i(rho(x - c_i)), evaluated with the +c and -c speeds paired:
 * rho + sum_c A_c [rho(x-c) + rho(x+c) - 2 rho] + B_c [rho(x-c)^2 - rho(x+c)^2].
 * One stored plane (rho - rhobar) instead of Q; the same results as the other
 * families up to rounding (not bitwise).  F64 or F32; periodic or reservoir ends.
 * Never chosen by LB_KS_KERNEL_AUTO. */
#define LB_KS_KERNEL_COLLAPSE 4

/* Reading of Eq. delta_M. */
#define LB_KS_DM_DERIVED 0 /* bracket (T2+1)/(2(T1+1)) - (T3+1)/(T2+1), as Eq. KS_trunc2 needs */
#define LB_KS_DM_PRINTED 1 /* bracket with (T3+1)/(T4+1) as printed */
/* Flag, combinable with either reading (D1Q7 only): an ablation of the weight
 * reading.  By default D1Q7 uses the D1Q5 sets w1, w2, w4 padded with zeros at
 * c = +-3 (Sec. 2.3), the choice for which delta f^eq cancels the alpha^2 d6 error
 * term; with this flag it uses w1, w2, w4 of the full 7-speed inverse of Appendix A's
 * moment matrix (Eq. cond_weight for p = 0..6), whose 6th moments vanish, so that
 * delta f^eq leaves the alpha^2 d6 term at its D1Q5 size with the opposite sign
 * instead of removing it.  A negative control, not a usable scheme. */
#define LB_KS_WEIGHTS_FULL_INVERSE 2

typedef struct lb_ks lb_ks_t; /* opaque handle */

typedef struct lb_ks_opts {
    int32_t precision;         /* LB_KS_F64 (default), LB_KS_F32, LB_KS_F16S */
    int32_t dm_variant;        /* LB_KS_DM_DERIVED (default) or LB_KS_DM_PRINTED, optionally
                                  | LB_KS_WEIGHTS_FULL_INVERSE */
    int32_t recentre_every;    /* R > 0: every R steps compute the FP64 mass of every run and add
                                  (M0 - M)/N to f_0 at each site; 0 = never (default for F64) */
    int32_t kernel;            /* LB_KS_KERNEL_* */
    int32_t steps_per_launch;  /* resident kernel: steps kept on chip per launch; 0 = auto.  For
                                  the tau = 1 collapse, 1 selects its streaming kernel */
    int32_t sites_per_thread;  /* resident kernel: register slots per thread (4,6,8,12,16,18,20 for
                                  F32/F16S; 4,6,8 for F64; the tau = 1 collapse: 8,16,32 for
                                  F32, 8,16 for F64); 0 = auto */
    int32_t threads_per_block; /* resident kernel: a multiple of 32 up to 512; 0 = auto */
    int32_t use_graph;         /* 1 (default): replay captured CUDA graphs for step sequences */
    int32_t autotune;          /* resident kernel: 1 = at init, time a few tilings (sites per thread,
                                  threads per block, split of the blocks between whole and
                                  segmented lattices) on these lattices for a short run and keep
                                  the fastest; 0 (default) = fixed defaults */
    void *stream;              /* cudaStream_t; NULL = legacy default stream */
    int32_t cluster_size;      /* resident kernel, whole lattices: blocks per work group.  1 = one
                                  thread block; 2 = a cluster of two blocks (distributed shared
                                  memory), which holds lattices of up to 2 x threads x sites per
                                  thread whole instead of cutting them into segments; 0 (default)
                                  = 2 when some lattice needs it, else 1 (the autotuner tries both) */
} lb_ks_opts;

/* Fill *opts with the defaults listed above. */
LB_KS_API void lb_ks_default_opts(lb_ks_opts *opts);

/*
 * Host precompute of one run's constants (no GPU needed).
 * Sec. 2: T1..T4 (Eq. T_form), J, K, M (Table 2), delta M (Eq. delta_M),
 * E (delta f^eq, Sec. 2.2), with alpha = dx and beta = dt (Eq. scaling).
 *   A[i], B[i] (i < scheme): f^eq_i(rho) = A_i rho + B_i rho^2.
 *   coef[9] (may be NULL): T1, T2, T3, T4, J, K, M, delta M, E.
 * Returns LB_KS_EINVAL for an unknown scheme, dx <= 0, dt <= 0, tau <= 1/2
 * or a non-finite result (T4 + 1 = 0 near tau = 0.908).
 */
LB_KS_API int lb_ks_params(int scheme, double dx, double dt, double tau, int dm_variant, double *A, double *B,
                 double *coef);

/*
 * Minimum stable relaxation time fitted in Sec. 3 (Eq. general_tau_formula with
 * Eq. A_B_fit_D1Q5 / Eq. A_B_fit_D1Q7) for lattice spacing dX and time step dT.
 * Returns NaN for an unknown scheme or non-positive dX, dT.  The fit was made
 * on the paper's front test; it is advice, not a stability guarantee.
 */
LB_KS_API double lb_ks_tau_fit(int scheme, double dX, double dT);

/*
 * Linear stability of the scheme (no GPU needed): the largest growth rate per
 * unit time, ln(max |lambda|) / dt over all Q eigenvalues lambda of the linearised
 * step about the uniform state rho_bar, at phases kappa = pi k / nk, k = 1..nk
 * (the amplification matrix of Eq. LB_equation_ordinary with f^eq linearised:
 * diag(exp(-i kappa c_j)) ((1 - 1/tau) I + (1/tau) a 1^T), a_j = A_j + 2 B_j rho_bar).
 * Sec. 3 does not define "stable"; this library calls a run linearly unstable when
 * the rate exceeds 1.05 x 1/4, the largest growth rate of the KS equation itself.
 * *growth receives the rate.  Errors: as lb_ks_params, and LB_KS_EINVAL for
 * growth == NULL or nk < 1.
 */
LB_KS_API int lb_ks_max_growth(int scheme, double dx, double dt, double tau, int dm_variant, double rho_bar, int nk,
                               double *growth);

/*
 * Create a handle for one periodic lattice of N sites on [0, L):
 * alpha = L / N, beta = dt, relaxation time tau (>= 1; T4 + 1 vanishes near
 * 0.908 and the paper uses tau >= 1, Sec. 3), and initial density
 * rho0[N] (FP64, host or device, read once).  Populations start at
 * equilibrium, f_i = f^eq_i(rho0).  opts may be NULL (defaults).
 * Errors: LB_KS_EINVAL (unknown scheme, N < 2 c_max + 1 or N > 2^30, L <= 0,
 * dt <= 0, tau < 1, non-finite rho0, bad opts), LB_KS_ENOMEM, LB_KS_ECUDA.  On error
 * *h is set to NULL.  Not an error: when the linear check of lb_ks_max_growth
 * (nk = 128, about rho = 0) finds the run unstable, the handle is created and
 * lb_ks_last_error(h) starts with "warning:" (batch handles: checked when the
 * batch has at most 64 distinct (L/N, dt, tau)).
 */
LB_KS_API int lb_ks_init(lb_ks_t **h, int scheme, int64_t N, double L, double dt, double tau, const double *rho0,
               const lb_ks_opts *opts);

/*
 * Create a handle for nruns independent periodic lattices advanced together
 * (one ensemble).  Run r has N[r] sites on [0, L[r]), time step dt[r] and
 * relaxation time tau[r]; rho0 holds the initial densities of all runs
 * concatenated in run order (sum N[r] values, FP64, host or device).
 * The same argument rules and errors as lb_ks_init apply to every run; a
 * batch of more than 2^34 sites in all (more than the device's memory holds in
 * any storage) is LB_KS_EINVAL.
 */
LB_KS_API int lb_ks_batch_init(lb_ks_t **h, int scheme, int32_t nruns, const int64_t *N, const double *L,
                     const double *dt, const double *tau, const double *rho0, const lb_ks_opts *opts);

/*
 * Create a handle for nruns lattices with fixed-value ends, the boundary of the
 * travelling-front test of Sec. 3 (Table 5): run r has N[r] nodes
 * X_j = j L[r] / (N[r] - 1), j = 0 .. N[r]-1, on [0, L[r]]; the end nodes and
 * c_max ghost nodes beyond each end are held at f^eq(rho_left[r]) (j <= 0) and
 * f^eq(rho_right[r]) (j >= N[r]-1) every step, so populations streaming in
 * from outside carry the boundary state and those streaming out are dropped.
 * rho0 (sum N[r] values, host or device) initialises the nodes; its two end
 * values are replaced by the boundary values.  These lattices run on the plain
 * kernel family (every node collides once and pushes plane i to node j + c_i when
 * that node is interior), or on the tau = 1 collapse when opts->kernel is
 * LB_KS_KERNEL_COLLAPSE; the guard's
 * re-centring is not allowed (mass flows through the ends: recentre_every must
 * be 0); lb_ks_rho and lb_ks_mass_energy cover the N[r] nodes.
 * Errors: as lb_ks_batch_init, plus LB_KS_EINVAL for NULL or non-finite
 * boundary values, opts->kernel STREAM/RESIDENT, or recentre_every != 0.
 */
LB_KS_API int lb_ks_batch_init_reservoir(lb_ks_t **h, int scheme, int32_t nruns, const int64_t *N,
                                         const double *L, const double *dt, const double *tau,
                                         const double *rho0, const double *rho_left, const double *rho_right,
                                         const lb_ks_opts *opts);

/*
 * Advance every run of the handle by n >= 0 time steps of
 * Eq. LB_equation_ordinary (each step: rho = sum_i f_i, f^eq, BGK collision,
 * periodic shift of f_i by c_i).  Asynchronous on the handle's stream.
 * Errors: LB_KS_EINVAL (n < 0), LB_KS_ECUDA, or a sticky error.
 */
LB_KS_API int lb_ks_step(lb_ks_t *h, int64_t n);

/*
 * Write rho = sum_i f_i at every site (FP64; runs concatenated in run order,
 * sum N[r] values) to out (host or device, caller-owned).  Waits for the stream.
 */
LB_KS_API int lb_ks_rho(lb_ks_t *h, double *out);

/*
 * FP64 mass sum_x rho(x) and energy sum_x rho(x)^2 of every run
 * (arrays of nruns values, host memory).  Either pointer may be NULL.
 * Waits for the stream; returns LB_KS_EUNSTABLE if a mass is not finite.
 */
LB_KS_API int lb_ks_mass_energy(lb_ks_t *h, double *mass, double *energy);

/* Number of bytes lb_ks_save writes for this handle. */
LB_KS_API int lb_ks_state_bytes(const lb_ks_t *h, size_t *bytes);

/*
 * Checkpoint: copy the full state (populations in their storage precision,
 * the step counter and the guard's reference masses) to buf (host memory of
 * at least lb_ks_state_bytes bytes).  lb_ks_load restores it into a handle
 * created with the same runs, scheme and precision.  Resuming from a
 * checkpoint gives bitwise the same result as running straight through.
 * Layout: a 64-byte header; nruns int64 lattice sizes; nruns records of run
 * constants; nruns FP64 reference masses; last, the populations: scheme
 * planes of `plane` elements in the storage precision (8, 4 or 2 bytes)
 * (one plane, rho - rhobar, for LB_KS_KERNEL_COLLAPSE: header word 5 is then 1),
 * plane = sum over runs of N rounded up to a multiple of 32, run r starting
 * at the sum of the rounded sizes of the runs before it.  Populations are
 * stored as f_0 - rhobar, f_1, ..., f_{Q-1} (divided by the run's scale for
 * F16S), rhobar and scale being the run's initial mean and storage scale.
 * lb_ks_load returns LB_KS_EINVAL, leaving the handle as it was, when the
 * buffer is shorter than lb_ks_state_bytes, its header (scheme, precision,
 * runs, plane) or lattice sizes differ from the handle's, a run record places
 * its run elsewhere in the arenas than the handle does (or differs in its
 * ends), a run's constants are not finite, or a step counter is negative.
 * The steps since the last guard are taken modulo this handle's
 * recentre_every, which may differ from the saving handle's.  A successful
 * load clears a sticky device error.
 */
LB_KS_API int lb_ks_save(lb_ks_t *h, void *buf, size_t bytes);
LB_KS_API int lb_ks_load(lb_ks_t *h, const void *buf, size_t bytes);

/* Steps advanced since init (or since the loaded checkpoint's start). */
LB_KS_API int64_t lb_ks_steps_done(const lb_ks_t *h);

/*
 * Describe the handle: kernel family actually used (LB_KS_KERNEL_*), resident
 * sites per thread, threads per block, steps per launch and blocks per work group
 * of whole lattices (1 or 2; all 0 when not resident), number of runs and total
 * sites.  Any pointer may be NULL.
 */
LB_KS_API int lb_ks_describe(const lb_ks_t *h, int *kernel, int *sites_per_thread, int *threads_per_block,
                   int *steps_per_launch, int *cluster_size, int32_t *nruns, int64_t *total_sites);

/*
 * The register-resident plan of the handle (no counterpart in the paper): the work
 * lists ("lanes") that run concurrently, one record of LB_KS_LANE_FIELDS int32 per
 * lane written to lanes[8 * l .. 8 * l + 7] for l < max_lanes:
 *   [0] blocks per work group (1, or 2 for a thread block cluster pair)
 *   [1] work groups launched (persistent grid)
 *   [2] bundles (work items of packed lattices) in the lane's queue
 *   [3] steps per launch
 *   [4] 1 if the lane holds lattice segments (longer than a work group holds)
 *   [5] pair lanes: steps between the halo exchanges of lattices held as two halves
 *       (0: none are)
 *   [6] 1 if single-block bundles run two to a pair work group on this lane's queue
 *   [7] lattices held as two halves
 * Returns the number of lanes (0 when the handle does not run the resident kernels),
 * or LB_KS_EINVAL (h NULL, max_lanes < 0, lanes NULL with max_lanes > 0).
 */
#define LB_KS_LANE_FIELDS 8
LB_KS_API int lb_ks_describe_lanes(const lb_ks_t *h, int32_t *lanes, int max_lanes);

/* Kernel launches issued by this handle since creation (a counter kept on the host). */
LB_KS_API int64_t lb_ks_launches(const lb_ks_t *h);

/*
 * Diagnostic (no counterpart in the paper): measured throughput of the FP32
 * (fp64 = 0) or FP64 (fp64 = 1) fused multiply-add pipes of the current device
 * in flop/s, from a short kernel of independent FMA chains.  Used to put the
 * resident kernel's arithmetic rate next to the machine's.  Allocates and
 * frees a small device buffer.  Errors: LB_KS_EINVAL, LB_KS_ECUDA.
 */
LB_KS_API int lb_ks_fma_peak(int fp64, double *flops_per_s);

/*
 * FP64 mass sum_x rho(x) and energy sum_x rho(x)^2 of one lattice whose
 * populations the caller holds in device memory, computed without allocating
 * any memory.  No counterpart in the paper: it is the guard's reduction
 * (lb_ks_mass_energy) for callers that cannot call cudaMalloc -- for instance a
 * host application whose device memory is all owned by its own pool allocator,
 * or a monitoring hook that must still work when the device is out of memory.
 *   f: populations in the library's layout: plane i (i < scheme) starts at
 *      element i * plane of f, site x at element x of its plane; element type
 *      double, float or __half for precision LB_KS_F64, LB_KS_F32, LB_KS_F16S
 *      (the populations section of a checkpoint written by lb_ks_save, run 0,
 *      has this layout).
 *   rho(x) = rhobar + scale * sum_i f_i(x): rhobar = 0 for FP64, the run's storage
 *      offset (its initial mean) for F32 and F16S; scale is the run's storage scale
 *      for F16S and must be 1 for FP64 and F32 (other values: LB_KS_EINVAL).
 *   out: 2 doubles (mass, energy), host or device memory.
 * The partial sums live in one static device array of 256 KB (2 x 16384 + 2
 * doubles), present on every device that loads the library until exit; it
 * limits N to 2^24 sites (larger N: LB_KS_EINVAL).  The first call on a device
 * looks the array's address up (cudaGetSymbolAddress) and must be made with
 * that device current; make that first call before any stream capture on the
 * device.  The address is kept for the life of the process: do not call this
 * entry point on a device after cudaDeviceReset of that device.  All calls share the array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Runs on stream (cudaStream_t, NULL = legacy default) and waits for it.
 * Errors: LB_KS_EINVAL (bad scheme/precision, NULL pointers, N < 1,
 * N > 2^24, plane < N, scale <= 0, scale != 1 for FP64 or F32), LB_KS_ECUDA.
 */
LB_KS_API int lb_ks_mass_energy_noalloc(int scheme, int precision, const void *f, int64_t plane, int64_t N,
                                        double rhobar, double scale, double *out, void *stream);

/* Testing aid for the link between the two blocks of a cluster pair (no counterpart
 * in the paper).  A lattice held as one ring across both blocks of a pair sends, every
 * step, the values that cross the block edge into the other block's shared memory, and
 * the receiving threads wait for them with a bounded wait.  With withhold_step >= 0,
 * block 1 of every pair sends nothing across the edge at that step of each launch
 * (counted from the launch's first step), so that the receiving wait in block 0 runs
 * out; wait_rounds is the number of try_wait rounds before a wait gives up (0: the
 * default, 2^22).  A wait that runs out is reported by the next call that checks the
 * handle's status as LB_KS_ETIMEOUT, which then sticks; the launch itself completes.
 * Only bundles with such a ring are affected (the plan's halves and single blocks
 * never wait on the other block).  Call before the first lb_ks_step (LB_KS_EINVAL
 * afterwards: captured step sequences keep the values they were captured with).
 * Errors: LB_KS_EINVAL (NULL handle, withhold_step < -1, called after a step). */
LB_KS_API int lb_ks_set_link_test(lb_ks_t *h, int32_t withhold_step, uint32_t wait_rounds);

/* Release the handle and its device memory.  NULL is ignored. */
LB_KS_API void lb_ks_free(lb_ks_t *h);

/* One-line reason for the last failure on h (or on the last failed
 * constructor when h is NULL).  Never NULL; valid until the next call on h. */
LB_KS_API const char *lb_ks_last_error(const lb_ks_t *h);

#ifdef __cplusplus
}
#endif

#endif /* LB_KS_H */
