/*
 * pm.h -- C ABI of the GB300 particle forward-map library (libpm_gb300.so).
 *
 * The library evaluates the parameter-to-observation map G(u) of
 * Borggaard, Glatt-Holtz & Krometis (arXiv:1808.10580) directly with backward
 * stochastic particles instead of solving the PDE on a grid:
 *   - Problem 1 / Algorithm 1 (time-dependent advection-diffusion, Eq.
 *     pde_diffusion): G_j(u) = theta(t_j, x_j) = E theta0(X_{t_j}) with
 *     dX = -v_u(X) ds + sqrt(2 kappa) dW, X_0 = x_j (Theorem 3.1, Eq. adr);
 *   - Problem 2 / Algorithm 2 (Dirichlet problem, Eq. bvp): G_j(u) =
 *     E[g(X_tau)] - E int_0^tau f(X_s) ds, tau the first exit time from the
 *     domain (Theorem 3.2, Eq. bvp_solution);
 * both with Euler-Maruyama steps (Eq. euler) and Monte Carlo averages over M
 * particles per observation.  v_u is the divergence-free velocity of a
 * Fourier stream function (Eq. v_expand).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Field.  psi(x) = sum_h a_h cos(2 pi k_h.x) + b_h sin(2 pi k_h.x) over the
 *   half-plane lattice H_K = {(m,n): m > 0, |n| <= K} U {(0,n): 0 < n <= K},
 *   ordered by m, then n ascending; u = (a_0, b_0, a_1, b_1, ...) has 2|H_K| =
 *   (2K+1)^2 - 1 doubles.  v = (-d psi/dx2, d psi/dx1), i.e. the paper's
 *   k_perp = (-k_y, k_x) direction.  Supported K: 0..6, 8, 10, 12, 16; the
 *   time-dependent and Dirichlet maps with float paths also take the wide
 *   bounds K = 24, 32, 40, 48, 56, 64 (N_u = 2400 ... 16640), and the
 *   time-dependent map with float paths K = 80 (N_u = 25920, which holds the
 *   |k|_2 <= 80 basis; FP32 pipes only, PM_TENSOR then runs the FP32 pipes);
 *   PM_EINVAL elsewhere.
 * Random numbers.  Step n of path i of observation j in instance b draws
 *   Philox4x32-10 (Salmon et al., SC'11) on counter {n/2, i, j, b} under key
 *   {seed & 0xffffffff, seed >> 32}; words (r0, r1) feed even n and (r2, r3)
 *   odd n; u = (2 (r >> 9) + 1) / 2^24; Box-Muller gives xi = sqrt(-2 ln u_a)
 *   (cos 2 pi u_b, sin 2 pi u_b).  Results therefore depend only on the inputs
 *   and the seed, never on launch shapes or the GPU count.
 * Steps.  Time-dependent: N_j = ceil(t_j/dt - 1e-9) steps, all of length dt
 *   except the last, t_j - (N_j - 1) dt; positions wrap into [0,1)^2 after each
 *   step (the tensor-core kernels: after every 32nd step and after a path's
 *   last; their harmonics of x and x - 1 are the same, so only rounding
 *   differs).  Dirichlet: domain |x| < R; a path exits at the first step n with
 *   |X_n|^2 >= R^2; g is evaluated at R X_n/|X_n|; int f = f_const n dt; a path
 *   that has not exited after max_steps contributes 0 and is counted as
 *   unexited.
 * Estimator.  mean_j = (1/M) sum_i g_i, var_j = unbiased sample variance
 *   (n - 1); both are accumulated in double precision in a fixed order, so
 *   repeated calls return identical bits.
 * Precision.  Default (PM_FP32): particle arithmetic in float, positions kept
 *   as compensated float pairs; reductions in double.  PM_FP64: particle
 *   arithmetic in double (the plain FP64 path).
 * Memory.  Pointers are host pointers unless PM_DEVICE_PTRS is set, in which
 *   case the per-observation arrays (x, t, mean, var, and the optional
 *   per-path outputs) are device pointers on the context's device.  The field
 *   coefficients u of pm_forward_timedep / pm_forward_dirichlet and the small
 *   description tables (theta0, boundary data) are always host pointers; they
 *   are packed into the kernel's launch parameters.  The caller owns all
 *   arrays; the library owns its context, its device workspace and its pinned
 *   staging buffers.
 * Synchronisation.  Calls return after their outputs are written unless
 *   PM_ASYNC is set together with PM_DEVICE_PTRS; then the work is queued on
 *   the context's stream and the outputs are valid once that stream has been
 *   synchronised.  (With host pointers the call always synchronises.)
 * Errors.  0 = success; negative = error (nothing useful written; message from
 *   pm_last_error()); positive = warning (outputs written).  No call aborts
 *   the process.  A context is used by one host thread at a time.
 */
#ifndef PM_H
#define PM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_OK 0
#define PM_EINVAL (-1)      /* bad argument: sizes, dt <= 0, unsupported K, NaN */
#define PM_ENOMEM (-2)      /* device or pinned host allocation failed */
#define PM_ECUDA (-3)       /* CUDA runtime error; message holds its string */
#define PM_ETIMEOUT (-4)    /* a bounded wait expired */
#define PM_WARN_UNEXITED 1  /* Dirichlet: some paths hit max_steps */

#define PM_FP32 0u
#define PM_FP64 1u
#define PM_DEVICE_PTRS 2u
#define PM_ASYNC 4u
/* Float paths: evaluate the velocity sum on the tensor cores (tcgen05 with a
 * three-term hi/lo split of TF32 operands for K <= 8 and of FP16 operands,
 * with W scaled by a power of two, from K = 10: about float accuracy, results
 * differ from the FP32-pipe kernels by rounding); supported for K in
 * {4, 5, 6, 8, 10, 12, 16} (and the wide K for the time-dependent and Dirichlet maps),
 * other K run on the FP32 pipes. */
#define PM_TENSOR 8u
/* pm_forward_timedep: observations at bit-identical points x
 * share their paths (Theorem 3.1: the value at t_j needs the path only up to
 * time t_j, so one path serves every t_j at the same x).  Such a group
 * draws its noise from the RNG stream of its
 * lowest observation index j0 (counter word j = j0 for every member); one path
 * i runs to the largest step count of the group and every member j records
 * theta0 where its own path ends (after N_j - 1 full steps and its last step
 * of length t_j - (N_j - 1) dt, with the noise of that step).  Each member's
 * estimate has the law it has without the flag, members of a group are
 * correlated, and a group costs max N_j steps per path instead of sum N_j.
 * With PM_DEVICE_PTRS the call copies x and t to the host to form the groups. */
#define PM_SHARE_PATHS 16u

#define PM_MAX_THETA0_MODES 64
#define PM_MAX_BOUNDARY_MODES 32

typedef struct pm_ctx pm_ctx;

/* Library version, 10000*major + 100*minor + patch. */
int pm_version(void);

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to queue all work on (NULL: the context creates and owns a stream; pass
 * cudaStreamLegacy to use the legacy default stream).
 * Returns PM_OK and stores the context in *out, or an error. */
int pm_create(pm_ctx** out, int device, void* cuda_stream);

/* Synchronises the context's stream and frees everything the context owns.
 * NULL is ignored. */
void pm_destroy(pm_ctx* ctx);

/* Message of the last failing call made by this host thread ("" if none). */
const char* pm_last_error(void);

/* The context's stream (a cudaStream_t). */
void* pm_stream(const pm_ctx* ctx);

/* Stream-function coefficients.  u: host pointer, 2|H_K| doubles. */
typedef struct pm_field {
    int32_t K;
    int32_t reserved;
    const double* u;
} pm_field;

/* theta0(x) = sum_q a_q cos(2 pi k_q.x) + b_q sin(2 pi k_q.x); k: [n][2] int32.
 * n <= PM_MAX_THETA0_MODES.  Host pointers. */
typedef struct pm_fourier {
    int32_t n;
    int32_t reserved;
    const int32_t* k;
    const double* a;
    const double* b;
} pm_fourier;

/* Disk of radius R centred at 0.  Boundary data at y = R (cos phi, sin phi):
 * g(y) = quad (y1^2 - y2^2) + sum_{m=1..n_ang} a[m-1] cos(m phi) + b[m-1] sin(m phi).
 * Forcing f = f_const.  n_ang <= PM_MAX_BOUNDARY_MODES.  Host pointers. */
typedef struct pm_dirichlet_data {
    double R;
    double quad;
    double f_const;
    int32_t n_ang;
    int32_t reserved;
    const double* a;
    const double* b;
} pm_dirichlet_data;

/* Optional per-call settings (NULL = all defaults). */
typedef struct pm_path_opts {
    int64_t path_offset; /* index i of the first path (shards of one estimate); default 0 */
    uint32_t instance;   /* b of the RNG counter; default 0 */
    int32_t reserved;
    double* g_out;       /* [n_obs][M] per-path values g_i, or NULL */
    double* x_out;       /* [n_obs][M][2] end (or exit) positions, or NULL */
} pm_path_opts;

/* Algorithm 1 (Section 3.1): time-dependent map G_j(u) = theta(t_j, x_j).
 *   field   stream-function coefficients (host)
 *   kappa   diffusion coefficient, >= 0 (sigma = sqrt(2 kappa) I, Eq. adr)
 *   theta0  initial condition (host)
 *   x       [n_obs][2] observation points; t [n_obs] observation times >= 0
 *   M       particles per observation, 1 <= M, path_offset + M <= 2^32
 *   dt      Euler-Maruyama step > 0
 *   seed    64-bit Philox key
 *   flags   PM_FP32 | PM_FP64, PM_DEVICE_PTRS, PM_ASYNC, PM_TENSOR, PM_SHARE_PATHS
 *   mean    [n_obs] output; var [n_obs] output or NULL
 * n_obs == 0 is a no-op.  Returns PM_OK or an error. */
int pm_forward_timedep(pm_ctx* ctx, const pm_field* field, double kappa, const pm_fourier* theta0,
                       const double* x, const double* t, int64_t n_obs, int64_t M, double dt,
                       uint64_t seed, uint32_t flags, double* mean, double* var,
                       const pm_path_opts* opts);

/* ------------------------------------------------------------------------- *
 * The optimal-forcing boundary-value problem of Section 4 (Eq. bvp:ex1) by
 * Algorithm 2 and Theorem 3.2: in the unit square (0,1)^2,
 *   -b . grad theta + kappa Laplace theta = sum_q F_q phi_q,
 *   phi_q(x) = exp(-w |x - c_q|^2),      theta = g on the boundary,
 *   g(y) = g_cos (cos(pi y1 / 2) + cos(pi y2 / 2)) / 2 + g_quad (y1^2 - y2^2)
 * (the paper's data: g_cos = 1, g_quad = 0).  Theorem 3.2 with dX = -b ds +
 * sqrt(2 kappa) dW gives theta(x; F) = E[g(X_tau)] - sum_q F_q E[int_0^tau
 * phi_q(X_s) ds], affine in F: one set of paths yields, per observation, the
 * n_src + 1 functionals from which theta(x; F) follows for every F.
 * Paths: Euler-Maruyama steps of length dt, noise as for pm_forward_dirichlet
 * (counter {n/2, i, j, instance}); the integrals by the left-point rule
 * sum_{m < n} phi_q(X_m) dt; exit at the first step outside the open square,
 * X_tau = that position clamped to the square; a path that reaches max_steps
 * contributes zeros and is counted in *n_unexited.
 * ------------------------------------------------------------------------- */
#define PM_MAX_SOURCES 8

typedef struct pm_square_bvp {
    double b[2];        /* constant drift (the paper: (1, 1)) */
    double kappa;       /* >= 0 */
    double w;           /* source width parameter (the paper: 4), >= 0 */
    double g_cos, g_quad;
    int32_t n_src;      /* 0 .. PM_MAX_SOURCES */
    int32_t reserved;
    const double* c;    /* [n_src][2] source centres (host) */
} pm_square_bvp;

/* mean, var: [n_obs][n_src + 1] (var may be NULL): for observation j, entry 0
 * is E[g(X_tau)] and entry q + 1 is E[int phi_q]; opts->g_out, if set,
 * receives the per-path values [n_obs][n_src + 1][M]; opts->x_out is not
 * used.  x: [n_obs][2].  Pointers follow PM_DEVICE_PTRS; PM_FP64 selects
 * double paths.  Returns PM_OK, PM_WARN_UNEXITED or an error. */
int pm_forward_square_bvp(pm_ctx* ctx, const pm_square_bvp* prob, const double* x, int64_t n_obs, int64_t M,
                          double dt, int64_t max_steps, uint64_t seed, uint32_t flags, double* mean, double* var,
                          int32_t* exit_step, int64_t* n_unexited, const pm_path_opts* opts);

/* The groups PM_SHARE_PATHS forms, computed on the host (no device, no
 * context): x [n_obs][2], t [n_obs] host arrays as for pm_forward_timedep.
 *   group_of[j]   group of observation j, numbered in launch order (groups
 *                 sorted by their largest step count, longest first, then by
 *                 stream); may be NULL
 *   stream_of[j]  RNG observation index its paths use (lowest index of its
 *                 group); may be NULL
 *   n_groups      number of groups; may be NULL
 *   steps_per_path  Euler steps one path index takes over all groups (sum of
 *                 the groups' largest N_j); may be NULL
 * Returns PM_OK, or PM_EINVAL for NULL x / t, n_obs < 0, dt <= 0, or a time
 * that is negative, not finite or needs more than 2^31 - 2 steps. */
int pm_path_groups(const double* x, const double* t, int64_t n_obs, double dt, int32_t* group_of,
                   int32_t* stream_of, int64_t* n_groups, int64_t* steps_per_path);

/* Algorithm 2 (Section 3.2): Dirichlet map G_j(u) = theta(x_j) in the disk.
 *   drift_scale  multiplies v_u (the drift is -drift_scale v_u)
 *   g            domain, boundary data and forcing (host)
 *   max_steps    cap on the steps of one path (>= 1)
 *   exit_step    [n_obs][M] steps taken to exit (-1 = capped), or NULL
 *   n_unexited   total capped paths, or NULL (host or device per flags)
 * Paths of uneven length are load-balanced by a persistent kernel in which
 * every lane takes a new path as soon as its current one exits; observations
 * are claimed in order of their driftless mean exit time, longest first (with
 * PM_DEVICE_PTRS the call reads x back to the host for that, a stream
 * synchronisation).  Results do not depend on the order.
 * Returns PM_OK, PM_WARN_UNEXITED (outputs written), or an error. */
int pm_forward_dirichlet(pm_ctx* ctx, const pm_field* field, double drift_scale, double kappa,
                         const pm_dirichlet_data* g, const double* x, int64_t n_obs, int64_t M,
                         double dt, int64_t max_steps, uint64_t seed, uint32_t flags,
                         double* mean, double* var, int32_t* exit_step, int64_t* n_unexited,
                         const pm_path_opts* opts);

/* Algorithm 2 in the disk with a general forcing and a state-dependent
 * diffusion (Theorem 3.2 with f(x) and sigma(x); Eq. euler or Eq. millstein):
 *   dX = -drift_scale v_u(X) ds + sigma(X) dW,
 *   sigma(x) = diag(s0[0] + s1[0] x_1, s0[1] + s1[1] x_2),
 * each coordinate driven by its own Brownian motion with a diffusion
 * coefficient of its own coordinate, so the Milstein correction is the scalar
 * one of Eq. millstein per coordinate:
 *   X_i <- X_i - drift_scale v_i dt + sigma_i(X) sqrt(dt) xi_i
 *               + (1/2) sigma_i(X) s1[i] (xi_i^2 - 1) dt      (milstein = 1),
 * without the last term for milstein = 0 (Euler-Maruyama); xi as for the
 * other maps.  The forcing is f(x) = g->f_const + sum_q F[q] exp(-w |x - c_q|^2),
 * integrated by the left-point rule dt sum_{m < n} f(X_m); the constant-
 * coefficient map is the case s0 = sqrt(2 kappa), s1 = 0, n_src = 0 (results
 * equal up to rounding).  Other arguments, outputs and return values as for
 * pm_forward_dirichlet: float or double paths on the FP32 / FP64 pipes (K up to
 * 16), or with PM_TENSOR (float paths, K in {4, 5, 6, 8, 10, 12, 16} and the
 * wide bounds 24 ... 64) the velocity sum on the tensor cores as in
 * pm_forward_dirichlet, the diffusion, Milstein and forcing terms unchanged. */
typedef struct pm_diffusion_forcing {
    double s0[2], s1[2];  /* sigma_i(x) = s0[i] + s1[i] x_i */
    int32_t milstein;     /* 1: Eq. millstein, 0: Eq. euler */
    int32_t n_src;        /* Gaussian sources, 0 .. PM_MAX_SOURCES */
    double w;             /* width parameter of the sources, >= 0 */
    const double* c;      /* [n_src][2] centres (host) */
    const double* F;      /* [n_src] amplitudes (host) */
} pm_diffusion_forcing;

int pm_forward_dirichlet_general(pm_ctx* ctx, const pm_field* field, double drift_scale, const pm_dirichlet_data* g,
                                 const pm_diffusion_forcing* df, const double* x, int64_t n_obs, int64_t M, double dt,
                                 int64_t max_steps, uint64_t seed, uint32_t flags, double* mean, double* var,
                                 int32_t* exit_step, int64_t* n_unexited, const pm_path_opts* opts);

/* ---------------------------------------------------------------------------
 * Batched map: many parameter samples in one persistent launch.
 *
 * B instances, each a time-dependent (Algorithm 1) or a Dirichlet
 * (Algorithm 2) problem with its own coefficients u_b, observation rows,
 * particle count, step and seed; all share the wave-number bound K, theta0
 * (time-dependent instances) and the disk data (Dirichlet instances).  The
 * observations of instance b are rows [row0, row0 + n_obs) of the batch's x
 * (and t); the rows of all instances must tile [0, n_rows) without overlap.
 * The RNG counter of an instance uses its `stream` as the instance word and
 * the row's offset j within the instance, so an instance gives the same
 * estimate as pm_forward_timedep / pm_forward_dirichlet with opts->instance =
 * stream and the same seed.  Giving several instances the same stream and
 * seed makes them share their Brownian increments (common random numbers:
 * the estimate is then a deterministic function of u alone).
 * Section 3.3 makes every path independent: one persistent kernel runs all
 * paths of all instances; each lane takes a new path of its warp's instance
 * as soon as its path ends, and warps move between instances as these run
 * out of paths, so uneven path lengths stay load-balanced.
 * The call sequence (coefficient staging, row preparation, persistent kernel,
 * reduction, copies) is captured once into a CUDA graph per call shape and
 * replayed on later calls with the same shape; a context created on the
 * legacy default stream launches directly instead (that stream cannot be
 * captured).  Float paths, double reductions; PM_FP64 is not supported here.
 * ------------------------------------------------------------------------- */
#define PM_KIND_TIMEDEP 0
#define PM_KIND_DIRICHLET 1

typedef struct pm_instance {
    int32_t kind;          /* PM_KIND_TIMEDEP or PM_KIND_DIRICHLET */
    uint32_t stream;       /* RNG instance word b of the counter {n/2, i, j, b} */
    const double* u;       /* 2|H_K| coefficients; host, or device with PM_DEVICE_PTRS */
    double kappa;          /* >= 0 */
    double dt;             /* > 0 */
    double drift_scale;    /* Dirichlet: drift is -drift_scale v_u (time-dependent: ignored, 1) */
    int64_t max_steps;     /* Dirichlet: cap on the steps of a path, >= 1 */
    int64_t row0;          /* first observation row */
    int64_t n_obs;         /* >= 1 rows */
    int64_t M;             /* >= 1 particles per observation */
    uint64_t seed;
} pm_instance;

typedef struct pm_batch {
    int32_t K;
    int32_t B;                       /* >= 1 instances */
    const pm_instance* inst;         /* host array [B] */
    const pm_fourier* theta0;        /* host; required if any instance is time-dependent */
    const pm_dirichlet_data* disk;   /* host; required if any instance is Dirichlet */
    const double* x;                 /* [n_rows][2] */
    const double* t;                 /* [n_rows]; read for time-dependent rows only */
    int64_t n_rows;
} pm_batch;

/* mean, var: [n_rows] (var may be NULL); n_unexited: total capped Dirichlet
 * paths (or NULL).  x, t, mean, var, n_unexited and the u pointers are device
 * pointers with PM_DEVICE_PTRS, else host pointers.  Returns PM_OK,
 * PM_WARN_UNEXITED, or an error. */
int pm_forward_batched(pm_ctx* ctx, const pm_batch* batch, uint32_t flags, double* mean, double* var,
                       int64_t* n_unexited);

/* Graph capture and replay of pm_forward_batched: on (1, default) or off (0). */
int pm_set_graph_mode(pm_ctx* ctx, int on);

/* ------------------------------------------------------------------------- *
 * Autotuner of the persistent launches (the batching pattern's block and
 * chunk shapes).  The Dirichlet and batched kernels run a persistent grid of
 * (CTAs per SM) x SMs whose lanes claim paths from counters; every path's
 * value is stored and reduced in path order, so results do not depend on
 * the grid and its one free shape is the number of CTAs per SM.
 *
 * pm_autotune_dirichlet / pm_autotune_batched time two forward calls (the
 * second measured) with the caller's problem and flags for every candidate
 * from 1 to the kernel's occupancy limit, keep the fastest in the context
 * for (kernel, K, PM_FP64 and PM_TENSOR bits) and store it in
 * *best_ctas_per_sm (may be NULL); for the tensor-core kernels they then
 * time the refill interval at that grid (pm_set_refill_pairs).  Arguments are those of the forward call
 * (PM_ASYNC is ignored; outputs go to scratch the call allocates and frees).
 * When the environment variable PM_AUTOTUNE_CACHE names a file, pm_create
 * reads this device's choices from it (a flat JSON object
 * {"<device name>|<kind>|<K>|<flags>": ctas_per_sm}) and the autotuners write
 * theirs back.  PM_AUTOTUNE=0 makes every launch use the occupancy limit.
 * Returns PM_OK or the error of the failing forward call.
 * ------------------------------------------------------------------------- */
#define PM_TUNE_DIRICHLET 0
#define PM_TUNE_BATCHED 1

int pm_autotune_dirichlet(pm_ctx* ctx, const pm_field* field, double drift_scale, double kappa,
                          const pm_dirichlet_data* g, const double* x, int64_t n_obs, int64_t M, double dt,
                          int64_t max_steps, uint64_t seed, uint32_t flags, int32_t* best_ctas_per_sm);
int pm_autotune_batched(pm_ctx* ctx, const pm_batch* batch, uint32_t flags, int32_t* best_ctas_per_sm);

/* Sets the CTAs per SM used for (kind, K, flags & (PM_FP64 | PM_TENSOR));
 * values above the occupancy limit are clamped to it, <= 0 removes the
 * setting.  kind: PM_TUNE_DIRICHLET or PM_TUNE_BATCHED. */
int pm_set_ctas_per_sm(pm_ctx* ctx, int32_t kind, int32_t K, uint32_t flags, int32_t ctas_per_sm);

/* The second free shape of the tensor-core forms of the persistent kernels
 * (flags containing PM_TENSOR): the pairs of Euler steps between two refills
 * of the lanes whose paths have ended (default for the disk maps: 16 when the
 * observations' mean driftless exit time (R^2 - |x|^2) / (4 kappa dt) is at
 * least 16384 steps, 8 from 4096, else 4, with kappa = (sigma_1(0)^2 +
 * sigma_2(0)^2) / 4 for the general map; for the batched map 8; every path's
 * random numbers are keyed by its own step index, so results do not depend
 * on it).  The
 * autotuners choose it after the CTAs per SM (coordinate descent over 1, 2,
 * 4, 8, 16); this sets it by hand (<= 0 removes the setting, at most 64). */
int pm_set_refill_pairs(pm_ctx* ctx, int32_t kind, int32_t K, uint32_t flags, int32_t pairs);

/* The shape in use for (kind, K, flags): CTAs per SM and refill pairs, 0 where
 * none was tuned or set (the launch then uses the occupancy limit and the
 * default interval).  Either output may be NULL. */
int pm_tuned_shape(pm_ctx* ctx, int32_t kind, int32_t K, uint32_t flags, int32_t* ctas_per_sm, int32_t* refill_pairs);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the forward map (the paper has no learned component;
 * this serves the delayed-acceptance pre-screen of pCN MCMC proposals).
 *
 * A 3-layer ReLU network u -> relu(W1 u + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3
 * with weights [out][in], trained on (u, G(u)) pairs by Adam on an FP32 master
 * copy; every matrix product runs on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation in tensor memory).  Loss: sum (y - target)^2 / (2 B n_out).
 * n_hidden must be a multiple of 128.  The network object lives on the
 * context's device; use it with one context at a time.
 * ------------------------------------------------------------------------- */
typedef struct pm_mlp pm_mlp;

typedef struct pm_train_opts {
    int32_t epochs;         /* passes over the data, >= 1 */
    int32_t batch;          /* rows per Adam step, >= 1 */
    float lr;               /* Adam step size */
    float beta1, beta2;     /* moment decays in [0, 1) */
    float eps;              /* > 0 */
    float weight_decay;     /* decoupled weight decay of the weight matrices (AdamW), >= 0 */
    float lr_decay;         /* the step size is multiplied by this after every epoch, in (0, 1] */
    uint64_t shuffle_seed;  /* seed of the per-epoch row shuffle */
} pm_train_opts;

/* Creates a network with seeded He-normal weights and zero biases. */
int pm_surrogate_create(pm_ctx* ctx, pm_mlp** out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed);
void pm_surrogate_destroy(pm_mlp* net);

/* Host FP32 parameters, row-major [out][in]: W1 [n_hidden][n_in], b1 [n_hidden],
 * W2 [n_hidden][n_hidden], b2, W3 [n_out][n_hidden], b3 [n_out].  Setting
 * them resets the Adam state. */
int pm_surrogate_set_params(pm_ctx* ctx, pm_mlp* net, const float* W1, const float* b1, const float* W2,
                            const float* b2, const float* W3, const float* b3);
int pm_surrogate_get_params(pm_ctx* ctx, const pm_mlp* net, float* W1, float* b1, float* W2, float* b2,
                            float* W3, float* b3);

/* One forward and backward pass on host arrays U [B][n_in], T [B][n_out]
 * without an update: the loss and the gradients (host, same layouts as the
 * parameters; any output may be NULL). */
int pm_surrogate_gradients(pm_ctx* ctx, pm_mlp* net, const float* U, const float* T, int64_t B, float* loss,
                           float* gW1, float* gb1, float* gW2, float* gb2, float* gW3, float* gb3);

/* Adam training on U [N][n_in], Y [N][n_out] (device pointers with
 * PM_DEVICE_PTRS); loss_history [epochs] receives each epoch's mean batch loss
 * (or NULL). */
int pm_surrogate_train(pm_ctx* ctx, pm_mlp* net, const float* U, const float* Y, int64_t N,
                       const pm_train_opts* opts, uint32_t flags, float* loss_history);

/* Y [B][n_out] = net(U [B][n_in]); pointers follow PM_DEVICE_PTRS. */
int pm_surrogate_infer(pm_ctx* ctx, const pm_mlp* net, const float* U, int64_t B, float* Y, uint32_t flags);

/* The gradient of the network with respect to its input, row by row: for
 * each row b, dU[b] = J(U[b])^T dY[b] with J the Jacobian dY/dU of the
 * network at U[b] (a vector-Jacobian product: the ReLU masks of the forward
 * pass at U[b], then the three weight matrices transposed, on the tensor
 * cores with BF16 operands and FP32 accumulation).  U [B][n_in], dY
 * [B][n_out], dU [B][n_in]; pointers follow PM_DEVICE_PTRS.  This makes the
 * surrogate differentiable in the parameter u, which the particle map is not
 * (the paper notes that its estimator has no Frechet derivative): gradient-
 * based MAP estimation runs on the surrogate. */
int pm_surrogate_input_gradient(pm_ctx* ctx, const pm_mlp* net, const float* U, const float* dY, int64_t B, float* dU,
                                uint32_t flags);

/* Parameters and Adam state to / from a binary file. */
int pm_surrogate_save(pm_ctx* ctx, const pm_mlp* net, const char* path);
int pm_surrogate_load(pm_ctx* ctx, pm_mlp** out, const char* path);

/* Diagnostic: C[M][ldc] (FP32) = A[M][K] . B[N][K]^T for BF16 A (row pitch
 * lda) and B (row pitch ldb), all device pointers, on the tensor-core GEMM
 * the surrogate uses.  M % 128 == 0, N % 64 == 0, K % 64 == 0. */
int pm_gemm_bf16(pm_ctx* ctx, const void* A, int32_t lda, const void* B, int32_t ldb, int32_t M, int32_t N,
                 int32_t K, float* C, int32_t ldc);

/* ---------------------------------------------------------------------------
 * pCN MCMC over the time-dependent map (Section 4.1: the paper samples its
 * posteriors with preconditioned Crank-Nicolson), plain or with delayed
 * acceptance (Christen & Fox 2005) through a surrogate network.
 *
 * Prior N(0, C) on the field coefficients with C = diag(|k_h|^-4); proposal
 * u' = sqrt(1 - beta^2) u + beta C^{1/2} xi; Phi(u) = sum_j (y_j - G_j(u))^2 /
 * (2 sigma^2).  Plain: accept with min(1, exp(Phi(u) - Phi(u'))).  Delayed
 * acceptance: stage 1 with the surrogate's Phi~, stage 2 only for the stage-1
 * survivors, accepting with min(1, exp(Phi(u) - Phi(u') - Phi~(u) + Phi~(u'))).
 * G is the particle map of Algorithm 1 evaluated for all needed proposals in
 * one batched launch with a single RNG stream and seed (so G is a
 * deterministic function of u), or, for testing, a linear map A u.
 * Randomness: proposal normals of chain c at step s from Philox counters
 * {s, c, q, 0x4D43} (normals 4q..4q+3 from two Box-Muller pairs), stage-1 and
 * stage-2 uniforms from {s, c, 0xFFFFFFFF, 1 or 2} (word 0), key = seed.
 * Chain states, misfits and the running sum of states live on the device.
 * ------------------------------------------------------------------------- */
typedef struct pm_pcn pm_pcn;

typedef struct pm_pcn_config {
    int32_t n_chains;
    int32_t K;                  /* field bound: n_u = (2K+1)^2 - 1 coefficients */
    double beta;                /* pCN step in (0, 1] */
    double sigma;               /* observation noise standard deviation */
    uint64_t seed;              /* proposals and acceptance tests */
    int64_t n_obs;
    const double* y;            /* [n_obs] data (host) */
    const double* A;            /* [n_obs][n_u] host: G(u) = A u (testing); NULL: particle map below */
    double kappa, dt;           /* particle map: Algorithm 1 */
    int64_t M;
    uint64_t path_seed;
    const pm_fourier* theta0;   /* host */
    const double* x;            /* [n_obs][2] host */
    const double* t;            /* [n_obs] host */
    uint32_t map_flags;         /* particle map: 0 (FP32 pipes) or PM_TENSOR; other bits rejected */
    uint32_t reserved;
    const double* screen_shift; /* [n_u] host or NULL (= 0): the surrogate input is (u - shift) * scale */
} pm_pcn_config;

typedef struct pm_pcn_stats {
    int64_t steps;              /* pCN steps of every chain */
    int64_t proposals;          /* steps x chains */
    int64_t stage1_accepts;     /* proposals that passed the surrogate screen */
    int64_t accepts;            /* accepted moves */
    int64_t forward_evals;      /* particle-map evaluations (instances) */
    double seconds;             /* device time of the run */
    double sq_jump;             /* sum over accepted moves of |(u' - u) / prior std|^2 (an efficiency measure) */
} pm_pcn_stats;

/* u0: [n_chains][n_u] host.  screen: NULL for plain pCN, else a surrogate
 * with n_in = n_u and n_out = n_obs whose input is (u - cfg->screen_shift) *
 * screen_scale (screen_scale [n_u] host, NULL = 1). */
int pm_pcn_create(pm_ctx* ctx, pm_pcn** out, const pm_pcn_config* cfg, const double* u0, const pm_mlp* screen,
                  const float* screen_scale);
int pm_pcn_run(pm_ctx* ctx, pm_pcn* chains, int64_t n_steps, pm_pcn_stats* stats);
/* Current states u [n_chains][n_u], misfits phi [n_chains], and the sum of all
 * states visited so far sum_u [n_u] over n_summed = steps x chains (any may be NULL). */
int pm_pcn_state(pm_ctx* ctx, const pm_pcn* chains, double* u, double* phi, double* sum_u, int64_t* n_summed);
void pm_pcn_destroy(pm_pcn* chains);

/* ---------------------------------------------------------------------------
 * Allocation-free variant (the paper has no counterpart; this is a library
 * convenience).
 *
 * For callers that cannot allocate device memory -- code that runs while
 * another allocator owns the device's memory, latency-critical loops where
 * cudaMalloc's implicit synchronisation is not acceptable, hosts that forbid
 * allocation after start-up.  Same arguments, kernels and results as
 * pm_forward_timedep with device pointers (x, t, mean, var on the current
 * device), but no context: work is queued on `cuda_stream` (NULL = legacy
 * default stream) on the current device, and the scratch comes from one
 * fixed device array of PM_NOALLOC_SCRATCH_BYTES that the library declares
 * and that every GPU which loads the library holds until the process exits.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress)
 *     in the current device's context, so a call after cudaDeviceReset finds
 *     the array where the new context loaded it.  Under CUDA's lazy module
 *     loading the first call on a device also loads the library's kernels
 *     (the driver may allocate for that, once): make one call on each device
 *     before the code that must not allocate, and before any stream capture.
 *   - Problems whose scratch (about n_obs * (48 + 16 * ceil(M/128)) bytes)
 *     exceeds PM_NOALLOC_SCRATCH_BYTES are rejected with PM_EINVAL.
 *   - x, t, mean and var must be device memory of the current device (or
 *     managed memory); anything else is rejected with PM_EINVAL before any
 *     work is queued.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and give wrong results;
 *     serialise them.
 *   - flags: PM_FP32 or PM_FP64, plus PM_ASYNC to return without waiting.
 *     With PM_ASYNC the call cannot report invalid observation inputs (NaN
 *     or negative times, non-finite points): they are detected on the GPU,
 *     and the flag that records them is only read by a synchronous call.
 * ------------------------------------------------------------------------- */
#define PM_NOALLOC_SCRATCH_BYTES (4u << 20)

int pm_forward_timedep_noalloc(const pm_field* field, double kappa, const pm_fourier* theta0,
                               const double* x, const double* t, int64_t n_obs, int64_t M, double dt,
                               uint64_t seed, uint32_t flags, double* mean, double* var,
                               void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Diagnostics: the building blocks of the particle step, exposed so that each
 * can be checked on its own against an independent implementation.
 * ------------------------------------------------------------------------- */

/* Philox4x32-10 of n counters ctr[n][4] under key {key0, key1} -> out[n][4].
 * Pointers follow PM_DEVICE_PTRS. */
int pm_philox(pm_ctx* ctx, const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n,
              uint32_t* out, uint32_t flags);

/* The normals (xi1, xi2) of steps n0 .. n0+count-1 of path (b, j, i) as the
 * kernels draw them, in the precision the flags select -> out[count][2]
 * (double): PM_FP64, PM_FP32 (the FP32-pipe kernels: sincospif for the
 * angle), or PM_FP32 | PM_TENSOR (the tensor-core kernels: the two steps of a
 * Philox block in one packed pass with the library's own sin and cos of 2 pi u,
 * see pm_sincos_turns).  Pointers follow PM_DEVICE_PTRS. */
int pm_normals(pm_ctx* ctx, uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0,
               int64_t count, double* out, uint32_t flags);

/* sin(2 pi x) and cos(2 pi x) of n float points x (device pointers), as the
 * tensor-core kernels form them for their harmonic recurrences: a quarter-turn
 * reduction and the Taylor series of sin and cos in turns (the library's own,
 * not the CUDA math library's).  Outputs s[n], c[n] (device). */
int pm_sincos_turns(pm_ctx* ctx, const float* x, int64_t n, float* s, float* c);

/* Velocity v_u at npts points x[npts][2] -> v[npts][2], evaluated by the same
 * device code as the particle step (product basis, trigonometric
 * recurrences) in the precision the flags select. */
int pm_velocity(pm_ctx* ctx, const pm_field* field, const double* x, int64_t npts, double* v,
                uint32_t flags);

/* ---------------------------------------------------------------------------
 * Measurement support.
 * ------------------------------------------------------------------------- */

/* When on, the context brackets the main particle kernel of each forward call
 * with CUDA events on its stream; pm_last_kernel_ms() then returns that
 * kernel's duration (synchronising on the end event). */
int pm_set_kernel_timing(pm_ctx* ctx, int on);
float pm_last_kernel_ms(pm_ctx* ctx);

/* Test setting for the failure path of the tensor-core kernels.  Their waits
 * for the tensor core (the per-step product of the PM_TENSOR particle kernels,
 * the pipeline stages of the GEMM) are bounded; a wait that runs out sets an
 * error flag, the kernel waits (with the full bound) for its own copies and
 * products still in flight, frees its tensor memory and returns, and the call
 * returns PM_ETIMEOUT.  pm_set_wait_limit makes the next call of
 * pm_forward_timedep, pm_forward_dirichlet or pm_gemm_bf16 on this context
 * give those waits at most `polls` polls (0: they give up without polling,
 * so the failure path runs deterministically); the setting then returns to
 * the full bound.  polls < 0 restores the full bound at once.  Calls that
 * give up return no valid results. */
int pm_set_wait_limit(pm_ctx* ctx, int64_t polls);

/* Number of kernels the context has launched since it was created. */
int64_t pm_launch_count(const pm_ctx* ctx);

/* Euler steps taken by all paths of the last forward call on this context
 * that synchronised (-1 after a PM_ASYNC call).  Dirichlet paths have
 * data-dependent lengths; this is the count throughput figures use. */
int64_t pm_last_step_count(const pm_ctx* ctx);

/* CTAs of the main particle kernel of the last forward call on this context
 * (persistent kernels: resident CTAs per SM x SMs, capped by the work), 0
 * before the first call. */
int64_t pm_last_grid(const pm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
