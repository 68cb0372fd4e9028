/*
 * pm_oracle.c -- plain, slow FP64 CPU oracle for the particle forward maps of
 * Borggaard, Glatt-Holtz & Krometis, "GPU-Accelerated Particle Methods for
 * Evaluation of Sparse Observations for PDE-Constrained Inverse Problems".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or table with the CUDA path (paper_1808_10580_gb300/csrc); the two
 * implement the same published definitions independently.
 *
 * What it computes, step by step, in the order the paper states it:
 *   - Brownian increments xi ~ N(0,1) (Eq. euler) from Philox4x32-10
 *     (Salmon, Moraes, Dror & Shaw, SC'11) and the Box-Muller transform;
 *   - the divergence-free velocity of a Fourier stream function, summed
 *     directly with sin/cos per mode (Eq. v_expand; Section 4.1);
 *   - Euler-Maruyama paths of dX = -v dt + sqrt(2 kappa) dW (Theorem 3.1,
 *     Eq. euler, sigma = sqrt(2 kappa) I as in Eq. adr);
 *   - Algorithm 1 (time-dependent problem): g = theta0(X_{t_j});
 *   - Algorithm 2 (Dirichlet problem): walk to first exit, g = g_bc(X_tau)
 *     minus the time integral of f (Theorem 3.2, Eq. bvp_solution).
 * Per-path values are returned; the estimator mean/variance are formed by the
 * caller with plain numpy (mean, unbiased variance).
 *
 * Readings of points where the paper is silent (the same on both sides):
 *   stream-function parameterisation and half-mode order; RNG counter layout
 *   and 23-bit uniforms; step count and last step; periodic wrap; exit test
 *   |X|^2 >= R^2 with radial projection; left-point integral of f; unexited
 *   paths contribute 0.
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared -pthread -lm
 * (-ffp-contract=off keeps results identical on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Section 4.3 / Table 2).             */
/* ------------------------------------------------------------------------ */

static const uint32_t PHILOX_MUL0 = 0xD2511F53u;
static const uint32_t PHILOX_MUL1 = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL0 = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_WEYL1 = 0xBB67AE85u; /* sqrt(3) - 1 */

/* One Philox S-box round: two 32x32->64 multiplies, then a permutation
 * that XORs the high halves with the untouched words and the round key. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_MUL0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_MUL1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {          /* key schedule: Weyl sequence bump between rounds */
            k[0] += PHILOX_WEYL0;
            k[1] += PHILOX_WEYL1;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

/* Batch form: n counters (4 words each) under one key. */
void or_philox_batch(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* Uniform in (0,1) from the top 23 bits of a word: (2q+1) / 2^24. */
static double uniform23(uint32_t r)
{
    uint32_t q = r >> 9;
    return (2.0 * (double)q + 1.0) / 16777216.0;
}

/* The two standard normals used by Euler step n of path (b, j, i):
 * counter {n/2, i, j, b}, key {seed lo, seed hi}; words (r0, r1) serve even
 * n and (r2, r3) odd n; Box-Muller: rho = sqrt(-2 ln u_a),
 * (xi1, xi2) = rho (cos 2 pi u_b, sin 2 pi u_b). */
void or_step_normals(uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n, double xi[2])
{
    uint32_t ctr[4] = {(uint32_t)(n >> 1), i, j, b};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    or_philox4x32_10(ctr, key, r);
    uint32_t ra = (n & 1) ? r[2] : r[0];
    uint32_t rb = (n & 1) ? r[3] : r[1];
    double ua = uniform23(ra), ub = uniform23(rb);
    double rho = sqrt(-2.0 * log(ua));
    xi[0] = rho * cos(2.0 * M_PI * ub);
    xi[1] = rho * sin(2.0 * M_PI * ub);
}

void or_normals(uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0, int64_t count,
                double* xi /* [count][2] */)
{
    for (int64_t n = 0; n < count; ++n) or_step_normals(seed, b, j, i, n0 + n, xi + 2 * n);
}

/* ------------------------------------------------------------------------ */
/* Stream-function modes and the velocity (Eq. v_expand).                   */
/* ------------------------------------------------------------------------ */

/* Half-plane lattice of |k|_inf <= K without 0: m > 0 with |n| <= K, or
 * m = 0 with 0 < n <= K; ordered by m, then n ascending. */
int64_t or_num_half_modes(int32_t K)
{
    if (K < 0) return 0;
    return (int64_t)K + (int64_t)K * (2 * K + 1);
}

void or_half_modes(int32_t K, int32_t* mn /* [H][2] */)
{
    int64_t h = 0;
    for (int32_t n = 1; n <= K; ++n) { mn[2 * h] = 0; mn[2 * h + 1] = n; ++h; }
    for (int32_t m = 1; m <= K; ++m)
        for (int32_t n = -K; n <= K; ++n) { mn[2 * h] = m; mn[2 * h + 1] = n; ++h; }
}

/* Number of lattice points k in Z^2 with |k|_2 <= r (closed disk, k = 0
 * included), the count the paper's N_u values follow. */
int64_t or_count_disk_modes(double r)
{
    int64_t c = 0;
    int32_t R = (int32_t)floor(r);
    for (int32_t m = -R; m <= R; ++m)
        for (int32_t n = -R; n <= R; ++n)
            if ((double)m * m + (double)n * n <= r * r) ++c;
    return c;
}

typedef struct {
    int32_t K;
    int64_t H;
    int32_t* mn;      /* [H][2] */
    const double* u;  /* [H][2]: (a_h, b_h) */
} field_t;

static int field_init(field_t* f, int32_t K, const double* u)
{
    f->K = K;
    f->H = or_num_half_modes(K);
    f->u = u;
    f->mn = NULL;
    if (f->H > 0) {
        f->mn = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)f->H);
        if (!f->mn) return -1;
        or_half_modes(K, f->mn);
    }
    return 0;
}

static void field_free(field_t* f) { free(f->mn); f->mn = NULL; }

/* psi = sum_h a_h cos(2 pi k_h.x) + b_h sin(2 pi k_h.x);
 * v = (-d psi/dx2, d psi/dx1), i.e. k_perp = (-k_y, k_x) as in Eq. v_expand.
 * Direct sum with one sin and one cos per mode. */
static void velocity_direct(const field_t* f, const double x[2], double v[2])
{
    double v1 = 0.0, v2 = 0.0;
    for (int64_t h = 0; h < f->H; ++h) {
        double m = (double)f->mn[2 * h], n = (double)f->mn[2 * h + 1];
        double a = f->u[2 * h], b = f->u[2 * h + 1];
        double th = 2.0 * M_PI * (m * x[0] + n * x[1]);
        double s = sin(th), c = cos(th);
        double dpsi = -a * s + b * c;          /* d/d(theta) of the mode */
        v1 -= 2.0 * M_PI * n * dpsi;           /* -d psi / dx2 */
        v2 += 2.0 * M_PI * m * dpsi;           /*  d psi / dx1 */
    }
    v[0] = v1;
    v[1] = v2;
}

void or_velocity(int32_t K, const double* u, int64_t npts, const double* x, double* v)
{
    field_t f;
    if (field_init(&f, K, u)) return;
    for (int64_t p = 0; p < npts; ++p) velocity_direct(&f, x + 2 * p, v + 2 * p);
    field_free(&f);
}

void or_stream_function(int32_t K, const double* u, int64_t npts, const double* x, double* psi)
{
    field_t f;
    if (field_init(&f, K, u)) return;
    for (int64_t p = 0; p < npts; ++p) {
        double s = 0.0;
        for (int64_t h = 0; h < f.H; ++h) {
            double th = 2.0 * M_PI * (f.mn[2 * h] * x[2 * p] + f.mn[2 * h + 1] * x[2 * p + 1]);
            s += f.u[2 * h] * cos(th) + f.u[2 * h + 1] * sin(th);
        }
        psi[p] = s;
    }
    field_free(&f);
}

/* theta0(x) = sum_q a_q cos(2 pi k_q.x) + b_q sin(2 pi k_q.x). */
static double theta0_eval(int32_t nq, const int32_t* k, const double* a, const double* b, const double x[2])
{
    double s = 0.0;
    for (int32_t q = 0; q < nq; ++q) {
        double th = 2.0 * M_PI * ((double)k[2 * q] * x[0] + (double)k[2 * q + 1] * x[1]);
        s += a[q] * cos(th) + b[q] * sin(th);
    }
    return s;
}

void or_theta0(int32_t nq, const int32_t* k, const double* a, const double* b, int64_t npts,
               const double* x, double* out)
{
    for (int64_t p = 0; p < npts; ++p) out[p] = theta0_eval(nq, k, a, b, x + 2 * p);
}

/* Boundary data on the circle |y| = R at angle phi = atan2(y2, y1):
 * g = quad (y1^2 - y2^2) + sum_{m=1..n_ang} a_m cos(m phi) + b_m sin(m phi). */
static double gbc_eval(double quad, int32_t n_ang, const double* a, const double* b, const double y[2])
{
    double phi = atan2(y[1], y[0]);
    double s = quad * (y[0] * y[0] - y[1] * y[1]);
    for (int32_t m = 1; m <= n_ang; ++m) s += a[m - 1] * cos(m * phi) + b[m - 1] * sin(m * phi);
    return s;
}

/* Step count for horizon t (a reading: the paper allows variable steps):
 * N = ceil(t/dt - 1e-9); every step is dt except the last, t - (N-1) dt. */
int64_t or_num_steps(double t, double dt)
{
    if (t <= 0.0) return 0;
    return (int64_t)ceil(t / dt - 1e-9);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: one path of the time-dependent problem.                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    field_t field;
    double kappa;
    int32_t nq;
    const int32_t* qk;
    const double* qa;
    const double* qb;
    const double* x;     /* [n_obs][2] */
    const double* t;     /* [n_obs] */
    int64_t n_obs;
    int64_t i0, npaths;  /* paths i0 .. i0+npaths-1 of every observation */
    double dt;
    uint64_t seed;
    uint32_t inst;       /* instance id b of the RNG counter */
    double* g;           /* [n_obs][npaths] */
    double* xend;        /* [n_obs][npaths][2] or NULL */
    const int64_t* jid;  /* RNG observation id of each row, or NULL for j */
    int64_t next;        /* work counter */
    pthread_mutex_t lock;
} td_job_t;

static void td_path(const td_job_t* J, int64_t j, int64_t i, double* g, double* xe)
{
    double X[2] = {J->x[2 * j], J->x[2 * j + 1]};
    int64_t N = or_num_steps(J->t[j], J->dt);
    for (int64_t n = 0; n < N; ++n) {
        double h = (n == N - 1) ? (J->t[j] - (double)(N - 1) * J->dt) : J->dt;
        double v[2], xi[2];
        velocity_direct(&J->field, X, v);
        or_step_normals(J->seed, J->inst, (uint32_t)(J->jid ? J->jid[j] : j), (uint32_t)i, n, xi);
        double sq = sqrt(2.0 * J->kappa * h);
        X[0] = X[0] - v[0] * h + sq * xi[0];
        X[1] = X[1] - v[1] * h + sq * xi[1];
        X[0] -= floor(X[0]);   /* periodic unit square */
        X[1] -= floor(X[1]);
    }
    *g = theta0_eval(J->nq, J->qk, J->qa, J->qb, X);
    if (xe) { xe[0] = X[0]; xe[1] = X[1]; }
}

static int64_t job_take(int64_t* next, pthread_mutex_t* lock, int64_t total, int64_t grain)
{
    pthread_mutex_lock(lock);
    int64_t w = *next;
    if (w < total) *next = w + grain;
    pthread_mutex_unlock(lock);
    return w;
}

static void* td_worker(void* arg)
{
    td_job_t* J = (td_job_t*)arg;
    int64_t total = J->n_obs * J->npaths;
    const int64_t grain = 16;
    for (;;) {
        int64_t w0 = job_take(&J->next, &J->lock, total, grain);
        if (w0 >= total) break;
        int64_t w1 = w0 + grain < total ? w0 + grain : total;
        for (int64_t w = w0; w < w1; ++w) {
            int64_t j = w / J->npaths, p = w % J->npaths;
            td_path(J, j, J->i0 + p, &J->g[w], J->xend ? &J->xend[2 * w] : NULL);
        }
    }
    return NULL;
}

static int resolve_threads(int32_t nthreads)
{
    if (nthreads > 0) return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* Per-path values g[j][p] of Algorithm 1 for paths i0..i0+npaths-1 of each
 * observation j.  Returns the number of threads used, or -1. */
int32_t or_timedep_paths(int32_t K, const double* u, double kappa,
                         int32_t nq, const int32_t* qk, const double* qa, const double* qb,
                         const double* x, const double* t, int64_t n_obs,
                         int64_t i0, int64_t npaths, double dt, uint64_t seed, uint32_t inst,
                         const int64_t* obs_id, int32_t nthreads, double* g, double* xend)
{
    td_job_t J;
    if (field_init(&J.field, K, u)) return -1;
    J.kappa = kappa; J.nq = nq; J.qk = qk; J.qa = qa; J.qb = qb;
    J.x = x; J.t = t; J.n_obs = n_obs; J.i0 = i0; J.npaths = npaths;
    J.dt = dt; J.seed = seed; J.inst = inst; J.g = g; J.xend = xend; J.jid = obs_id; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    int nt = resolve_threads(nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, td_worker, &J);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    field_free(&J.field);
    return nt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: one path of the Dirichlet problem in the disk |x| < R.      */
/* ------------------------------------------------------------------------ */

typedef struct {
    field_t field;
    double drift_scale, kappa;
    double R, quad, f_const;
    int32_t n_ang;
    const double* ga;
    const double* gb;
    const double* x;
    int64_t n_obs, i0, npaths;
    double dt;
    int64_t max_steps;
    uint64_t seed;
    uint32_t inst;
    double* g;
    int64_t* exit_step;  /* [n_obs][npaths]: steps taken to exit, -1 if capped */
    double* xend;        /* [n_obs][npaths][2] or NULL: position at exit */
    const int64_t* jid;  /* RNG observation id of each row, or NULL for j */
    int64_t next;
    pthread_mutex_t lock;
} dr_job_t;

static void dr_path(const dr_job_t* J, int64_t j, int64_t i, double* g, int64_t* nexit, double* xe)
{
    double X[2] = {J->x[2 * j], J->x[2 * j + 1]};
    double R2 = J->R * J->R;
    int64_t n = 0;
    int exited = (X[0] * X[0] + X[1] * X[1] >= R2);
    double sq = sqrt(2.0 * J->kappa * J->dt);
    while (!exited && n < J->max_steps) {
        double v[2], xi[2];
        velocity_direct(&J->field, X, v);
        or_step_normals(J->seed, J->inst, (uint32_t)(J->jid ? J->jid[j] : j), (uint32_t)i, n, xi);
        X[0] = X[0] - J->drift_scale * v[0] * J->dt + sq * xi[0];
        X[1] = X[1] - J->drift_scale * v[1] * J->dt + sq * xi[1];
        ++n;
        exited = (X[0] * X[0] + X[1] * X[1] >= R2);
    }
    if (xe) { xe[0] = X[0]; xe[1] = X[1]; }
    if (!exited) {           /* chi_{tau < infinity} = 0: contributes nothing */
        *g = 0.0;
        *nexit = -1;
        return;
    }
    double r = sqrt(X[0] * X[0] + X[1] * X[1]);
    double y[2] = {J->R * X[0] / r, J->R * X[1] / r};
    double integral_f = 0.0;   /* left-point sum of f(X_m) dt over the n steps */
    for (int64_t m = 0; m < n; ++m) integral_f += J->f_const * J->dt;
    *g = gbc_eval(J->quad, J->n_ang, J->ga, J->gb, y) - integral_f;
    *nexit = n;
}

static void* dr_worker(void* arg)
{
    dr_job_t* J = (dr_job_t*)arg;
    int64_t total = J->n_obs * J->npaths;
    const int64_t grain = 4;
    for (;;) {
        int64_t w0 = job_take(&J->next, &J->lock, total, grain);
        if (w0 >= total) break;
        int64_t w1 = w0 + grain < total ? w0 + grain : total;
        for (int64_t w = w0; w < w1; ++w) {
            int64_t j = w / J->npaths, p = w % J->npaths;
            dr_path(J, j, J->i0 + p, &J->g[w], &J->exit_step[w], J->xend ? &J->xend[2 * w] : NULL);
        }
    }
    return NULL;
}

int32_t or_dirichlet_paths(int32_t K, const double* u, double drift_scale, double kappa,
                           double R, double quad, double f_const, int32_t n_ang,
                           const double* ga, const double* gb,
                           const double* x, int64_t n_obs, int64_t i0, int64_t npaths,
                           double dt, int64_t max_steps, uint64_t seed, uint32_t inst,
                           const int64_t* obs_id, int32_t nthreads, double* g, int64_t* exit_step,
                           double* xend)
{
    dr_job_t J;
    if (field_init(&J.field, K, u)) return -1;
    J.drift_scale = drift_scale; J.kappa = kappa; J.R = R; J.quad = quad; J.f_const = f_const;
    J.n_ang = n_ang; J.ga = ga; J.gb = gb; J.x = x; J.n_obs = n_obs; J.i0 = i0; J.npaths = npaths;
    J.dt = dt; J.max_steps = max_steps; J.seed = seed; J.inst = inst;
    J.g = g; J.exit_step = exit_step; J.xend = xend; J.jid = obs_id; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    int nt = resolve_threads(nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, dr_worker, &J);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    field_free(&J.field);
    return nt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2 in the disk with a general forcing and a state-dependent      */
/* diffusion (Theorem 3.2 with sigma(x), f(x)).                              */
/*   dX = -d v(X) ds + sigma(X) dW,  sigma(x) = diag(s0_1 + s1_1 x_1,        */
/*                                                   s0_2 + s1_2 x_2),       */
/* each coordinate driven by its own Brownian motion and its own diffusion,  */
/* so Eq. millstein applies coordinate by coordinate:                        */
/*   X_i <- X_i - d v_i dt + sigma_i sqrt(dt) xi_i                           */
/*               + (1/2) sigma_i sigma_i' (xi_i^2 - 1) dt   (Milstein),      */
/* sigma_i' = s1_i, all evaluated at the step's start point (the last term   */
/* left out for Euler-Maruyama, Eq. euler).                                  */
/*   f(x) = f_const + sum_q F_q exp(-w |x - c_q|^2),                          */
/* integrated by the left-point rule sum_{m < n} f(X_m) dt.  Exit, boundary  */
/* data and unexited paths as in the constant-coefficient disk problem.      */
/* ------------------------------------------------------------------------ */

typedef struct {
    field_t field;
    double drift_scale, s0[2], s1[2];
    int32_t milstein;
    double R, quad, f_const;
    int32_t n_ang;
    const double* ga;
    const double* gb;
    int32_t n_src;
    double w;
    const double* c;
    const double* F;
    const double* x;
    int64_t n_obs, i0, npaths;
    double dt;
    int64_t max_steps;
    uint64_t seed;
    uint32_t inst;
    double* g;
    int64_t* exit_step;
    double* xend;
    const int64_t* jid;
    int64_t next;
    pthread_mutex_t lock;
} dg_job_t;

static double general_forcing(const dg_job_t* J, const double X[2])
{
    double f = J->f_const;
    for (int q = 0; q < J->n_src; ++q) {
        const double d0 = X[0] - J->c[2 * q], d1 = X[1] - J->c[2 * q + 1];
        f += J->F[q] * exp(-J->w * (d0 * d0 + d1 * d1));
    }
    return f;
}

static void dg_path(const dg_job_t* J, int64_t j, int64_t i, double* g, int64_t* nexit, double* xe)
{
    double X[2] = {J->x[2 * j], J->x[2 * j + 1]};
    const double R2 = J->R * J->R;
    const double sdt = sqrt(J->dt);
    int64_t n = 0;
    int exited = (X[0] * X[0] + X[1] * X[1] >= R2);
    double integral_f = 0.0;
    while (!exited && n < J->max_steps) {
        double v[2], xi[2];
        integral_f += general_forcing(J, X) * J->dt;   /* left point: f at X_n */
        velocity_direct(&J->field, X, v);
        or_step_normals(J->seed, J->inst, (uint32_t)(J->jid ? J->jid[j] : j), (uint32_t)i, n, xi);
        for (int k = 0; k < 2; ++k) {
            const double sig = J->s0[k] + J->s1[k] * X[k];
            double Xn = X[k] - J->drift_scale * v[k] * J->dt + sig * sdt * xi[k];
            if (J->milstein) Xn += 0.5 * sig * J->s1[k] * (xi[k] * xi[k] - 1.0) * J->dt;
            X[k] = Xn;
        }
        ++n;
        exited = (X[0] * X[0] + X[1] * X[1] >= R2);
    }
    if (xe) { xe[0] = X[0]; xe[1] = X[1]; }
    if (!exited) {
        *g = 0.0;
        *nexit = -1;
        return;
    }
    const double r = sqrt(X[0] * X[0] + X[1] * X[1]);
    const double y[2] = {J->R * X[0] / r, J->R * X[1] / r};
    *g = gbc_eval(J->quad, J->n_ang, J->ga, J->gb, y) - integral_f;
    *nexit = n;
}

static void* dg_worker(void* arg)
{
    dg_job_t* J = (dg_job_t*)arg;
    const int64_t total = J->n_obs * J->npaths;
    const int64_t grain = 4;
    for (;;) {
        const int64_t w0 = job_take(&J->next, &J->lock, total, grain);
        if (w0 >= total) break;
        const int64_t w1 = w0 + grain < total ? w0 + grain : total;
        for (int64_t w = w0; w < w1; ++w) {
            const int64_t j = w / J->npaths, p = w % J->npaths;
            dg_path(J, j, J->i0 + p, &J->g[w], &J->exit_step[w], J->xend ? &J->xend[2 * w] : NULL);
        }
    }
    return NULL;
}

int32_t or_dirichlet_general_paths(int32_t K, const double* u, double drift_scale, const double* s0,
                                   const double* s1, int32_t milstein, double R, double quad, double f_const,
                                   int32_t n_ang, const double* ga, const double* gb, int32_t n_src, double w,
                                   const double* c, const double* F, const double* x, int64_t n_obs, int64_t i0,
                                   int64_t npaths, double dt, int64_t max_steps, uint64_t seed, uint32_t inst,
                                   const int64_t* obs_id, int32_t nthreads, double* g, int64_t* exit_step,
                                   double* xend)
{
    dg_job_t J;
    if (field_init(&J.field, K, u)) return -1;
    J.drift_scale = drift_scale;
    J.s0[0] = s0[0]; J.s0[1] = s0[1]; J.s1[0] = s1[0]; J.s1[1] = s1[1];
    J.milstein = milstein;
    J.R = R; J.quad = quad; J.f_const = f_const; J.n_ang = n_ang; J.ga = ga; J.gb = gb;
    J.n_src = n_src; J.w = w; J.c = c; J.F = F;
    J.x = x; J.n_obs = n_obs; J.i0 = i0; J.npaths = npaths; J.dt = dt; J.max_steps = max_steps;
    J.seed = seed; J.inst = inst; J.g = g; J.exit_step = exit_step; J.xend = xend; J.jid = obs_id; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    const int nt = resolve_threads(nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, dg_worker, &J);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    field_free(&J.field);
    return nt;
}

/* ------------------------------------------------------------------------ */
/* The optimal-forcing boundary-value problem of Section 4 (Eq. bvp:ex1),    */
/* by Algorithm 2 / Theorem 3.2 in the unit square:                          */
/*   -b . grad theta + kappa Laplace theta = sum_q F_q phi_q(x),             */
/*   phi_q(x) = exp(-w |x - c_q|^2),  theta = g on the boundary,             */
/*   g(y) = g_cos (cos(pi y1 / 2) + cos(pi y2 / 2)) / 2 + g_quad (y1^2 - y2^2).*/
/* theta(x; F) = E[g(X_tau)] - sum_q F_q E[int_0^tau phi_q(X_s) ds] with     */
/* dX = -b ds + sqrt(2 kappa) dW.  One path returns the n_src + 1 values     */
/* (g(X_tau), sum_m phi_1(X_m) dt, ..., sum_m phi_n(X_m) dt), m < n_exit.    */
/* Exit: the first step with X outside the open square; X_tau is the exit    */
/* position clamped to the square.  A path that reaches max_steps returns    */
/* zeros (the chi_{tau < infinity} of Theorem 3.2) and exit step -1.         */
/* ------------------------------------------------------------------------ */

typedef struct {
    double b[2], kappa, w, g_cos, g_quad;
    int32_t n_src;
    const double* c;
    const double* x;
    int64_t n_obs, i0, npaths;
    double dt;
    int64_t max_steps;
    uint64_t seed;
    uint32_t inst;
    double* out;         /* [n_obs][n_src + 1][npaths] */
    int64_t* exit_step;  /* [n_obs][npaths] */
    const int64_t* jid;
    int64_t next;
    pthread_mutex_t lock;
} sq_job_t;

static int outside_unit_square(const double X[2])
{
    return X[0] <= 0.0 || X[0] >= 1.0 || X[1] <= 0.0 || X[1] >= 1.0;
}

static void sq_path(const sq_job_t* J, int64_t j, int64_t i, int64_t w)
{
    const int64_t nf = J->n_src + 1, P = J->npaths, p = w % P;
    double* o = J->out + (j * nf) * P + p;  /* value q at o[q * P] */
    double X[2] = {J->x[2 * j], J->x[2 * j + 1]};
    double sums[16];
    for (int q = 0; q < J->n_src; ++q) sums[q] = 0.0;
    const double sq = sqrt(2.0 * J->kappa * J->dt);
    int64_t n = 0;
    int exited = outside_unit_square(X);
    while (!exited && n < J->max_steps) {
        for (int q = 0; q < J->n_src; ++q) {  /* left-point rule: phi at X_n */
            const double d0 = X[0] - J->c[2 * q], d1 = X[1] - J->c[2 * q + 1];
            sums[q] += exp(-J->w * (d0 * d0 + d1 * d1)) * J->dt;
        }
        double xi[2];
        or_step_normals(J->seed, J->inst, (uint32_t)(J->jid ? J->jid[j] : j), (uint32_t)i, n, xi);
        X[0] = X[0] - J->b[0] * J->dt + sq * xi[0];
        X[1] = X[1] - J->b[1] * J->dt + sq * xi[1];
        ++n;
        exited = outside_unit_square(X);
    }
    if (!exited) {
        for (int64_t q = 0; q < nf; ++q) o[q * P] = 0.0;
        J->exit_step[j * P + p] = -1;
        return;
    }
    const double y0 = X[0] < 0.0 ? 0.0 : (X[0] > 1.0 ? 1.0 : X[0]);
    const double y1 = X[1] < 0.0 ? 0.0 : (X[1] > 1.0 ? 1.0 : X[1]);
    const double pi = 3.14159265358979323846;
    o[0] = J->g_cos * 0.5 * (cos(0.5 * pi * y0) + cos(0.5 * pi * y1)) + J->g_quad * (y0 * y0 - y1 * y1);
    for (int q = 0; q < J->n_src; ++q) o[(q + 1) * P] = sums[q];
    J->exit_step[j * P + p] = n;
}

static void* sq_worker(void* arg)
{
    sq_job_t* J = (sq_job_t*)arg;
    const int64_t total = J->n_obs * J->npaths;
    const int64_t grain = 16;
    for (;;) {
        const int64_t w0 = job_take(&J->next, &J->lock, total, grain);
        if (w0 >= total) break;
        const int64_t w1 = w0 + grain < total ? w0 + grain : total;
        for (int64_t w = w0; w < w1; ++w) sq_path(J, w / J->npaths, J->i0 + w % J->npaths, w);
    }
    return NULL;
}

int32_t or_square_bvp_paths(const double* b, double kappa, int32_t n_src, const double* c, double w,
                            double g_cos, double g_quad, const double* x, int64_t n_obs, int64_t i0,
                            int64_t npaths, double dt, int64_t max_steps, uint64_t seed, uint32_t inst,
                            const int64_t* obs_id, int32_t nthreads, double* out, int64_t* exit_step)
{
    if (n_src < 0 || n_src > 16) return -1;
    sq_job_t J;
    J.b[0] = b[0]; J.b[1] = b[1]; J.kappa = kappa; J.w = w; J.g_cos = g_cos; J.g_quad = g_quad;
    J.n_src = n_src; J.c = c; J.x = x; J.n_obs = n_obs; J.i0 = i0; J.npaths = npaths; J.dt = dt;
    J.max_steps = max_steps; J.seed = seed; J.inst = inst; J.out = out; J.exit_step = exit_step;
    J.jid = obs_id; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    const int nt = resolve_threads(nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, sq_worker, &J);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    return nt;
}
