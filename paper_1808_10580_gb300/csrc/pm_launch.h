// pm_launch.h -- host-side launch descriptors shared by the C ABI (pm_api.cu)
// and the per-precision kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pm {

constexpr int kMaxTheta0 = 64;    // PM_MAX_THETA0_MODES
constexpr int kMaxBoundary = 32;  // PM_MAX_BOUNDARY_MODES

// Per-observation record built on the device from (x_j, t_j): start point,
// step count N_j, length and noise scale of the last step.
struct ObsRec {
    double x1, x2;
    double h_last;  // t_j - (N_j - 1) dt
    double s_last;  // sqrt(2 kappa h_last)
    int32_t nsteps;
    int32_t pad;
};

// Sizes of the velocity coefficient table for wave-number bound K.
inline constexpr int table_size(int K) { return (K + 1) * (K + 1) * 8; }

struct TimedepLaunch {
    const double* coef;  // host: pre-scaled product-basis table, table_size(K) entries
    int nq;              // theta0 modes (host arrays)
    const int32_t* qk;
    const double* qa;
    const double* qb;
    const ObsRec* obs;       // device [n_obs]
    const int32_t* order;    // device [n_obs] processing order, or nullptr
    double2* part;           // device [n_obs * chunks] (sum g, sum g^2) per CTA
    double* g_out;           // device [n_obs * M] or nullptr
    double* x_out;           // device [n_obs * M * 2] or nullptr
    double dt, s_dt;         // regular step and sqrt(2 kappa dt)
    int64_t M, path_offset;
    int32_t n_obs, chunks;
    uint32_t inst, key0, key1;
};

struct DirichletLaunch {
    const double* coef;      // host table
    double drift_scale;
    double R, quad, f_const;
    int n_ang;
    const double* ga;        // host [n_ang]
    const double* gb;
    const double* x;         // device [n_obs][2]
    int64_t n_obs, M;
    double dt, s_dt;
    int64_t max_steps;
    unsigned long long* counter;     // device, zero on entry: next unclaimed path
    unsigned long long* n_unexited;  // device, zero on entry
    double* g;                       // device [n_obs * M] per-path values
    int32_t* exit_step;              // device [n_obs * M] or nullptr
    double* x_out;                   // device [n_obs * M * 2] or nullptr
    int64_t path_offset;
    uint32_t inst, key0, key1;
    int grid;                        // persistent CTAs
};

// Kernel block size of the time-dependent kernel (one path per thread).
constexpr int kTimedepBlock = 128;
// Block size of the persistent Dirichlet kernel.
constexpr int kDirichletBlock = 128;

template <typename Real, int K> cudaError_t launch_timedep(const TimedepLaunch& L, cudaStream_t s);
template <typename Real, int K> cudaError_t launch_dirichlet(const DirichletLaunch& L, cudaStream_t s);
template <typename Real, int K> cudaError_t launch_velocity(const double* coef, const double* x, int64_t n,
                                                            double* v, cudaStream_t s);
template <typename Real, int K> int dirichlet_blocks_per_sm();

// Stores `msg` as the calling thread's pm_last_error() text; returns `code`.
int set_error(int code, const char* msg);

// Support kernels (pm_support.cu).
cudaError_t launch_prep_timedep(const double* x, const double* t, int64_t n_obs, double dt, double kappa,
                                ObsRec* rec, int32_t* order, unsigned int* err, cudaStream_t s);
cudaError_t launch_reduce(const double2* part, int64_t n_obs, int32_t chunks, int64_t M, double* mean,
                          double* var, cudaStream_t s);
cudaError_t launch_reduce_paths(const double* g, int64_t n_obs, int64_t M, double* mean, double* var,
                                cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_normals(uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0, int64_t count,
                           double* out, bool fp64, cudaStream_t s);

}  // namespace pm
