// pm_launch.h -- host-side launch descriptors shared by the C ABI (pm_api.cu)
// and the per-precision kernel translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pm {

constexpr int kMaxTheta0 = 64;    // PM_MAX_THETA0_MODES
constexpr int kMaxBoundary = 32;  // PM_MAX_BOUNDARY_MODES
// Full bound of a tensor-core wait (mbarrier polls, a few seconds at most).
constexpr uint32_t kWaitPolls = 1u << 22;

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
__host__ __device__ inline constexpr int table_size(int K) { return (K + 1) * (K + 1) * 8; }

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
    // Shared paths (PM_SHARE_PATHS): n_groups records {m0, m1, stream, nmax}
    // (members[m0..m1) sorted by step count), in launch order; nullptr: one
    // observation per CTA row of the grid (order[] or identity).
    const int4* groups = nullptr;  // device [n_groups]
    const int32_t* members = nullptr;  // device [n_obs]
    int32_t n_groups = 0;
    // Wide K (K > 16): device buffer of wide_table_floats(K) floats that the
    // launcher fills with its coefficient table before the kernel reads it.
    float* table_dev = nullptr;
    // Tensor-core kernels: polls of the per-step MMA wait before it gives up
    // (the full bound unless a test lowers it, see pm_set_wait_limit).
    uint32_t wait_limit = kWaitPolls;
};

// Paths per CTA of the time-dependent tensor-core kernel at K: two 128-row
// particle tiles at K = 56, one otherwise (see td_sets in pm_timedep_tc.cuh).
inline int td_tc_rows(int K) { return K == 56 ? 256 : 128; }

// Wave-number bounds of the time-dependent map beyond the unrolled kernels.
inline bool wide_K(int K) { return K == 24 || K == 32 || K == 40 || K == 48 || K == 56 || K == 64; }
// The widest bound, K = 80 (N_u = 25,920, which holds the paper's 20,081
// coefficients of |k|_2 <= 80): the time-dependent map with float paths on the
// FP32 pipes only (its 8 (K+1)^2-float table, 210 KB, still fits one CTA's
// shared memory; the tensor-core tiles of this bound would not).
inline bool simt_wide_K(int K) { return K == 80; }

// Floats of the device table a wide-K launch needs: the product-basis table
// (8 (K+1)^2) of the FP32-pipe kernel or the padded W^T of the tensor-core
// kernel (NP rows of 2 ceil((2K+1)/8) chunks of 4 TF32, or of
// 2 ceil((2K+1)/16) chunks of 8 FP16; NP = 4K+1 rounded up to 16), whichever
// is largest.
inline int64_t wide_table_floats(int K)
{
    const int64_t simt = 8 * (int64_t)(K + 1) * (K + 1);
    const int64_t np = (4 * K + 1 + 15) / 16 * 16;
    const int64_t tf32 = np * 4 * (2 * ((2 * K + 1 + 7) / 8));
    const int64_t f16 = np * 8 * (2 * ((2 * K + 1 + 15) / 16));
    const int64_t tc = tf32 > f16 ? tf32 : f16;
    return simt > tc ? simt : tc;
}

// Algorithm 2 with a general forcing and a state-dependent diffusion (see
// pm_forward_dirichlet_general): sigma_i(x) = s0[i] + s1[i] x_i, the Milstein
// term when `milstein`, f = f_const + sum_q F[q] exp(-w |x - c_q|^2).
constexpr int kMaxSources = 8;  // PM_MAX_SOURCES
struct DirichletGeneral {
    double s0[2], s1[2];
    int milstein;
    int n_src;
    double w;
    double c[2 * kMaxSources];
    double F[kMaxSources];
};

struct DirichletLaunch {
    const double* coef;      // host table
    double drift_scale;
    double R, quad, f_const;
    int n_ang;
    const double* ga;        // host [n_ang]
    const double* gb;
    const double* x;         // device [n_obs][2]
    const int32_t* order = nullptr;  // device [n_obs]: observation whose paths are claimed in slot s
    int64_t n_obs, M;
    double dt, s_dt;
    int64_t max_steps;
    unsigned long long* counter;     // device, zero on entry: next unclaimed path
    unsigned long long* n_unexited;  // device, zero on entry
    unsigned long long* steps;       // device, zero on entry: total Euler steps
    double* g;                       // device [n_obs * M] per-path values
    int32_t* exit_step;              // device [n_obs * M] or nullptr
    double* x_out;                   // device [n_obs * M * 2] or nullptr
    int64_t path_offset;
    uint32_t inst, key0, key1;
    int grid;                        // persistent CTAs
    uint32_t wait_limit = kWaitPolls;  // tensor-core kernel: polls of the per-step MMA wait
    const DirichletGeneral* gen = nullptr;  // host: general forcing and diffusion, or nullptr
    int refill_pairs = 4;            // tensor-core kernel: pairs of steps between lane refills
    // Wide K (K > 16, float paths): device buffer of wide_table_floats(K)
    // floats that the launcher fills with its coefficient table.
    float* table_dev = nullptr;
};

// Kernel block size of the time-dependent kernel (one path per thread).
constexpr int kTimedepBlock = 128;
// Paths (threads) per CTA of the FP32-pipe time-dependent kernel at K: 256
// where one CTA's shared-memory copy of the velocity table (32 (K+1)^2 bytes)
// leaves no room for a second CTA on the SM (K = 64, 80), so that each
// scheduler still has two warps to hide the table loads, and at K = 56, where
// two 128-thread CTAs with a 104 KB table each measured 1.6x slower (3.88
// against 2.47 s on the 300 x 1e4-path workload); kTimedepBlock otherwise.
constexpr int td_simt_rows(int K)
{
    return K > 16 && (K >= 56 || 2 * 32 * (K + 1) * (K + 1) > 227 * 1024) ? 2 * kTimedepBlock : kTimedepBlock;
}
// Block size of the persistent Dirichlet kernel.
constexpr int kDirichletBlock = 128;

template <typename Real, int K> cudaError_t launch_timedep(const TimedepLaunch& L, cudaStream_t s);
template <typename Real, int K> cudaError_t launch_dirichlet(const DirichletLaunch& L, cudaStream_t s);
template <typename Real, int K> cudaError_t launch_velocity(const double* coef, const double* x, int64_t n,
                                                            double* v, cudaStream_t s);
template <typename Real, int K> int dirichlet_blocks_per_sm();
template <typename Real, int K> cudaError_t launch_dirichlet_general(const DirichletLaunch& L, cudaStream_t s);
template <typename Real, int K> int dirichlet_general_blocks_per_sm();

// Stores `msg` as the calling thread's pm_last_error() text; returns `code`.
int set_error(int code, const char* msg);

// Support kernels (pm_support.cu).
cudaError_t launch_prep_timedep(const double* x, const double* t, int64_t n_obs, double dt, double kappa,
                                ObsRec* rec, int32_t* order, unsigned int* err, cudaStream_t s,
                                unsigned long long* steps = nullptr, int64_t M = 0);
cudaError_t launch_reduce(const double2* part, int64_t n_obs, int32_t chunks, int64_t M, double* mean,
                          double* var, cudaStream_t s);
// Per-path values g [n_obs][M] -> mean, var.  For M > kReducePathChunk the
// reduction runs in two passes through `part` ([n_obs][reduce_path_chunks(M)]
// scratch); with part == nullptr, or shorter rows, one CTA per observation.
constexpr int64_t kReducePathChunk = 8192;
int32_t reduce_path_chunks(int64_t M);
cudaError_t launch_reduce_paths(const double* g, int64_t n_obs, int64_t M, double* mean, double* var,
                                cudaStream_t s, double2* part = nullptr);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                          cudaStream_t s);
cudaError_t launch_sincos_turns(const float* x, int64_t n, float* s, float* c, cudaStream_t st);
cudaError_t launch_normals(uint64_t seed, uint32_t b, uint32_t j, uint32_t i, int64_t n0, int64_t count,
                           double* out, bool fp64, bool packed, cudaStream_t s);

}  // namespace pm

namespace pm {

// ---- batched forward map (pm_batched.cuh, pm_batched_support.cu) ----
template <typename Real>
struct Theta0Table {
    int32_t n;
    int32_t k1[kMaxTheta0];
    int32_t k2[kMaxTheta0];
    Real a[kMaxTheta0];
    Real b[kMaxTheta0];
};

struct BatchInstDev {
    const double* u;      // device coefficients [2|H_K|]
    int32_t kind;         // 0 time-dependent, 1 Dirichlet
    int32_t n_obs;
    int64_t M;
    int64_t row0;         // first row of the batch arrays
    int64_t path_base;    // path (j, i) of the instance is g[path_base + j*M + i]
    int64_t n_paths;      // n_obs * M
    int64_t max_steps;
    double dt, kappa, drift_scale;
    uint32_t key0, key1;
    uint32_t stream;      // RNG instance word
    uint32_t pad;
};

struct RowRec {
    double x1, x2;
    double h_last, s_last;
    int32_t nsteps;
    int32_t pad;
};

struct BatchKernelParams {
    Theta0Table<float> th;
    double ga[kMaxBoundary];
    double gb[kMaxBoundary];
    double R, quad, f_const;
    int32_t n_ang;
    float R2hi, R2lo;
    float band;                        // exits_disk: 2^-16 R2hi
    const BatchInstDev* inst;
    const RowRec* rows;
    const float* tables;               // [B][table_size(K)]
    unsigned long long* next_path;     // [B] per-instance path counters (zero on entry)
    unsigned long long* n_unexited;
    unsigned long long* steps;         // total Euler steps taken (all paths)
    double* g;                         // per-path values
    unsigned* tc_err;                  // set when a tensor-core wait expires (tensor-core kernel)
    int32_t B;
    int32_t refill_pairs;              // tensor-core kernel: pairs of steps between lane refills
};

template <int K> cudaError_t launch_batched(const BatchKernelParams& p, int grid, cudaStream_t s);
template <int K> int batched_blocks_per_sm();
// Velocity tables of all instances on the device (Eq. v_expand, the same fold
// as the host staging): tables[b][table_size(K)] from inst[b].u.
cudaError_t launch_stage_tables(const BatchInstDev* inst, int B, int K, float* tables, cudaStream_t s);
// Per-row records (start point, step count, last step) of every instance.
cudaError_t launch_prep_rows(const BatchInstDev* inst, int B, int max_obs, const double* x, const double* t,
                             RowRec* rows, unsigned* err, cudaStream_t s);
// Per-row mean and variance from the per-path values.
cudaError_t launch_reduce_rows(const BatchInstDev* inst, int B, int max_obs, const double* g, double* mean,
                               double* var, cudaStream_t s);

// Time-dependent map with the velocity sum on the tensor cores (pm_timedep_tc.cuh);
// *err is set when a bounded wait expires.
namespace tdtc {
template <int K> cudaError_t launch_timedep_tc(const TimedepLaunch& L, unsigned* err, cudaStream_t s);
template <int K> cudaError_t launch_dirichlet_tc(const DirichletLaunch& L, unsigned* err, cudaStream_t s);
template <int K> int dirichlet_tc_blocks_per_sm(bool gen = false);
template <int K> cudaError_t launch_batched_tc(const BatchKernelParams& p, int grid, cudaStream_t s);
template <int K> int batched_tc_blocks_per_sm();
}

}  // namespace pm
