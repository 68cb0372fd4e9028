// pm_general_step.cuh -- the per-step terms of Algorithm 2 with a general
// forcing and a state-dependent diffusion (Theorem 3.2 with f(x) and
// sigma(x)), shared by the FP32-pipe kernel (pm_dirichlet_general.cu) and the
// tensor-core kernel (pm_dirichlet_tc.cuh), so that the two differ only in how
// the velocity sum is evaluated.
//
//   dX = -d v(X) ds + sigma(X) dW,  sigma(x) = diag(s0_1 + s1_1 x_1, s0_2 + s1_2 x_2):
// each coordinate has its own Brownian motion and a diffusion coefficient of
// its own coordinate, so the Milstein scheme (Eq. millstein) applies
// coordinate by coordinate,
//   X_i <- X_i - d v_i dt + sigma_i sqrt(dt) xi_i + (1/2) sigma_i s1_i (xi_i^2 - 1) dt,
// sigma_i at the step's start point (without the last term: Euler-Maruyama,
// Eq. euler).  The forcing f(x) = f_const + sum_q F_q exp(-w |x - c_q|^2) is
// integrated by the left-point rule, dt sum_{m < n} f(X_m), in a compensated
// sum (float paths) or in double.
#pragma once
#include <cmath>
#include "pm_device.cuh"
#include "pm_launch.h"

namespace pm {

template <typename Real>
struct ForcingSum;
template <>
struct ForcingSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct ForcingSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ float exp_g(float a) { return expf(a); }
__device__ __forceinline__ double exp_g(double a) { return exp(a); }

// The coefficients of the general step in the path precision.
template <typename Real>
struct GeneralCoef {
    Real s0[2], s1[2];  // sigma_i(x) = s0[i] + s1[i] x_i
    Real sqdt;          // sqrt(dt)
    Real half_dt_m;     // dt / 2 with the Milstein term, else 0
    Real w;
    Real fc;            // f_const
    Real c[2 * kMaxSources];
    Real F[kMaxSources];
    int32_t n_src;

    void set(const DirichletGeneral& G, double dt, double f_const)
    {
        for (int k = 0; k < 2; ++k) {
            s0[k] = (Real)G.s0[k];
            s1[k] = (Real)G.s1[k];
        }
        sqdt = (Real)std::sqrt(dt);
        half_dt_m = G.milstein ? (Real)(0.5 * dt) : (Real)0;
        w = (Real)G.w;
        fc = (Real)f_const;
        n_src = G.n_src;
        for (int q = 0; q < kMaxSources; ++q) {
            const bool on = q < G.n_src;
            c[2 * q] = on ? (Real)G.c[2 * q] : (Real)0;
            c[2 * q + 1] = on ? (Real)G.c[2 * q + 1] : (Real)0;
            F[q] = on ? (Real)G.F[q] : (Real)0;
        }
    }

    // f(X) at the step's start point.
    __device__ __forceinline__ Real forcing(Real x1, Real x2) const
    {
        Real f = fc;
        for (int q = 0; q < n_src; ++q) {
            const Real a = x1 - c[2 * q], b = x2 - c[2 * q + 1];
            f += F[q] * exp_g(-w * (a * a + b * b));
        }
        return f;
    }

    // Coordinate i's increment: -d v dt + sigma sqrt(dt) xi (+ Milstein).
    __device__ __forceinline__ Real increment(int i, Real x, Real v, Real drift_dt, Real xi) const
    {
        const Real sig = s0[i] + s1[i] * x;
        Real d = -v * drift_dt + (sig * sqdt) * xi;
        d += ((sig * s1[i]) * half_dt_m) * (xi * xi - (Real)1);
        return d;
    }
};

}  // namespace pm
