// pm_device.cuh -- device building blocks of the particle step (sm_103a).
//
//  * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11)
//    and the Box-Muller transform: the Brownian increments xi ~ N(0,1) of the
//    Euler-Maruyama step (Eq. euler).
//  * The divergence-free velocity of a Fourier stream function (Eq. v_expand),
//    evaluated in a separable product basis with trigonometric recurrences.
//  * Compensated (hi, lo) float positions.
//
// Conventions shared with the host code (pm_api.cu) and fixed by the library's
// input format (include/pm.h):
//   RNG: step n of path i of observation j in instance b uses Philox on counter
//   {n/2, i, j, b} under key {seed lo32, seed hi32}; words (r0, r1) serve even n,
//   (r2, r3) odd n; u = (2 (r >> 9) + 1) 2^-24; rho = sqrt(-2 ln u_a);
//   xi = rho (cos 2 pi u_b, sin 2 pi u_b).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pm {

// --------------------------------------------------------------------------
// Philox4x32-10
// --------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kMul0 * c.x, hi0 = __umulhi(kMul0, c.x);
        const uint32_t lo1 = kMul1 * c.z, hi1 = __umulhi(kMul1, c.z);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    return c;
}

// The same generator with its round keys precomputed (rk[2r] = k0 + r W0,
// rk[2r+1] = k1 + r W1, modulo 2^32; round_keys below): where the keys are
// the same for every thread, the table sits in the kernel-parameter bank and
// each key is an operand of the XOR, with no additions in the rounds.
__device__ __forceinline__ u32x4 philox4x32_10_rk(u32x4 c, const uint32_t (&rk)[20])
{
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kMul0 * c.x, hi0 = __umulhi(kMul0, c.x);
        const uint32_t lo1 = kMul1 * c.z, hi1 = __umulhi(kMul1, c.z);
        c = u32x4{hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0};
    }
    return c;
}

inline void round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[20])
{
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

// Uniform in (0, 1) from the top 23 bits: (2q + 1) 2^-24, exact in float.
template <typename Real>
__device__ __forceinline__ Real uniform23(uint32_t r)
{
    return (Real)((r >> 9) * 2u + 1u) * (Real)5.9604644775390625e-08;  // 2^-24
}

__device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
__device__ __forceinline__ float log_(float a) { return logf(a); }
__device__ __forceinline__ double log_(double a) { return log(a); }
__device__ __forceinline__ float sqrt_(float a) { return sqrtf(a); }
__device__ __forceinline__ double sqrt_(double a) { return sqrt(a); }

// sin and cos of 2 pi x for both halves of x (the particle's two coordinates,
// each in [0, 1) or at most a few units from it), for the harmonic
// recurrences.  Reduction to a quarter turn: q = rint(4x) by the rounding of
// 4x + 1.5 2^23 (exact for |4x| < 2^22; the low bits of that sum are q), and
// r = x - q/4 in [-1/8, 1/8], formed exactly by one FMA; with t = 2 pi r in
// [-pi/4, pi/4] the Taylor series of sin t to t^9 and of cos t to t^10 (the
// next terms are below 1.8e-9 and 1.2e-10), written in r with the
// coefficients (-1)^k (2 pi)^n / n!, evaluated by Horner's rule on packed
// pairs; then the rotation by q quarter turns, (sin, cos) -> (cos, -sin) per
// quarter.  Measured in an FP32 emulation against float64 sin/cos: absolute
// error below 8.4e-8, relative below 1.7 ulp away from the exact zeros.
__device__ __forceinline__ float2 pair(float v) { return make_float2(v, v); }

__device__ __forceinline__ void sincos_turns2(float2 x, float2& s, float2& c)
{
    constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
    const float2 t = __ffma2_rn(x, pair(4.0f), pair(kRound));
    const float2 q = __fadd2_rn(t, pair(-kRound));
    const float2 r = __ffma2_rn(q, pair(-0.25f), x);
    const float2 r2 = __fmul2_rn(r, r);
    float2 ps = __ffma2_rn(r2, pair(42.058692932128906f), pair(-76.70585632324219f));
    ps = __ffma2_rn(r2, ps, pair(81.6052474975586f));
    ps = __ffma2_rn(r2, ps, pair(-41.34170150756836f));
    ps = __ffma2_rn(r2, ps, pair(6.2831854820251465f));
    const float2 S = __fmul2_rn(r, ps);
    float2 pc = __ffma2_rn(r2, pair(-26.42625617980957f), pair(60.2446403503418f));
    pc = __ffma2_rn(r2, pc, pair(-85.45681762695312f));
    pc = __ffma2_rn(r2, pc, pair(64.93939208984375f));
    pc = __ffma2_rn(r2, pc, pair(-19.739208221435547f));
    const float2 C = __ffma2_rn(r2, pc, pair(1.0f));
    const uint32_t q0 = __float_as_uint(t.x), q1 = __float_as_uint(t.y);
    const float s0 = (q0 & 1u) ? C.x : S.x, c0 = (q0 & 1u) ? S.x : C.x;
    const float s1 = (q1 & 1u) ? C.y : S.y, c1 = (q1 & 1u) ? S.y : C.y;
    s = make_float2(__uint_as_float(__float_as_uint(s0) ^ ((q0 & 2u) << 30)),
                    __uint_as_float(__float_as_uint(s1) ^ ((q1 & 2u) << 30)));
    c = make_float2(__uint_as_float(__float_as_uint(c0) ^ (((q0 + 1u) & 2u) << 30)),
                    __uint_as_float(__float_as_uint(c1) ^ (((q1 + 1u) & 2u) << 30)));
}

// The pair of normals from words (ra, rb).
template <typename Real>
__device__ __forceinline__ void box_muller(uint32_t ra, uint32_t rb, Real& xi1, Real& xi2)
{
    const Real ua = uniform23<Real>(ra), ub = uniform23<Real>(rb);
    const Real rho = sqrt_((Real)-2 * log_(ua));
    Real s, c;
    sincos2pi(ub, &s, &c);
    xi1 = rho * c;
    xi2 = rho * s;
}

// Float uniforms by bits: 0x3F800000 | (r >> 9) is 1 + q 2^-23 with q the top
// 23 bits of r, and subtracting 1 - 2^-24 is exact (the operands lie within a
// factor of two of each other), which leaves (2q + 1) 2^-24, the value of
// uniform23, without an integer-to-float conversion.
__device__ __forceinline__ float one_plus_mantissa(uint32_t r) { return __uint_as_float(0x3F800000u | (r >> 9)); }

// The normals of two consecutive steps from one Philox block, packed (the
// tensor-core kernels): .x from words (a0, b0), .y from (a1, b1); the same
// transform as box_muller<float> with the angle's sin and cos from
// sincos_turns2 (error below 1e-7) instead of sincospif, so the two forms agree
// to that error, not bit for bit.  The FP32-pipe kernels keep the scalar form:
// there the extra code of the series changed the compiler's register
// allocation of the velocity loop and cost up to 3.7x (K = 64).
__device__ __forceinline__ void box_muller2(uint32_t a0, uint32_t b0, uint32_t a1, uint32_t b1, float2& xi1,
                                            float2& xi2)
{
    const float2 ua = __fadd2_rn(make_float2(one_plus_mantissa(a0), one_plus_mantissa(a1)), pair(-0x1.fffffep-1f));
    const float2 ub = __fadd2_rn(make_float2(one_plus_mantissa(b0), one_plus_mantissa(b1)), pair(-0x1.fffffep-1f));
    const float2 l = __fmul2_rn(make_float2(logf(ua.x), logf(ua.y)), pair(-2.0f));
    const float2 rho = make_float2(sqrtf(l.x), sqrtf(l.y));
    float2 s, c;
    sincos_turns2(ub, s, c);
    xi1 = __fmul2_rn(rho, c);
    xi2 = __fmul2_rn(rho, s);
}

// --------------------------------------------------------------------------
// Velocity of the stream function in the product basis.
//
// psi = sum_{m,n >= 0} A C1m C2n + B C1m S2n + G S1m C2n + D S1m S2n with
// C1m = cos 2 pi m x1, S1m = sin 2 pi m x1 (and C2n, S2n in x2).  Then
//   v1 = -d2 psi = sum_m C1m P1c(m) + S1m P1s(m),
//   v2 =  d1 psi = sum_m C1m P2c(m) + S1m P2s(m),
//   P1c = sum_n e0 S2n + e1 C2n,  P1s = sum_n e2 S2n + e3 C2n,
//   P2c = sum_n f0 C2n + f1 S2n,  P2s = sum_n f2 C2n + f3 S2n,
// with the pre-scaled table (built on the host, pm_api.cu: stage_coefficients)
//   e = 2 pi n (A, -B, G, -D),  f = 2 pi m (G, D, -A, -B).
// Each real coefficient costs exactly two FMAs (one per velocity component).
// Table layout: Coef[(m (K+1) + n) * 8 + {e0..e3, f0..f3}].
// --------------------------------------------------------------------------
template <int K>
__host__ __device__ constexpr int coef_count() { return (K + 1) * (K + 1) * 8; }

template <typename Real, int K>
struct FieldTable { Real c[coef_count<K>()]; };

// Powers e^{2 pi i n x} for n = 0..K by complex recurrence from e^{2 pi i x}.
template <typename Real, int K>
__device__ __forceinline__ void fourier_powers(Real x, Real (&C)[K + 1], Real (&S)[K + 1])
{
    Real s1, c1;
    sincos2pi(x, &s1, &c1);
    C[0] = (Real)1;
    S[0] = (Real)0;
    if constexpr (K >= 1) { C[1] = c1; S[1] = s1; }
#pragma unroll
    for (int n = 2; n <= K; ++n) {
        // even n from the square of n/2 (shorter dependency chain), odd from n-1
        const int a = (n & 1) ? n - 1 : n / 2;
        const int b = n - a;
        C[n] = C[a] * C[b] - S[a] * S[b];
        S[n] = S[a] * C[b] + C[a] * S[b];
    }
}

template <typename Real>
struct Quad { Real x, y, z, w; };

// Coefficient sources.  `quad(i)` yields entries 4i .. 4i+3 of the table.
// ParamTable: the table lives in the kernel-parameter bank; after unrolling
// every index is a compile-time constant, so each coefficient becomes an FMA
// operand and costs no instruction.
template <typename Real, int K>
struct ParamTable {
    const FieldTable<Real, K>& f;
    __device__ __forceinline__ Quad<Real> quad(int i) const
    {
        return Quad<Real>{f.c[4 * i], f.c[4 * i + 1], f.c[4 * i + 2], f.c[4 * i + 3]};
    }
};

// SharedTable: the table lives in shared memory; each quad is one broadcast
// 128-bit load.  The kernel places a compiler barrier at the top of every step
// so that these loads cannot be hoisted out of the path loop (which would need
// one register per coefficient), while inside a step they can be scheduled
// ahead of their uses.
struct SharedTable {
    const float4* base;
    __device__ __forceinline__ Quad<float> quad(int i) const
    {
        const float4 v = base[i];
        return Quad<float>{v.x, v.y, v.z, v.w};
    }
};

// Wave-number bounds above this are "wide": the table (8 (K+1)^2 floats, more
// than the kernel-parameter bank holds from K = 32 on) is staged in shared
// memory, and the loop over m stays rolled (the unrolled sum would be some
// 10^4 instructions, far beyond the instruction cache).
constexpr int kMaxUnrolledK = 16;

// P particles at once (each coefficient quad is fetched once and serves all P).
template <typename Real, int K, int P, typename Tab>
__device__ __forceinline__ void velocity(const Tab& tab, const Real (&x1)[P], const Real (&x2)[P],
                                         Real (&v1)[P], Real (&v2)[P])
{
    constexpr bool kRolled = K > kMaxUnrolledK;
    Real C2[P][K + 1], S2[P][K + 1], c1[P], s1[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        fourier_powers<Real, K>(x2[q], C2[q], S2[q]);
        sincos2pi(x1[q], &s1[q], &c1[q]);
        v1[q] = (Real)0;
        v2[q] = (Real)0;
    }
    // m = 0: only the v1 part (d1 of a function of x2 alone vanishes).
#pragma unroll
    for (int n = 1; n <= K; ++n) {
        const Quad<Real> E = tab.quad((0 * (K + 1) + n) * 2);
#pragma unroll
        for (int q = 0; q < P; ++q) v1[q] = fma_(E.x, S2[q][n], fma_(E.y, C2[q][n], v1[q]));
    }
    Real C1m[P], S1m[P];
#pragma unroll
    for (int q = 0; q < P; ++q) { C1m[q] = (Real)1; S1m[q] = (Real)0; }
#pragma unroll(kRolled ? 1 : K)
    for (int m = 1; m <= K; ++m) {
        Real p1c[P], p1s[P], p2c[P], p2s[P];
        const Quad<Real> F0 = tab.quad((m * (K + 1)) * 2 + 1);  // n = 0 column: f0 and f2
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const Real cn = C1m[q] * c1[q] - S1m[q] * s1[q];
            S1m[q] = S1m[q] * c1[q] + C1m[q] * s1[q];
            C1m[q] = cn;
            // n = 0 column: C20 = 1, S20 = 0, and its v1 factor 2 pi n vanishes.
            p1c[q] = (Real)0;
            p1s[q] = (Real)0;
            p2c[q] = F0.x;
            p2s[q] = F0.z;
        }
#pragma unroll
        for (int n = 1; n <= K; ++n) {
            const int o = (m * (K + 1) + n) * 2;
            const Quad<Real> E = tab.quad(o), F = tab.quad(o + 1);
#pragma unroll
            for (int q = 0; q < P; ++q) {
                p1c[q] = fma_(E.x, S2[q][n], fma_(E.y, C2[q][n], p1c[q]));
                p1s[q] = fma_(E.z, S2[q][n], fma_(E.w, C2[q][n], p1s[q]));
                p2c[q] = fma_(F.x, C2[q][n], fma_(F.y, S2[q][n], p2c[q]));
                p2s[q] = fma_(F.z, C2[q][n], fma_(F.w, S2[q][n], p2s[q]));
            }
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            v1[q] = fma_(C1m[q], p1c[q], fma_(S1m[q], p1s[q], v1[q]));
            v2[q] = fma_(C1m[q], p2c[q], fma_(S1m[q], p2s[q], v2[q]));
        }
    }
}

// --------------------------------------------------------------------------
// Positions.  Float paths keep X = hi + lo (compensated), so the position is
// carried to ~2^-48 while the velocity is evaluated at hi.  Double paths keep
// one double.
// --------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

template <typename Real> struct Coord;

template <> struct Coord<float> {
    float hi, lo;
    __device__ __forceinline__ void set(double x) { hi = (float)x; lo = (float)(x - (double)hi); }
    __device__ __forceinline__ void add(float d)
    {
        float s, e;
        two_sum(hi, d + lo, s, e);
        hi = s;
        lo = e;
    }
    // Periodic wrap into [0, 1): subtract floor(hi) exactly, keeping the rounding in lo.
    __device__ __forceinline__ void wrap()
    {
        if (hi < 0.0f || hi >= 1.0f) {
            const float f = floorf(hi);
            float s, e;
            two_sum(hi, -f, s, e);
            hi = s;
            lo += e;
            if (hi >= 1.0f) hi -= 1.0f;  // hi rounded up to exactly 1
        }
    }
    __device__ __forceinline__ float val() const { return hi; }
    __device__ __forceinline__ double full() const { return (double)hi + (double)lo; }
};

template <> struct Coord<double> {
    double hi;
    __device__ __forceinline__ void set(double x) { hi = x; }
    __device__ __forceinline__ void add(double d) { hi = hi + d; }
    __device__ __forceinline__ void wrap() { hi = hi - floor(hi); }
    __device__ __forceinline__ double val() const { return hi; }
    __device__ __forceinline__ double full() const { return hi; }
};

// Fractional part of k1 x1 + k2 x2 (integer k) for positions X = hi + lo,
// formed with exact product errors so that high wave numbers keep their phase.
__device__ __forceinline__ float phase_frac(int k1, int k2, const Coord<float>& a, const Coord<float>& b)
{
    const float f1 = (float)k1, f2 = (float)k2;
    const float p1 = f1 * a.hi, e1 = fmaf(f1, a.hi, -p1);
    const float p2 = f2 * b.hi, e2 = fmaf(f2, b.hi, -p2);
    const float r1 = p1 - rintf(p1), r2 = p2 - rintf(p2);
    return (r1 + r2) + (e1 + e2 + fmaf(f1, a.lo, f2 * b.lo));
}

__device__ __forceinline__ double phase_frac(int k1, int k2, const Coord<double>& a, const Coord<double>& b)
{
    const double p = (double)k1 * a.hi + (double)k2 * b.hi;
    return p - rint(p);
}

// Sign of |X|^2 - R^2 for a compensated position, with exact product and sum
// errors so that the exit decision matches a double-precision test.
__device__ __forceinline__ float radial_excess(const Coord<float>& a, const Coord<float>& b, float R2hi, float R2lo)
{
    const float p1 = a.hi * a.hi, e1 = fmaf(a.hi, a.hi, -p1);
    const float p2 = b.hi * b.hi, e2 = fmaf(b.hi, b.hi, -p2);
    float s, es;
    two_sum(p1, p2, s, es);
    float d, ed;
    two_sum(s, -R2hi, d, ed);
    const float cross = 2.0f * fmaf(a.hi, a.lo, b.hi * b.lo);
    return d + (ed + es + e1 + e2 + cross - R2lo);
}

// The exit decision radial_excess(a, b, R2hi, R2lo) >= 0, with a float test
// first.  For a compensated position (|lo| <= ulp(hi) / 2) the float value
// q = a.hi^2 + b.hi^2 is within 2^-22 (relative) of the exact |X|^2, and R^2 =
// R2hi + R2lo within 2^-24, so wherever q - R2hi exceeds `band` = 2^-16 R2hi in
// magnitude its sign is that of |X|^2 - R^2 (a margin of 2^5 over the bound);
// only inside the band, a few millionths of R^2 wide, the exact form runs.
// The decision is the same as the exact form's in every case.
__device__ __forceinline__ bool exits_disk(const Coord<float>& a, const Coord<float>& b, float R2hi, float R2lo,
                                           float band)
{
    const float d = fmaf(a.hi, a.hi, b.hi * b.hi) - R2hi;
    if (fabsf(d) > band) return d > 0.f;
    return radial_excess(a, b, R2hi, R2lo) >= 0.f;
}

// Double paths: |X|^2 with each product and the sum rounded once (no fused
// multiply-add), compared with R^2.
__device__ __forceinline__ double radial_excess(const Coord<double>& a, const Coord<double>& b, double R2hi, double)
{
    return __dadd_rn(__dmul_rn(a.hi, a.hi), __dmul_rn(b.hi, b.hi)) - R2hi;
}

}  // namespace pm
