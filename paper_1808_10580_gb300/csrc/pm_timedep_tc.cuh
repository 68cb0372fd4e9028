// pm_timedep_tc.cuh -- Algorithm 1 with the velocity sum on the tensor cores.
//
// The velocity of the stream function (Eq. v_expand) in the product basis is
//   v1 = P(0) + sum_{m>=1} C1m P1c(m) + S1m P1s(m),   v2 = sum_{m>=1} C1m P2c(m) + S1m P2s(m),
// where every partial sum P(.)(m) is linear in the x2 harmonics
//   a = (S2_1, C2_1, S2_2, C2_2, ..., S2_K, C2_K, 1)   (interleaved; see acol_s).
// For the 128 particles of a CTA this is one matrix product per Euler step,
//   P[128 x (4K+1)] = A[128 x (2K+1)] . W[(2K+1) x (4K+1)],
// issued as tcgen05.mma with the FP32 accumulator in tensor memory: kind::tf32
// for K <= 8, kind::f16 with FP16 operands from K = 10 (see Shape).  Both
// operand types keep 11 significant bits, so every operand is split
// x = hi + lo and three products hi.hi + lo.hi + hi.lo are accumulated (the
// lo.lo term and the rounding of lo, ~2^-21 relative, are dropped): close to
// float accuracy.  The remaining 4K+1 FMAs per particle, the harmonics, the
// noise and the Euler step stay on the FP32 pipes.
//
// Per step: every thread writes its particle's row of A (hi and lo) into a
// K-major tile (layout at tile_off), four harmonics at a time; a CTA barrier
// hands the tile to the tensor core (one thread issues 3 KS MMAs and commits
// to an mbarrier); the threads compute the step's noise (and, in some
// kernels, the x1 harmonics) while it runs, and every thread reads its
// accumulator columns back with tcgen05.ld, four per m.
#pragma once
#include <algorithm>
#include <cmath>
#include <cuda_fp16.h>
#include "pm_gemm_tc.cuh"
#include "pm_kernels.cuh"

namespace pm {
namespace tdtc {

// F ("folded"): the constant column of A (the n = 0 terms of v2) and the
// m = 0 column of P (the x1-independent part of v1) leave the product and are
// summed on the FP32 pipes (4K FMAs per particle), so that A has 2K columns
// and P 4K: for K a multiple of 4 that saves 16 columns of N and, where 2K + 1
// would start a new k-step, a k-step.
//
// H ("half"): the operands are FP16 instead of TF32 (kind::f16).  FP16 keeps
// the same 11 significant bits as TF32, so the same hi + lo split and three
// products give the same accuracy, with half the tile bytes and twice the MMA
// rate; W is scaled by a power of two so that its entries sit in FP16's
// normal range, and the accumulator is scaled back exactly.
template <int K, bool F = false, bool H = false>
struct Shape {
    static constexpr bool FOLD = F;
    static constexpr bool HALF = H;
    static constexpr int EPC = H ? 8 : 4;             // operand elements per 16-byte chunk
    static constexpr int KD = F ? 2 * K : 2 * K + 1;  // A columns used
    static constexpr int KS = (KD + 2 * EPC - 1) / (2 * EPC);  // MMA k-steps (two chunks each)
    static constexpr int KC = 2 * KS;                 // 16-byte chunks per tile row
    static constexpr int WS = EPC * KC;               // row stride of W (elements)
    static constexpr int MC = 8 * ((K + 1) / 2);      // columns of the m >= 1 sums (pairs of m, see pcol)
    static constexpr int NC = F ? MC : MC + 1;        // accumulator columns used
    static constexpr int NP = (NC + 15) / 16 * 16;    // MMA N (multiple of 16)
    static constexpr int SBO = KC * 128;              // bytes between 8-row groups of a tile
    static constexpr int A_BYTES = 128 * KC * 16;     // 128 rows x KC chunks
    static constexpr int B_BYTES = NP * KC * 16;      // NP rows x KC chunks
    static constexpr int SMEM = 2 * A_BYTES + 2 * B_BYTES + 128 + 64;
    // allocation: a power of 2 >= 32
    static constexpr uint32_t TMEM_COLS = NP <= 64 ? 64u : NP <= 128 ? 128u : 256u;
    // CTAs per SM the kernels are compiled for: what the 228 KB of shared memory
    // (1 KB reserved each) and the 512 TMEM columns hold, at most 8 (32 warps)
    static constexpr int CTAS_SMEM = 233472 / (SMEM + 1024);
    static constexpr int CTAS_TMEM = 512 / (int)TMEM_COLS;
    static constexpr int MIN_CTAS = CTAS_SMEM < CTAS_TMEM ? (CTAS_SMEM < 8 ? CTAS_SMEM : 8) : (CTAS_TMEM < 8 ? CTAS_TMEM : 8);
    // the same with at most 6 (kernels that hold the x1 harmonics across the MMA wait)
    static constexpr int MIN_CTAS6 = MIN_CTAS < 6 ? MIN_CTAS : 6;
    // W^T travels in the kernel-parameter bank up to 16 KB, else in global memory.
    static constexpr bool W_PARAM = NP * WS * 4 <= 16384;
    static_assert(NP <= 256, "accumulator within 256 TMEM columns (one MMA: N <= 256)");
    static_assert(MIN_CTAS >= 1, "tiles fit shared memory");
};

// The time-dependent kernel folds where that removes padding (K a multiple of
// 4) and measured faster: not at K = 4 (the product is too small for the
// saving to pay for the FMAs), nor at K = 24 (measured 91 ms against 81 ms
// unfolded on the 300 x 1e4-path workload).
template <int K>
constexpr bool fold_of() { return K % 4 == 0 && K >= 8 && K != 24; }
// FP16 operands where they measured faster: from K = 10 on (K <= 8: the
// product is small and the wider split costs more than the MMA time it saves).
template <int K>
constexpr bool half_of() { return K >= 10; }
template <int K>
using TdShape = Shape<K, fold_of<K>(), half_of<K>()>;

// Particle tiles of 128 rows per CTA of the time-dependent kernel: two where
// one tile's CTA already fills the SM's shared memory with W and a second
// tile still fits beside it, so that the SM has two sets of particles to
// alternate; the two tiles share the coefficient tiles.  K = 56 (measured
// 227.8 against 235.6 ms on the 300 x 1e4-path workload); at K = 48 one and
// two tiles measured the same (181.0 and 180.7 ms).  (Mirrored by td_tc_rows
// in pm_launch.h.)
template <int K>
constexpr int td_sets() { return K == 56 ? 2 : 1; }

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both K-major.
template <int NP>
__host__ __device__ constexpr uint32_t idesc_tf32() { return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(128 >> 4) << 24); }

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B (both the
// same type), both K-major.
template <int NP>
__host__ __device__ constexpr uint32_t idesc_f16() { return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(128 >> 4) << 24); }

// hi = a rounded to FP16, lo = (a - hi) rounded to FP16, two values packed per
// word (a0 in the low half); the dropped remainder is ~2^-22 |a|.  a - hi is
// formed by the mixed-precision FMA (FP16 operands, FP32 addend) hi * (-1) + a,
// which is exact, so no separate widening of hi is needed.
__device__ __forceinline__ void split_f16x2(float a0, float a1, uint32_t& hi, uint32_t& lo)
{
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(a1), "f"(a0));
    float r0, r1;
    asm("{\n .reg .b16 h0, h1, m1;\n mov.b32 {h0, h1}, %2;\n mov.b16 m1, 0xBC00;\n"
        " fma.rn.f32.f16 %0, h0, m1, %3;\n fma.rn.f32.f16 %1, h1, m1, %4;\n}\n"
        : "=f"(r0), "=f"(r1)
        : "r"(hi), "f"(a0), "f"(a1));
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r1), "f"(r0));
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Tiles are K-major without swizzling: 8 x 16-byte core matrices (8 rows x 4
// tf32 or 8 fp16, 128 contiguous bytes), the KC core matrices of an 8-row
// group side by side (128 B apart along K), 8-row groups SBO = KC x 128 B
// apart.  One MMA k-step (8 tf32 or 16 fp16: 32 bytes) spans two core
// matrices along K.
// Byte offset of 16-byte chunk c of row r.
template <int KC>
__device__ __forceinline__ uint32_t tile_off(int r, int c) { return (uint32_t)((r >> 3) * (KC * 128) + (r & 7) * 16 + c * 128); }

// Shared-memory matrix descriptor of such a tile: leading-dimension (K) byte
// offset 128 B between core matrices, stride-dimension byte offset SBO
// between 8-row groups, no swizzle.
template <int SBO>
__device__ __forceinline__ uint64_t tile_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // swizzle mode 0
}

// Descriptor start-address units (16 B) per k-step: two core matrices.
constexpr uint64_t kKStep = 256 >> 4;

// CTAs of a tensor-core kernel that fit on one SM at once, from its register
// count, its shared memory and the 512 tensor-memory columns (each CTA
// allocates tmem_cols).  Persistent grids are this many CTAs per SM.
inline int resident_ctas(const void* fn, int threads, int dyn_smem, int tmem_cols)
{
    int dev = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int regs_sm = 65536, smem_sm = 0, max_blocks = 32, max_thr = 2048, reserved = 0;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&max_blocks, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&max_thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int warps = (threads + 31) / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
    int nb = regs_warp > 0 ? regs_sm / (regs_warp * warps) : max_blocks;
    const int smem_cta = dyn_smem + (int)fa.sharedSizeBytes + reserved;
    if (smem_cta > 0 && smem_sm > 0) nb = std::min(nb, smem_sm / smem_cta);
    nb = std::min(nb, max_thr / threads);
    nb = std::min(nb, max_blocks);
    nb = std::min(nb, 512 / tmem_cols);
    return std::max(nb, 1);
}

template <int K>
struct Params {
    // W^T: row nc (accumulator column), entry k (A column); in W, or at Wg.
    float W[TdShape<K>::W_PARAM ? TdShape<K>::NP * TdShape<K>::WS : 1];
    const float* Wg;
    // Folded shape: the m = 0 coefficients of v1 (S2_n at n-1, C2_n at K+n-1)
    // and the n = 0 coefficients of v2 (C1m at m-1, S1m at K+m-1); read in
    // pairs over consecutive n (m), so 8-byte aligned.
    alignas(8) float T0[2 * K];
    alignas(8) float N0[2 * K];
    float inv_s;              // FP16 operands: 1 / (power-of-two scale of W)
    Theta0Table<float> th;
    const ObsRec* obs;
    const int32_t* order;
    double2* part;
    double* g_out;
    double* x_out;
    float dt, s_dt;
    int64_t M, path_offset;
    int32_t n_obs, chunks;
    uint32_t inst, key0, key1;
    uint32_t rk[20];          // Philox round keys of (key0, key1)
    unsigned* err;
    uint32_t wait_limit;      // polls of the per-step MMA wait (tc::kWaitLimit unless a test lowers it)
    const int4* groups;       // shared paths: {m0, m1, stream, nmax} per grid row, or nullptr
    const int32_t* members;   // [n_obs] observation indices of the groups
};

template <int NP>
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc_f16<NP>()), "r"(accumulate)
        : "memory");
}

template <int NP>
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc_tf32<NP>()), "r"(accumulate)
        : "memory");
}

// 16 accumulator columns of this thread's lane; the wait is part of the same
// statement, so the outputs are valid when it ends.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// hi = a with its 13 low mantissa bits cleared (exact in TF32), lo = a - hi
// (exact in float); the tensor core reduces lo to TF32 itself, an error of at
// most 2^-20 |a|.
__device__ __forceinline__ void split_tf32(float a, float& hi, float& lo)
{
    hi = __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
    lo = a - hi;
}

// Exponent e of the power-of-two scale of W for FP16 operands: the largest
// |entry| times 2^e lies in [2^13, 2^14) (e = 0 for a zero W).
__host__ __device__ inline int w_scale_exp(float wmax)
{
    if (!(wmax > 0.f)) return 0;
    int E = 0;
    frexpf(wmax, &E);  // wmax = f 2^E, f in [1/2, 1)
    const int e = 14 - E;
    return e < -60 ? -60 : (e > 60 ? 60 : e);
}

// The coefficient tiles (hi / lo) of the B operand from W^T: entry k of row nc
// is w(nc * WS + k), already scaled for FP16 operands.
template <typename S, typename Load>
__device__ __forceinline__ void stage_B(uint8_t* B_hi, uint8_t* B_lo, int tid, Load w)
{
    for (int q = tid; q < S::NP * S::KC; q += (int)blockDim.x) {
        const int r = q / S::KC, c = q - r * S::KC;
        if constexpr (S::HALF) {
            uint32_t hv[4], lv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i0 = r * S::WS + 8 * c + 2 * e;
                split_f16x2(w(i0), w(i0 + 1), hv[e], lv[e]);
            }
            *reinterpret_cast<uint4*>(B_hi + tile_off<S::KC>(r, c)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<uint4*>(B_lo + tile_off<S::KC>(r, c)) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
        } else {
            float4 h, l;
            float* hv = &h.x;
            float* lv = &l.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float x = w(r * S::WS + 4 * c + e);
                hv[e] = to_tf32(x);
                lv[e] = to_tf32(x - hv[e]);
            }
            *reinterpret_cast<float4*>(B_hi + tile_off<S::KC>(r, c)) = h;
            *reinterpret_cast<float4*>(B_lo + tile_off<S::KC>(r, c)) = l;
        }
    }
}

// Host: scales W (and the n = 0 terms of a folded shape, N0[2K]) by 2^e for
// FP16 operands; returns 2^-e, the factor that undoes it.
template <typename S>
float scale_W_host(float* W, float* N0, int nN0)
{
    if constexpr (!S::HALF) {
        return 1.f;
    } else {
        float wmax = 0.f;
        for (int q = 0; q < S::NP * S::WS; ++q) wmax = std::max(wmax, std::fabs(W[q]));
        const int e = w_scale_exp(wmax);
        const float sc = std::ldexp(1.f, e);
        for (int q = 0; q < S::NP * S::WS; ++q) W[q] *= sc;
        for (int q = 0; q < nN0; ++q) N0[q] *= sc;
        return std::ldexp(1.f, -e);
    }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, const float4& v)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// Tiles at shared address sb: A_hi, A_lo (A_BYTES each), then B_hi, B_lo; a
// thread's row of the particle tiles starts at sb + tile_off(r, 0), chunk c
// 128 c bytes further, the lo tile lo_off bytes after the hi tile.
__device__ __forceinline__ void st_shared_v4u(uint32_t addr, const uint32_t (&v)[4])
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}

// Layouts of A and P.  A columns interleave the x2 harmonics: S2_n at 2(n-1),
// C2_n at 2(n-1)+1 (n = 1..K), the constant 1 at 2K (unfolded shape).  P
// takes the m >= 1 sums in blocks of eight columns per pair of wave numbers
// (m, m+1), m odd: P1c(m), P1c(m+1), P1s(m), P1s(m+1), P2c(m), P2c(m+1),
// P2s(m), P2s(m+1) (for odd K the last block's m+1 = K+1 columns are zero);
// P(0) follows them at column MC = 8 ceil(K/2) in the unfolded shape.  The
// pairs of a block start at even columns, so each lands in an aligned
// register pair of tcgen05.ld and meets the x1 harmonics of the same pair of
// wave numbers in one packed FMA (see velocity_stream); and a thread
// produces and consumes the harmonics four wave numbers at a time (one
// 16-column load per group of four) instead of holding all K at once.
__host__ __device__ constexpr int acol_s(int n) { return 2 * (n - 1); }
__host__ __device__ constexpr int acol_c(int n) { return 2 * (n - 1) + 1; }
template <bool F>
__host__ __device__ constexpr int pcol(int m, int j) { return 8 * ((m - 1) / 2) + 2 * j + ((m - 1) & 1); }
__host__ __device__ constexpr int p0col(int K) { return 8 * ((K + 1) / 2); }

// Whether the position is wrapped into [0, 1) after step n (other than a
// path's last step, after which it always is): every 32nd step (between
// wraps a position drifts at most 32 steps outside the cell; sincos_turns2
// reduces any |x| < 2^20 exactly).  The kernels that must give the same
// bits (the single-problem and batched time-dependent steps) share this
// schedule, keyed by the path's own step.
__device__ __forceinline__ bool wrap_due(int n) { return (n & 31) == 31; }

// Packed FP32 pairs (sm_100 and later: one instruction for two independent
// float operations, each rounded exactly as its scalar form).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Euler step of both coordinates (Eq. euler), two at a time: per coordinate
// the operations of em_update<float> and Coord<float>::add (increment
// s xi - v h by one FMA, then added to (hi, lo) with the compensated two-sum),
// so the results are those of the scalar form bit for bit.
__device__ __forceinline__ void em_update2(Coord<float>& X1, Coord<float>& X2, float v1, float v2, float h, float s,
                                           float xi1, float xi2)
{
    const float2 d = __ffma2_rn(make_float2(s, s), make_float2(xi1, xi2),
                                __fmul2_rn(make_float2(-v1, -v2), make_float2(h, h)));
    const float2 a = make_float2(X1.hi, X2.hi);
    const float2 b = __fadd2_rn(d, make_float2(X1.lo, X2.lo));
    const float2 sm = __fadd2_rn(a, b);
    const float2 bp = __fadd2_rn(sm, neg2(a));
    const float2 e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(sm, neg2(bp)))), __fadd2_rn(b, neg2(bp)));
    X1.hi = sm.x;
    X2.hi = sm.y;
    X1.lo = e.x;
    X2.lo = e.y;
}

// e^{i n 2 pi x} for n = 4g + j (j = 1..4), group by group: e^{i j 2 pi x}
// from one sin/cos and products, times the group base e^{i 4g 2 pi x}, which
// is the j = 4 harmonic of the group before (a recurrence of depth g + 2).
// The values of a group come as pairs over j, C12 = (C_{4g+1}, C_{4g+2}),
// C34 = (C_{4g+3}, C_{4g+4}) and likewise S12, S34, each pair from one packed
// multiply and one packed FMA per component:
//   C_n = bc c_j - bs s_j,   S_n = bs c_j + bc s_j   (FMA of the first product),
// with the base (bc, bs) held in both halves of a pair.  Group 0 is e^{i j 2 pi x}
// itself (the base is 1).
struct Harm4 {
    float2 c12, c34, s12, s34;  // cos / sin of j 2 pi x, j = 1..4, paired over j
    float2 bc, bs;              // the current group base, in both halves
    // from sin and cos of 2 pi x (sincos_turns2)
    __device__ __forceinline__ void init(float s1, float c1)
    {
        const float c2 = fmaf(c1, c1, -s1 * s1), s2 = 2.f * (s1 * c1);
        const float c3 = fmaf(c2, c1, -s2 * s1), s3 = fmaf(s2, c1, c2 * s1);
        const float c4 = fmaf(c2, c2, -s2 * s2), s4 = 2.f * (s2 * c2);
        c12 = make_float2(c1, c2);
        c34 = make_float2(c3, c4);
        s12 = make_float2(s1, s2);
        s34 = make_float2(s3, s4);
        bc = make_float2(c4, c4);  // base of group 1
        bs = make_float2(s4, s4);
    }
    // Group G's harmonics (G in order: 0, 1, 2, ...); from G = 1 on the base
    // must be that of group G (advance() after each group).  With HALF, only
    // C12 / S12 (the last group of K = 4g + 2).
    template <int G, bool HALF = false>
    __device__ __forceinline__ void group(float2& C12, float2& S12, float2& C34, float2& S34) const
    {
        if constexpr (G == 0) {
            C12 = c12; S12 = s12; C34 = c34; S34 = s34;
        } else {
            const float2 nbs = neg2(bs);
            C12 = __ffma2_rn(bc, c12, __fmul2_rn(nbs, s12));
            S12 = __ffma2_rn(bs, c12, __fmul2_rn(bc, s12));
            if constexpr (!HALF) {
                C34 = __ffma2_rn(bc, c34, __fmul2_rn(nbs, s34));
                S34 = __ffma2_rn(bs, c34, __fmul2_rn(bc, s34));
            }
        }
    }
    // The base of the next group: the j = 4 harmonic of group G >= 1 just formed.
    __device__ __forceinline__ void advance(const float2& C34, const float2& S34)
    {
        bc = make_float2(C34.y, C34.y);
        bs = make_float2(S34.y, S34.y);
    }
};

// Harmonic groups of a coordinate, as the velocity sum consumes them: G = the
// group index, Q = groups of four wave numbers, with K <= 4Q.
template <int K>
constexpr int harm_groups() { return (K + 3) / 4; }

// This thread's row of A from its x2, written as hi / lo tiles at row and
// row + lo_off, eight columns (four harmonics) at a time; folded shape: returns
// the m = 0 part of v1, p0 = sum_n T0[n-1] S2_n + T0[K+n-1] C2_n (eight
// independent partial sums, paired: this runs before the step's barrier).
template <int K, bool F, bool H, int G = 0>
__device__ __forceinline__ void write_row_groups(uint32_t row, uint32_t lo_off, Harm4& h, const float* T0, float2 (&ps)[4])
{
    constexpr int NCOL = 2 * K + (F ? 0 : 1);
    if constexpr (8 * G < NCOL) {
        float2 C12, S12, C34 = make_float2(0.f, 0.f), S34 = make_float2(0.f, 0.f);
        constexpr bool half = 4 * G + 2 >= K;  // only n = 4G+1, 4G+2 exist
        h.template group<G, half>(C12, S12, C34, S34);
        if constexpr (G >= 1 && 4 * G + 4 < K) h.advance(C34, S34);  // (group 1's base comes from init)
        // columns (S_n, C_n) for n = 4G+1 .. 4G+4, zero / the unit column beyond K
        float v[8] = {S12.x, C12.x, S12.y, C12.y, S34.x, C34.x, S34.y, C34.y};
        if constexpr (F) {
            // 4G+j <= K for all j: folded shapes have K a multiple of 4
            const float2* t0 = reinterpret_cast<const float2*>(T0);
            ps[0] = __ffma2_rn(t0[2 * G], S12, ps[0]);
            ps[1] = __ffma2_rn(t0[2 * G + 1], S34, ps[1]);
            ps[2] = __ffma2_rn(t0[K / 2 + 2 * G], C12, ps[2]);
            ps[3] = __ffma2_rn(t0[K / 2 + 2 * G + 1], C34, ps[3]);
        }
        if constexpr (H) {
            uint32_t hv[4], lv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (4 * G + q + 1 <= K) {
                    split_f16x2(v[2 * q], v[2 * q + 1], hv[q], lv[q]);
                } else {  // the unit column (FP16 1.0 = 0x3C00 in the low half) or zero padding: exact
                    hv[q] = (!F && 8 * G + 2 * q == 2 * K) ? 0x3C00u : 0u;
                    lv[q] = 0u;
                }
            }
            st_shared_v4u(row + 128u * G, hv);
            st_shared_v4u(row + lo_off + 128u * G, lv);
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (4 * G + e / 2 + 1 > K) v[e] = (!F && 8 * G + e == 2 * K) ? 1.f : 0.f;
#pragma unroll
            for (int half_ = 0; half_ < 2; ++half_) {
                float4 hi, lo;
                split_tf32(v[4 * half_], hi.x, lo.x);
                split_tf32(v[4 * half_ + 1], hi.y, lo.y);
                split_tf32(v[4 * half_ + 2], hi.z, lo.z);
                split_tf32(v[4 * half_ + 3], hi.w, lo.w);
                st_shared_v4(row + 128u * (2 * G + half_), hi);
                st_shared_v4(row + lo_off + 128u * (2 * G + half_), lo);
            }
        }
        write_row_groups<K, F, H, G + 1>(row, lo_off, h, T0, ps);
    }
}

template <int K, bool F, bool H>
__device__ __forceinline__ float write_row_stream(uint32_t row, uint32_t lo_off, float s2, float c2, const float* T0)
{
    Harm4 h;
    h.init(s2, c2);
    float2 ps[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    write_row_groups<K, F, H>(row, lo_off, h, T0, ps);
    if constexpr (F) return ((ps[0].x + ps[0].y) + (ps[1].x + ps[1].y)) + ((ps[2].x + ps[2].y) + (ps[3].x + ps[3].y));
    return 0.f;
}

// Sources of the x1 harmonics, group by group, both from the same Harm4
// sequence (so results do not depend on the choice): computed as the
// velocity sum needs them (few registers, after the MMA wait), or all before
// the wait into arrays (overlapping the MMA, K + 1 pairs of registers).
struct HarmStream {
    Harm4 h;
    __device__ __forceinline__ void init(float s1, float c1) { h.init(s1, c1); }
    template <int G, bool HALF>
    __device__ __forceinline__ void group(float2& C12, float2& S12, float2& C34, float2& S34)
    {
        h.template group<G, HALF>(C12, S12, C34, S34);
        if constexpr (G >= 1 && !HALF) h.advance(C34, S34);
    }
};

template <int K>
struct HarmArray {
    static constexpr int Q = harm_groups<K>();
    float2 c12[Q], s12[Q], c34[Q], s34[Q];
    template <int G>
    __device__ __forceinline__ void fill(Harm4& h)
    {
        if constexpr (G < Q) {
            constexpr bool half = 4 * G + 2 >= K;
            c34[G] = s34[G] = make_float2(0.f, 0.f);
            h.template group<G, half>(c12[G], s12[G], c34[G], s34[G]);
            if constexpr (G >= 1 && !half) h.advance(c34[G], s34[G]);
            fill<G + 1>(h);
        }
    }
    __device__ __forceinline__ void init(float s1, float c1)
    {
        Harm4 h;
        h.init(s1, c1);
        fill<0>(h);
    }
    template <int G, bool HALF>
    __device__ __forceinline__ void group(float2& C12, float2& S12, float2& C34, float2& S34) const
    {
        C12 = c12[G]; S12 = s12[G]; C34 = c34[G]; S34 = s34[G];
    }
};

// The velocity from this lane's accumulator row and the x1 harmonics (source
// src, initialised from x1), one 16-column load per group of four wave
// numbers:
//   v1 = P(0) + sum_m C1m P1c(m) + S1m P1s(m),
//   v2 = sum_m C1m (P2c(m) + N0c(m)) + S1m (P2s(m) + N0s(m)),
// with P(0) and N0 from the FP32 pipes in the folded shape.  Each of the four
// sums advances as a packed pair over (m, m+1), m odd (the column blocks of
// pcol), so every packed FMA takes an aligned pair of accumulator columns and
// a harmonic pair of the group as they come; the halves (odd and even m) are
// added at the end.  FP16 operands: the sums over the accumulator carry the
// scale of W, removed by inv_s.
template <int K, bool F, bool H, int G, typename Src>
__device__ __forceinline__ void velocity_groups(uint32_t t_row, Src& src, const float* N0, float& p0, float2 (&acc)[4])
{
    constexpr int NP = ((F ? p0col(K) : p0col(K) + 1) + 15) / 16 * 16;
    if constexpr (16 * G < NP) {
        float a[16];
        tmem_ld16(t_row + 16u * G, a);
        if constexpr (4 * G < K) {
            constexpr bool half = 4 * G + 2 >= K;
            float2 C12, S12, C34, S34;
            src.template group<G, half>(C12, S12, C34, S34);
#pragma unroll
            for (int b = 0; b < (half ? 1 : 2); ++b) {  // the blocks (m, m+1), m = 4G+1 and 4G+3
                const float2 C = b ? C34 : C12, S = b ? S34 : S12;
                const float* e = a + 8 * b;
                float2 p2c = make_float2(e[4], e[5]), p2s = make_float2(e[6], e[7]);
                if constexpr (F) {
                    const float2* n0 = reinterpret_cast<const float2*>(N0);
                    p2c = __fadd2_rn(p2c, n0[2 * G + b]);          // N0c(m), N0c(m+1)
                    p2s = __fadd2_rn(p2s, n0[K / 2 + 2 * G + b]);  // N0s(m), N0s(m+1)
                }
                acc[0] = __ffma2_rn(C, make_float2(e[0], e[1]), acc[0]);
                acc[1] = __ffma2_rn(S, make_float2(e[2], e[3]), acc[1]);
                acc[2] = __ffma2_rn(C, p2c, acc[2]);
                acc[3] = __ffma2_rn(S, p2s, acc[3]);
            }
        }
        if constexpr (!F && p0col(K) >= 16 * G && p0col(K) < 16 * G + 16) p0 = a[p0col(K) - 16 * G];
        velocity_groups<K, F, H, G + 1>(t_row, src, N0, p0, acc);
    }
}

template <int K, bool F, bool H, typename Src>
__device__ __forceinline__ void velocity_stream(uint32_t t_row, Src& src, const float* N0, float p0_in, float inv_s,
                                                float& v1, float& v2)
{
    float2 acc[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float p0 = p0_in;
    velocity_groups<K, F, H, 0>(t_row, src, N0, p0, acc);
    const float v1c = acc[0].x + acc[0].y, v1s = acc[1].x + acc[1].y;
    const float v2c = acc[2].x + acc[2].y, v2s = acc[3].x + acc[3].y;
    if constexpr (H) {
        if constexpr (F) v1 = p0 + inv_s * (v1c + v1s);  // N0 carries the scale of W
        else v1 = inv_s * (p0 + (v1c + v1s));
        v2 = inv_s * (v2c + v2s);
    } else {
        v1 = p0 + (v1c + v1s);
        v2 = v2c + v2s;
    }
}

// One Euler step's product, issued by one thread: P = A_hi W_hi + A_lo W_hi +
// A_hi W_lo over the KS k-steps, then a commit to the step's mbarrier.
// The three products of one 128-row particle tile (descriptors ah, al) with
// the coefficient tiles (bh, bl) into the accumulator at tmem, no commit.
template <int K, bool F = false, bool H = false>
__device__ __forceinline__ void issue_tile_mma(uint32_t tmem, uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl)
{
    using S = Shape<K, F, H>;
    if constexpr (H) {
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_f16<S::NP>(tmem, ah + kKStep * k, bh + kKStep * k, k > 0 ? 1u : 0u);
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_f16<S::NP>(tmem, al + kKStep * k, bh + kKStep * k, 1u);
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_f16<S::NP>(tmem, ah + kKStep * k, bl + kKStep * k, 1u);
    } else {
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_tf32<S::NP>(tmem, ah + kKStep * k, bh + kKStep * k, k > 0 ? 1u : 0u);
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_tf32<S::NP>(tmem, al + kKStep * k, bh + kKStep * k, 1u);
#pragma unroll
        for (int k = 0; k < S::KS; ++k) mma_tf32<S::NP>(tmem, ah + kKStep * k, bl + kKStep * k, 1u);
    }
}

// One Euler step's product for a CTA with one particle tile, issued by one
// thread, then a commit to the step's mbarrier.
template <int K, bool F = false, bool H = false>
__device__ __forceinline__ void issue_step_mma(uint32_t tmem, uint32_t sb, uint32_t bar)
{
    using S = Shape<K, F, H>;
    const uint64_t ah = tile_desc<S::SBO>(sb), al = tile_desc<S::SBO>(sb + S::A_BYTES);
    const uint64_t bh = tile_desc<S::SBO>(sb + 2 * S::A_BYTES), bl = tile_desc<S::SBO>(sb + 2 * S::A_BYTES + S::B_BYTES);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    issue_tile_mma<K, F, H>(tmem, ah, al, bh, bl);
    tc::mma_commit(bar);
}

// The time-dependent kernel streams the x1 harmonics (HarmStream), which keeps
// it within 64 registers and 8 CTAs per SM where shared memory allows (K = 10:
// 26.7 ms; computing them during the product at 6 CTAs per SM measured slower
// at every K, e.g. 20.1 against 19.9 ms at K = 4 and 27.1 against 25.9 at K = 8).

// Shared memory, threads and tensor-memory columns of the time-dependent kernel.
template <int K>
struct TdLaunch {
    using S = TdShape<K>;
    static constexpr int SETS = td_sets<K>();
    static constexpr int THREADS = 128 * SETS;
    static constexpr int SMEM = SETS == 1 ? S::SMEM : 2 * SETS * S::A_BYTES + 2 * S::B_BYTES + 128 + 64;
    static constexpr uint32_t TMEM_COLS = SETS == 1 ? S::TMEM_COLS : 512u;  // set s at column 256 s
    static constexpr int MIN_CTAS = SETS == 1 ? S::MIN_CTAS : 1;
    static_assert(SETS == 1 || (S::NP <= 256 && SMEM + 1024 <= 233472), "two tiles fit");
};

// LIMIT: the per-step MMA wait takes the launch's poll limit (a test lowered
// it, pm_set_wait_limit); otherwise the compile-time full bound, with no
// per-step test of the setting.
template <int K, bool LIMIT = false>
__global__ void __launch_bounds__(TdLaunch<K>::THREADS, TdLaunch<K>::MIN_CTAS)
    timedep_tc_kernel(const __grid_constant__ Params<K> p)
{
    using S = TdShape<K>;
    using LC = TdLaunch<K>;
    constexpr bool F = S::FOLD;
    constexpr bool H = S::HALF;
    constexpr int SETS = LC::SETS, ROWS = LC::THREADS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    // A tiles of ROWS rows (set s = rows 128 s .. 128 s + 127), then W's tiles.
    uint8_t* A_hi = smem;
    uint8_t* A_lo = smem + SETS * S::A_BYTES;
    uint8_t* B_hi = smem + 2 * SETS * S::A_BYTES;
    uint8_t* B_lo = B_hi + S::B_BYTES;
    uint64_t* bar = (uint64_t*)(B_lo + S::B_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar_a = tc::smem_u32(bar);

    // Coefficient tiles (hi / lo) and zero padding of the particle tiles.
    if constexpr (S::W_PARAM) stage_B<S>(B_hi, B_lo, tid, [&](int q) { return p.W[q]; });
    else stage_B<S>(B_hi, B_lo, tid, [&](int q) { return __ldg(p.Wg + q); });
    for (int c = 0; c < S::KC; ++c) {
        *reinterpret_cast<float4*>(A_hi + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(A_lo + tile_off<S::KC>(tid, c)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (tid == 0) {
        tc::mbar_init(bar_a, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                     "r"(LC::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // warp w reads TMEM lanes 32 (w mod 4) of its set's accumulator (columns 256 s)
    const uint32_t t_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 256);

    const uint32_t row = tile_off<S::KC>(tid, 0);
    const uint32_t sb = tc::smem_u32(A_hi);  // A_hi, A_lo, B_hi, B_lo back to back
    const int slot = blockIdx.x / p.chunks;
    const int cidx = blockIdx.x - slot * p.chunks;
    // The observations this grid row serves: a group at one point x whose
    // members (sorted by step count) share the paths, or one observation.
    int m0, m1, stream;
    if (p.groups) {
        const int4 G = p.groups[slot];
        m0 = G.x;
        m1 = G.y;
        stream = G.z;
    } else {
        stream = p.order ? p.order[slot] : slot;
        m0 = stream;
        m1 = stream + 1;
    }
    auto member = [&](int m) { return p.groups ? p.members[m] : m; };
    const int64_t i = (int64_t)cidx * ROWS + tid;
    const bool active = i < p.M;
    Coord<float> X1, X2;
    {
        const ObsRec o = p.obs[member(m0)];
        X1.set(o.x1);
        X2.set(o.x2);
    }
    const uint32_t pid = (uint32_t)(p.path_offset + (active ? i : 0));
    // Member m's path ends at (Y1, Y2): theta0, per-path outputs, and the CTA's
    // (sum, sum of squares) for that observation.  Uniform over the CTA.
    auto finish = [&](int m, const Coord<float>& Y1, const Coord<float>& Y2, bool ok) {
        const int jm = member(m);
        double g = 0.0;
        if (ok && active) {
            g = theta0_eval(p.th, Y1, Y2);
            const int64_t w = (int64_t)jm * p.M + i;
            if (p.g_out) p.g_out[w] = g;
            if (p.x_out) { p.x_out[2 * w] = Y1.full(); p.x_out[2 * w + 1] = Y2.full(); }
        }
        const double2 sum = block_sum2<ROWS>(g, g * g);
        if (tid == 0) p.part[(int64_t)jm * p.chunks + cidx] = sum;
        __syncthreads();  // block_sum2's scratch is reused by the next member
    };
    auto steps_of = [&](int m) { return m < m1 ? p.obs[member(m)].nsteps : -1; };
    int m = m0;  // next member to finish
    while (steps_of(m) == 0) finish(m++, X1, X2, true);
    const int N = m < m1 ? steps_of(m1 - 1) : 0;
    int stop = steps_of(m) - 1;  // the step at which member m takes its last step
    bool failed = false;
    int n = 0;  // the step; after the loop, n - 1 is the last step whose product was issued
    float2 z1 = make_float2(0.f, 0.f), z2 = z1;  // the normals of the even step (.x) and the next (.y)

    for (; n < N; ++n) {
        // sin and cos of 2 pi x of both coordinates, then the row of A: x2
        // harmonics (hi and lo); folded: the m = 0 part of v1 here.
        float2 sx, cx;
        sincos_turns2(make_float2(X1.val(), X2.val()), sx, cx);
        const float p0 = write_row_stream<K, F, H>(sb + row, (uint32_t)(SETS * S::A_BYTES), sx.y, cx.y, p.T0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // One barrier per step: the rows are in place, and a wait that gave up
        // in the previous step (any thread) ends the loop for the whole CTA.
        if (__syncthreads_or(failed)) { failed = true; break; }
        if (tid == 0) {
            if constexpr (SETS == 1) {
                issue_step_mma<K, F, H>(tmem, sb, bar_a);
            } else {
                const uint32_t b0 = sb + 2 * SETS * S::A_BYTES;
                const uint64_t bh = tile_desc<S::SBO>(b0), bl = tile_desc<S::SBO>(b0 + S::B_BYTES);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int st = 0; st < SETS; ++st) {
                    const uint32_t a0 = sb + st * S::A_BYTES;
                    issue_tile_mma<K, F, H>(tmem + 256u * st, tile_desc<S::SBO>(a0),
                                            tile_desc<S::SBO>(a0 + SETS * S::A_BYTES), bh, bl);
                }
                tc::mma_commit(bar_a);
            }
        }
        // While the product runs: the Brownian increment and the x1 harmonics.
        if ((n & 1) == 0) {
            const u32x4 r = philox4x32_10_rk(u32x4{(uint32_t)(n >> 1), pid, (uint32_t)stream, p.inst}, p.rk);
            box_muller2(r.x, r.y, r.z, r.w, z1, z2);
        }
        const float xi1 = (n & 1) ? z1.y : z1.x, xi2 = (n & 1) ? z2.y : z2.x;
        HarmStream h1;
        h1.init(sx.x, cx.x);
        // (the full bound unless a test lowered it: the common path keeps the
        // compile-time bound)
        if constexpr (LIMIT) failed = !tc::mbar_wait(bar_a, (uint32_t)(n & 1), p.wait_limit);
        else failed = !tc::mbar_wait(bar_a, (uint32_t)(n & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float v1, v2;
        velocity_stream<K, F, H>(t_row, h1, p.N0, p0, p.inv_s, v1, v2);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // Members whose last step is this one take it with their own length.
        while (n == stop) {
            const ObsRec o = p.obs[member(m)];
            const float hh = (float)o.h_last, ss = (float)o.s_last;
            Coord<float> Y1 = X1, Y2 = X2;
            em_update2(Y1, Y2, v1, v2, hh, ss, xi1, xi2);
            Y1.wrap();
            Y2.wrap();
            finish(m++, Y1, Y2, true);
            stop = steps_of(m) - 1;
        }
        if (n + 1 < N) {
            em_update2(X1, X2, v1, v2, p.dt, p.s_dt, xi1, xi2);
            // Periodic wrap after every 32nd step (wrap_due): the harmonics
            // of x and x - 1 are the same bits (sincos_turns2 reduces x
            // exactly), so between wraps a position may stand a few steps
            // outside [0, 1); a path's last step always wraps.
            if (wrap_due(n)) {
                X1.wrap();
                X2.wrap();
            }
        }
    }
    failed = __syncthreads_or(failed);
    if (failed && tid == 0) atomicExch(p.err, 1u);
    while (m < m1) finish(m++, X1, X2, false);  // only after a failed wait
    // No product may still write tensor memory when it is freed: after a wait
    // that gave up, wait (full bound) for the last one issued.
    if (failed && n > 0) tc::mbar_wait(bar_a, (uint32_t)((n - 1) & 1));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(LC::TMEM_COLS) : "memory");
    }
}

// W^T of the product-basis table t[(m (K+1) + n) 8 + q] (e0..e3, f0..f3).
template <int K, bool F = false, bool H = false>
void build_W(const double* t, float* W)
{
    using S = Shape<K, F, H>;
    for (int q = 0; q < S::NP * S::WS; ++q) W[q] = 0.f;
    auto T = [&](int m, int n, int q) { return t[(size_t)(m * (K + 1) + n) * 8 + q]; };
    auto set = [&](int col, int row, double v) { W[col * S::WS + row] = (float)v; };
    // A columns: S2_n at acol_s(n), C2_n at acol_c(n), the constant at 2K (unfolded).
    for (int m = 1; m <= K; ++m) {
        const int c1c = pcol<F>(m, 0), c1s = pcol<F>(m, 1), c2c = pcol<F>(m, 2), c2s = pcol<F>(m, 3);
        for (int n = 1; n <= K; ++n) {
            set(c1c, acol_s(n), T(m, n, 0)); set(c1c, acol_c(n), T(m, n, 1));
            set(c1s, acol_s(n), T(m, n, 2)); set(c1s, acol_c(n), T(m, n, 3));
            set(c2c, acol_c(n), T(m, n, 4)); set(c2c, acol_s(n), T(m, n, 5));
            set(c2s, acol_c(n), T(m, n, 6)); set(c2s, acol_s(n), T(m, n, 7));
        }
        if constexpr (!F) {
            set(c2c, 2 * K, T(m, 0, 4));
            set(c2s, 2 * K, T(m, 0, 6));
        }
    }
    if constexpr (!F) {
        for (int n = 1; n <= K; ++n) {  // m = 0: v1 only, accumulator column 4K
            set(p0col(K), acol_s(n), T(0, n, 0));
            set(p0col(K), acol_c(n), T(0, n, 1));
        }
    }
}

template <int K>
cudaError_t launch_timedep_tc(const TimedepLaunch& L, unsigned* err, cudaStream_t stream)
{
    using S = TdShape<K>;
    Params<K> p;
    p.Wg = nullptr;
    {
        auto T = [&](int m, int n, int q) { return L.coef[(size_t)(m * (K + 1) + n) * 8 + q]; };
        for (int n = 1; n <= K; ++n) {
            p.T0[n - 1] = (float)T(0, n, 0);      // multiplies S2_n
            p.T0[K + n - 1] = (float)T(0, n, 1);  // multiplies C2_n
            p.N0[n - 1] = (float)T(n, 0, 4);      // n = 0 term of P2c(m = n)
            p.N0[K + n - 1] = (float)T(n, 0, 6);  // n = 0 term of P2s(m = n)
        }
    }
    // FP16 operands: W (and the n = 0 terms that join its columns) times 2^e,
    // with the largest entry in [2^13, 2^14), far inside FP16's range.
    std::vector<float> Wv((size_t)(S::NP * S::WS));
    build_W<K, S::FOLD, S::HALF>(L.coef, Wv.data());
    p.inv_s = scale_W_host<S>(Wv.data(), p.N0, S::FOLD ? 2 * K : 0);
    if constexpr (S::W_PARAM) {
        for (size_t q = 0; q < Wv.size(); ++q) p.W[q] = Wv[q];
    } else {
        // Into the caller's device buffer (the host vector is read before the
        // copy call returns).
        if (!L.table_dev) return cudaErrorInvalidValue;
        std::vector<float>& W = Wv;
        const cudaError_t e = cudaMemcpyAsync(L.table_dev, W.data(), W.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        p.Wg = L.table_dev;
    }
    p.th.n = L.nq;
    for (int q = 0; q < kMaxTheta0; ++q) {
        const bool on = q < L.nq;
        p.th.k1[q] = on ? L.qk[2 * q] : 0;
        p.th.k2[q] = on ? L.qk[2 * q + 1] : 0;
        p.th.a[q] = on ? (float)L.qa[q] : 0.f;
        p.th.b[q] = on ? (float)L.qb[q] : 0.f;
    }
    p.obs = L.obs;
    p.order = L.order;
    p.part = L.part;
    p.g_out = L.g_out;
    p.x_out = L.x_out;
    p.dt = (float)L.dt;
    p.s_dt = (float)L.s_dt;
    p.M = L.M;
    p.path_offset = L.path_offset;
    p.n_obs = L.n_obs;
    p.chunks = L.chunks;
    p.inst = L.inst;
    p.key0 = L.key0;
    p.key1 = L.key1;
    round_keys(L.key0, L.key1, p.rk);
    p.err = err;
    p.wait_limit = L.wait_limit;
    p.groups = L.groups;
    p.members = L.members;
    using LC = TdLaunch<K>;
    const bool limited = L.wait_limit < tc::kWaitLimit;
    cudaError_t e = cudaFuncSetAttribute(limited ? timedep_tc_kernel<K, true> : timedep_tc_kernel<K, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, LC::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)(L.groups ? L.n_groups : L.n_obs) * L.chunks;
    if (limited) timedep_tc_kernel<K, true><<<(unsigned)grid, LC::THREADS, LC::SMEM, stream>>>(p);
    else timedep_tc_kernel<K, false><<<(unsigned)grid, LC::THREADS, LC::SMEM, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace tdtc
}  // namespace pm

#define PM_INSTANTIATE_TC(K) \
    template cudaError_t pm::tdtc::launch_timedep_tc<K>(const pm::TimedepLaunch&, unsigned*, cudaStream_t);
