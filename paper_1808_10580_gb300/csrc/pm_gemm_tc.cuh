// pm_gemm_tc.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) for
// the surrogate network:  C[M x N] = A[M x K] . B[N x K]^T, both operands
// K-major BF16, FP32 accumulation in tensor memory, fused epilogue.
//
// One CTA computes a 128 x BN tile (BN = 64 or 256) with 4 warps:
//   warp 0 / lane 0  TMA producer: 128B-swizzled 128x64 (A) and BNx64 (B) tiles
//                    into a 4-stage shared-memory ring (mbarrier expect-tx);
//   warp 1 / lane 0  MMA issuer: four tcgen05.mma (K = 16 each) per stage into a
//                    128 x BN FP32 accumulator in TMEM; tcgen05.commit frees the
//                    stage, and a final commit signals the epilogue;
//   warps 0-3        epilogue: tcgen05.ld of rows 32w..32w+31, bias / ReLU /
//                    ReLU-mask, BF16 row-major, BF16 transposed and FP32 stores.
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// flag, skips its remaining work, frees its TMEM and returns.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pm_launch.h"

namespace pm {
namespace tc {

constexpr int BM = 128, BN = 64, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;            // 16 KB
constexpr int B_BYTES = BN * BK * 2;            // 8 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // 24 KB (a multiple of 1024)
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 64;

// Tile width N of one CTA: 64 (many small tiles: the network's shapes) or 256
// (large products: four times the reuse of each A tile, one CTA per SM).
template <int BN_>
struct GemmCfg {
    static constexpr int BN = BN_;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr uint32_t TMEM_COLS = (uint32_t)BN;
    // Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
    // K-major, N = BN, M = BM.
    static constexpr uint32_t IDESC =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    static_assert(BN % 16 == 0 && BN <= 256, "MMA N");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};
constexpr uint32_t kWaitLimit = kWaitPolls;     // bounded spins (a few seconds at most)

struct Epilogue {
    const float* bias;           // [N] or nullptr
    int relu;                    // max(0, .)
    const __nv_bfloat16* mask;   // multiply by (mask[row][col] > 0), or nullptr
    int ld_mask;
    __nv_bfloat16* out_bf16;     // row-major [M][ld_out] or nullptr
    int ld_out;
    __nv_bfloat16* out_bf16_t;   // transposed [N][ld_out_t] or nullptr
    int ld_out_t;
    float* out_f32;              // row-major [M][ld_f32] or nullptr
    int ld_f32;
    int M_valid, N_valid;        // rows/columns beyond these are stored as 0
};

struct GemmParams {  // aligned as its tensor maps require
    CUtensorMap tmA;             // A: [M][K] BF16, box {64, 128}, 128B swizzle
    CUtensorMap tmB;             // B: [N][K] BF16, box {64, BN}, 128B swizzle
    Epilogue ep;
    int M, N, K;
    unsigned* err;               // set to 1 when a bounded wait expires
    uint32_t wait_limit;         // polls of a progress wait (kWaitLimit unless a test lowers it)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the completion of the phase with the given parity: at
// most `limit` polls (0: give up without polling).  Waits that drain a
// CTA's own copies and products before it frees tensor memory and exits
// always take the full bound kWaitLimit; the waits that make progress take
// the launch's limit, which a test may lower (pm_set_wait_limit).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit = kWaitLimit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzling:
// rows of 64 BF16 (128 B), 8-row groups 1024 B apart, tile base 1024-aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                     // leading-dimension byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride-dimension byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    // (the wait is in the same statement: the outputs are valid when it ends)
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// The GEMM kernel itself is compiled in one translation unit only (pm_mlp.cu
// defines PM_DEFINE_GEMM_KERNEL); other users of this header take the helpers.
#ifdef PM_DEFINE_GEMM_KERNEL
template <int BN_>
__global__ void __launch_bounds__(128, 1) gemm_bf16_tc_kernel(const __grid_constant__ GemmParams p)
{
    using G = GemmCfg<BN_>;
    constexpr int BN = G::BN, STAGE_BYTES = G::STAGE_BYTES;
    constexpr uint32_t TMEM_COLS = G::TMEM_COLS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 1);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), accum = smem_u32(bars + 2 * STAGES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int num_k = p.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // Producer.
        int issued = 0;
        for (int kt = 0; kt < num_k; ++kt) {
            const int s = kt % STAGES;
            const uint32_t use = (uint32_t)(kt / STAGES);
            if (kt >= STAGES && !mbar_wait(empty0 + 8 * s, (use & 1u) ^ 1u, p.wait_limit)) { atomicExch(p.err, 1u); break; }
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
            mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
            tma_load_2d(sa, &p.tmA, kt * BK, m0, full0 + 8 * s);
            tma_load_2d(sb, &p.tmB, kt * BK, n0, full0 + 8 * s);
            ++issued;
        }
        // No copy may still be writing this CTA's shared memory when it exits:
        // wait (bounded) for the last fill of every stage that was used.
        for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
            mbar_wait(full0 + 8 * (kt % STAGES), (uint32_t)(kt / STAGES) & 1u);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer.
        for (int kt = 0; kt < num_k; ++kt) {
            const int s = kt % STAGES;
            if (!mbar_wait(full0 + 8 * s, (uint32_t)(kt / STAGES) & 1u, p.wait_limit)) { atomicExch(p.err, 1u); break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * STAGE_BYTES), sb = sa + A_BYTES;
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sb);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)  // K = 16 per instruction: advance 32 bytes within the swizzled row
                mma_bf16(tmem, da + 2 * k, db + 2 * k, G::IDESC, (kt > 0 || k > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(accum);  // fires when every MMA issued above has completed
    }
    __syncwarp();

    // Epilogue: warp w reads accumulator lanes (rows) 32w .. 32w+31.
    const bool ok = mbar_wait(accum, 0, p.wait_limit);
    if (!ok) {
        if (lane == 0) atomicExch(p.err, 1u);
        // The issuer commits `accum` on every path, after its last product:
        // wait for it (full bound) so that no product still writes tensor
        // memory when it is freed below.
        mbar_wait(accum, 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && *(volatile unsigned*)p.err == 0u) {
        const Epilogue& e = p.ep;
        const int row = m0 + warp * 32 + lane;
        const bool row_ok = row < e.M_valid;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int col0 = n0 + c0;
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int col = col0 + q;
                float x = v[q];
                if (e.bias) x += e.bias[col];
                if (e.relu) x = fmaxf(x, 0.0f);
                if (e.mask && !(__bfloat162float(e.mask[(size_t)row * e.ld_mask + col]) > 0.0f)) x = 0.0f;
                if (!row_ok || col >= e.N_valid) x = 0.0f;
                v[q] = x;
            }
            if (e.out_f32) {
                float4* dst = reinterpret_cast<float4*>(e.out_f32 + (size_t)row * e.ld_f32 + col0);
#pragma unroll
                for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            if (e.out_bf16) {
                __nv_bfloat162* dst = reinterpret_cast<__nv_bfloat162*>(e.out_bf16 + (size_t)row * e.ld_out + col0);
#pragma unroll
                for (int q = 0; q < 16; ++q) dst[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            }
            if (e.out_bf16_t) {
#pragma unroll
                for (int q = 0; q < 32; ++q) e.out_bf16_t[(size_t)(col0 + q) * e.ld_out_t + row] = __float2bfloat16_rn(v[q]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}
#endif  // PM_DEFINE_GEMM_KERNEL

}  // namespace tc
}  // namespace pm
