// pm_mlp.cu -- the learned surrogate u -> G(u): a 3-layer ReLU network trained
// and evaluated on the GPU with the tcgen05 BF16 GEMM (pm_gemm_tc.cuh).
//
// Layout.  Weights are stored [out][in] with in and out padded to multiples of
// 64 (the padding stays exactly zero).  The FP32 master copy of all parameters
// (W1, b1, W2, b2, W3, b3) is one contiguous buffer, and so are their
// gradients and the two Adam moments, so one kernel updates everything.
// After each update the weights are cast to BF16 twice: row-major (operand B
// of the forward GEMMs) and transposed (operand B of the backward data GEMMs).
// Activations of a batch are kept as BF16 row-major and BF16 transposed (the
// operands of the weight-gradient GEMMs, which contract over the batch).
//
// One training step on a batch of B rows (padded to Bp, a multiple of 128):
//   F1  H1 = relu(U W1^T + b1)      F2  H2 = relu(H1 W2^T + b2)      F3  Y = H2 W3^T + b3
//   loss: dY = (Y - T) / (B n_out),  L = sum (Y - T)^2 / (2 B n_out)
//   gW3 = dY^T H2                   dH2 = (dY W3) * [H2 > 0]
//   gW2 = dH2^T H1                  dH1 = (dH2 W2) * [H1 > 0]
//   gW1 = dH1^T U                   gb_l = column sums of dH_l (fixed order)
//   Adam (Kingma & Ba 2015) on the FP32 master copy, then BF16 casts.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pm.h"
#define PM_DEFINE_GEMM_KERNEL
#include "pm_gemm_tc.cuh"
#include "pm_internal.h"

using namespace pm;
using bf16 = __nv_bfloat16;

namespace {

// ---------------------------------------------------------------------------
// Tensor maps (the CUDA driver API's encoder, fetched once through the runtime)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

int get_encoder()
{
    if (g_encode) return PM_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(PM_ECUDA, "cuTensorMapEncodeTiled is not available");
    g_encode = (EncodeTiledFn)fn;
    return PM_OK;
}

// Row-major BF16 matrix [rows][ld] (cols used), tiles of box_rows x 64.
bool make_map(CUtensorMap* m, const bf16* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows)
{
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {ld * sizeof(bf16)};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t es[2] = {1, 1};
    return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

tc::Epilogue no_epilogue(int M, int N)
{
    tc::Epilogue e;
    memset(&e, 0, sizeof e);
    e.M_valid = M;
    e.N_valid = N;
    return e;
}

// C = A B^T with A [M][K] (ld lda), B [N][K] (ld ldb): M % 128, N % 64, K % 64 == 0.
int gemm(pm_ctx* c, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, const tc::Epilogue& ep,
         unsigned* err, uint32_t wait_limit = kWaitPolls)
{
    if (M % tc::BM || N % tc::BN || K % tc::BK || M <= 0 || N <= 0 || K <= 0)
        return fail(PM_EINVAL, "gemm shape %d x %d x %d is not a multiple of 128 x 64 x 64", M, N, K);
    if ((lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16))
        return fail(PM_EINVAL, "gemm operands must be 16-byte aligned with row pitch a multiple of 8");
    int rc = get_encoder();
    if (rc) return rc;
    tc::GemmParams p;
    memset(&p, 0, sizeof p);
    if (!make_map(&p.tmA, A, (uint64_t)M, (uint64_t)K, (uint64_t)lda, tc::BM) ||
        !make_map(&p.tmB, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, tc::BN))
        return fail(PM_ECUDA, "tensor map encoding failed");
    p.ep = ep;
    p.M = M;
    p.N = N;
    p.K = K;
    p.err = err;
    p.wait_limit = wait_limit;
    // 256-wide tiles when the product has enough of them for two waves over the
    // SMs; otherwise 64-wide tiles (more CTAs for the network's small shapes).
    const bool wide = (N % 256 == 0) && (int64_t)(M / tc::BM) * (N / 256) >= 2 * (int64_t)c->sm_count;
    if (wide && !make_map(&p.tmB, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, 256))
        return fail(PM_ECUDA, "tensor map encoding failed");
    static bool attr_set[2][64] = {};
    if (!attr_set[wide][c->device & 63]) {
        if (wide)
            PM_CUDA(cudaFuncSetAttribute(tc::gemm_bf16_tc_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::GemmCfg<256>::SMEM_BYTES),
                    "gemm smem attribute");
        else
            PM_CUDA(cudaFuncSetAttribute(tc::gemm_bf16_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::GemmCfg<64>::SMEM_BYTES),
                    "gemm smem attribute");
        attr_set[wide][c->device & 63] = true;
    }
    if (wide) {
        dim3 grid((unsigned)(M / tc::BM), (unsigned)(N / 256));
        tc::gemm_bf16_tc_kernel<256><<<grid, 128, tc::GemmCfg<256>::SMEM_BYTES, c->stream>>>(p);
    } else {
        dim3 grid((unsigned)(M / tc::BM), (unsigned)(N / tc::BN));
        tc::gemm_bf16_tc_kernel<64><<<grid, 128, tc::GemmCfg<64>::SMEM_BYTES, c->stream>>>(p);
    }
    PM_CUDA(cudaGetLastError(), "gemm launch");
    count_launch(c);
    return PM_OK;
}

int pad64(int v) { return (v + 63) / 64 * 64; }
int pad128(int v) { return (v + 127) / 128 * 128; }

// ---------------------------------------------------------------------------
// Element-wise kernels
// ---------------------------------------------------------------------------

// Batch rows perm[b] (b < B) of U [*, n_in] and T [*, n_out] -> BF16 Ub [Bp][Kin],
// its transpose Ut [Kin][Bp], and FP32 targets Tb [Bp][Nout]; zero padding.
__global__ void gather_batch_kernel(const float* __restrict__ U, const float* __restrict__ T,
                                    const int64_t* __restrict__ perm, int64_t off, int B, int Bp, int n_in, int Kin,
                                    int n_out, int Nout, bf16* __restrict__ Ub, bf16* __restrict__ Ut,
                                    float* __restrict__ Tb)
{
    const int b = blockIdx.x;
    const bool live = b < B;
    const int64_t r = live ? (perm ? perm[off + b] : off + b) : 0;
    for (int cidx = threadIdx.x; cidx < Kin; cidx += blockDim.x) {
        const float v = (live && cidx < n_in) ? U[r * n_in + cidx] : 0.0f;
        const bf16 h = __float2bfloat16_rn(v);
        Ub[(size_t)b * Kin + cidx] = h;
        Ut[(size_t)cidx * Bp + b] = h;
    }
    if (Tb)
        for (int o = threadIdx.x; o < Nout; o += blockDim.x) Tb[(size_t)b * Nout + o] = (live && o < n_out) ? T[r * n_out + o] : 0.0f;
}

// dY = (Y - T) / (B n_out) on the live block, 0 elsewhere; per-row loss partials.
__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ Tb, int B, int Bp, int n_out,
                            int Nout, bf16* __restrict__ dYb, bf16* __restrict__ dYt, float* __restrict__ dYf,
                            double* __restrict__ row_loss)
{
    const int b = blockIdx.x;
    const double scale = 1.0 / ((double)B * n_out);
    double acc = 0.0;
    for (int o = threadIdx.x; o < Nout; o += blockDim.x) {
        float g = 0.0f;
        if (b < B && o < n_out) {
            const double d = (double)Y[(size_t)b * Nout + o] - (double)Tb[(size_t)b * Nout + o];
            acc += d * d;
            g = (float)(d * scale);
        }
        dYf[(size_t)b * Nout + o] = g;
        const bf16 h = __float2bfloat16_rn(g);
        dYb[(size_t)b * Nout + o] = h;
        dYt[(size_t)o * Bp + b] = h;
    }
    __shared__ double red[128];
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
        row_loss[b] = s * 0.5 * scale;
    }
}

// A given output cotangent dY [B][n_out] (FP32) -> BF16 dYb [Bp][Nout], zero padding.
__global__ void set_cotangent_kernel(const float* __restrict__ dY, int B, int n_out, int Nout, bf16* __restrict__ dYb)
{
    const int b = blockIdx.x;
    for (int o = threadIdx.x; o < Nout; o += blockDim.x)
        dYb[(size_t)b * Nout + o] = __float2bfloat16_rn((b < B && o < n_out) ? dY[(size_t)b * n_out + o] : 0.0f);
}

__global__ void sum_rows_kernel(const double* __restrict__ v, int n, float* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += v[k];
        *out = (float)s;
    }
}

// Column sums (bias gradients), rows in order: one thread per column.
__global__ void colsum_kernel(const float* __restrict__ X, int rows, int cols, int ld, float* __restrict__ out)
{
    const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (cidx >= cols) return;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += X[(size_t)r * ld + cidx];
    out[cidx] = (float)s;
}

// Adam on the whole parameter buffer, with decoupled weight decay (AdamW,
// Loshchilov & Hutter 2019) on the weight matrices; the three bias ranges
// [bo_k, bo_k + bn_k) are not decayed.
struct BiasRanges { int64_t o[3], n[3]; };

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float wd, BiasRanges br)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float g = G[q];
    const float mq = b1 * m[q] + (1.0f - b1) * g;
    const float vq = b2 * v[q] + (1.0f - b2) * g * g;
    m[q] = mq;
    v[q] = vq;
    const float mh = mq / c1, vh = vq / c2;
    bool bias = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) bias = bias || (q >= br.o[k] && q < br.o[k] + br.n[k]);
    const float p = P[q];
    P[q] = p - lr * (mh / (sqrtf(vh) + eps) + (bias ? 0.0f : wd * p));
}

// FP32 [rows][cols] -> BF16 row-major and transposed copies.
__global__ void cast_kernel(const float* __restrict__ W, int rows, int cols, bf16* __restrict__ Wb,
                            bf16* __restrict__ Wt)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)rows * cols) return;
    const int r = (int)(q / cols), cidx = (int)(q % cols);
    const bf16 h = __float2bfloat16_rn(W[q]);
    Wb[q] = h;
    Wt[(size_t)cidx * rows + r] = h;
}

}  // namespace

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
struct pm_mlp {
    int n_in = 0, H = 0, n_out = 0, Kin = 0, Nout = 0;
    int device = 0;
    int64_t P = 0;                    // parameter count of the padded layout
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float* params = nullptr;          // FP32 master [P]
    float* grads = nullptr;           // [P]
    float* m = nullptr;               // Adam moments [P]
    float* v = nullptr;
    int64_t step = 0;
    bf16 *W1b = nullptr, *W1t = nullptr, *W2b = nullptr, *W2t = nullptr, *W3b = nullptr, *W3t = nullptr;
    // batch workspace (capacity Bcap rows)
    int Bcap = 0;
    void* act = nullptr;
    bf16 *Ub, *Ut, *H1, *H1t, *H2, *H2t, *dYb, *dYt, *dH2b, *dH2t, *dH1b, *dH1t;
    float *Y, *Tb, *dYf, *dH2f, *dH1f, *loss;
    double* row_loss;
    unsigned* err;
};

namespace {

void mlp_free_act(pm_mlp* n)
{
    if (n->act) cudaFree(n->act);
    n->act = nullptr;
    n->Bcap = 0;
}

int mlp_reserve(pm_ctx* c, pm_mlp* n, int Bp)
{
    if (Bp <= n->Bcap) return PM_OK;
    PM_CUDA(cudaStreamSynchronize(c->stream), "surrogate resize");
    mlp_free_act(n);
    const int Kin = n->Kin, H = n->H, No = n->Nout;
    Bump b(nullptr);
    auto plan = [&](Bump& bp) {
        n->Ub = bp.take<bf16>((size_t)Bp * Kin); n->Ut = bp.take<bf16>((size_t)Kin * Bp);
        n->H1 = bp.take<bf16>((size_t)Bp * H); n->H1t = bp.take<bf16>((size_t)H * Bp);
        n->H2 = bp.take<bf16>((size_t)Bp * H); n->H2t = bp.take<bf16>((size_t)H * Bp);
        n->dYb = bp.take<bf16>((size_t)Bp * No); n->dYt = bp.take<bf16>((size_t)No * Bp);
        n->dH2b = bp.take<bf16>((size_t)Bp * H); n->dH2t = bp.take<bf16>((size_t)H * Bp);
        n->dH1b = bp.take<bf16>((size_t)Bp * H); n->dH1t = bp.take<bf16>((size_t)H * Bp);
        n->Y = bp.take<float>((size_t)Bp * No); n->Tb = bp.take<float>((size_t)Bp * No);
        n->dYf = bp.take<float>((size_t)Bp * No);
        n->dH2f = bp.take<float>((size_t)Bp * H); n->dH1f = bp.take<float>((size_t)Bp * H);
        n->loss = bp.take<float>(64);
        n->row_loss = bp.take<double>((size_t)Bp);
        n->err = bp.take<unsigned>(64);
    };
    plan(b);
    PM_CUDA(cudaMalloc(&n->act, b.off), "surrogate activations");
    PM_CUDA(cudaMemsetAsync(n->act, 0, b.off, c->stream), "clear activations");
    Bump real(n->act);
    plan(real);
    n->Bcap = Bp;
    return PM_OK;
}

int mlp_cast_weights(pm_ctx* c, pm_mlp* n)
{
    struct { int64_t off; int rows, cols; bf16 *b, *t; } mats[3] = {
        {n->oW1, n->H, n->Kin, n->W1b, n->W1t}, {n->oW2, n->H, n->H, n->W2b, n->W2t}, {n->oW3, n->Nout, n->H, n->W3b, n->W3t}};
    for (auto& mt : mats) {
        const int64_t cnt = (int64_t)mt.rows * mt.cols;
        cast_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, c->stream>>>(n->params + mt.off, mt.rows, mt.cols, mt.b, mt.t);
        PM_CUDA(cudaGetLastError(), "cast kernel");
        count_launch(c);
    }
    return PM_OK;
}

// Forward pass on the gathered batch (Ub already filled); Bp padded rows, B live rows.
int mlp_forward(pm_ctx* c, pm_mlp* n, int B, int Bp)
{
    tc::Epilogue e = no_epilogue(B, n->H);
    e.bias = n->params + n->ob1; e.relu = 1;
    e.out_bf16 = n->H1; e.ld_out = n->H; e.out_bf16_t = n->H1t; e.ld_out_t = Bp;
    int rc = gemm(c, n->Ub, n->Kin, n->W1b, n->Kin, Bp, n->H, n->Kin, e, n->err);
    if (rc) return rc;
    e = no_epilogue(B, n->H);
    e.bias = n->params + n->ob2; e.relu = 1;
    e.out_bf16 = n->H2; e.ld_out = n->H; e.out_bf16_t = n->H2t; e.ld_out_t = Bp;
    if ((rc = gemm(c, n->H1, n->H, n->W2b, n->H, Bp, n->H, n->H, e, n->err))) return rc;
    e = no_epilogue(B, n->n_out);
    e.bias = n->params + n->ob3;
    e.out_f32 = n->Y; e.ld_f32 = n->Nout;
    return gemm(c, n->H2, n->H, n->W3b, n->H, Bp, n->Nout, n->H, e, n->err);
}

// Loss and all gradients into n->grads (after mlp_forward and the targets in Tb).
int mlp_backward(pm_ctx* c, pm_mlp* n, int B, int Bp)
{
    loss_kernel<<<Bp, 128, 0, c->stream>>>(n->Y, n->Tb, B, Bp, n->n_out, n->Nout, n->dYb, n->dYt, n->dYf, n->row_loss);
    PM_CUDA(cudaGetLastError(), "loss kernel");
    sum_rows_kernel<<<1, 32, 0, c->stream>>>(n->row_loss, Bp, n->loss);
    PM_CUDA(cudaGetLastError(), "loss sum");
    count_launch(c, 2);
    float* g = n->grads;
    // gW3 = dY^T H2: [Nout x Bp] x [H x Bp]^T
    tc::Epilogue e = no_epilogue(n->Nout, n->H);
    e.out_f32 = g + n->oW3; e.ld_f32 = n->H;
    int rc = gemm(c, n->dYt, Bp, n->H2t, Bp, n->Nout, n->H, Bp, e, n->err);
    if (rc) return rc;
    // dH2 = (dY W3) * [H2 > 0]: [Bp x Nout] x [H x Nout]^T
    e = no_epilogue(B, n->H);
    e.mask = n->H2; e.ld_mask = n->H;
    e.out_bf16 = n->dH2b; e.ld_out = n->H; e.out_bf16_t = n->dH2t; e.ld_out_t = Bp; e.out_f32 = n->dH2f; e.ld_f32 = n->H;
    if ((rc = gemm(c, n->dYb, n->Nout, n->W3t, n->Nout, Bp, n->H, n->Nout, e, n->err))) return rc;
    // gW2 = dH2^T H1
    e = no_epilogue(n->H, n->H);
    e.out_f32 = g + n->oW2; e.ld_f32 = n->H;
    if ((rc = gemm(c, n->dH2t, Bp, n->H1t, Bp, n->H, n->H, Bp, e, n->err))) return rc;
    // dH1 = (dH2 W2) * [H1 > 0]
    e = no_epilogue(B, n->H);
    e.mask = n->H1; e.ld_mask = n->H;
    e.out_bf16 = n->dH1b; e.ld_out = n->H; e.out_bf16_t = n->dH1t; e.ld_out_t = Bp; e.out_f32 = n->dH1f; e.ld_f32 = n->H;
    if ((rc = gemm(c, n->dH2b, n->H, n->W2t, n->H, Bp, n->H, n->H, e, n->err))) return rc;
    // gW1 = dH1^T U
    e = no_epilogue(n->H, n->Kin);
    e.out_f32 = g + n->oW1; e.ld_f32 = n->Kin;
    if ((rc = gemm(c, n->dH1t, Bp, n->Ut, Bp, n->H, n->Kin, Bp, e, n->err))) return rc;
    // bias gradients
    colsum_kernel<<<(n->Nout + 127) / 128, 128, 0, c->stream>>>(n->dYf, Bp, n->Nout, n->Nout, g + n->ob3);
    colsum_kernel<<<(n->H + 127) / 128, 128, 0, c->stream>>>(n->dH2f, Bp, n->H, n->H, g + n->ob2);
    colsum_kernel<<<(n->H + 127) / 128, 128, 0, c->stream>>>(n->dH1f, Bp, n->H, n->H, g + n->ob1);
    PM_CUDA(cudaGetLastError(), "bias gradients");
    count_launch(c, 3);
    return PM_OK;
}

int check_err(pm_ctx* c, pm_mlp* n)
{
    unsigned e = 0;
    PM_CUDA(cudaMemcpyAsync(&e, n->err, 4, cudaMemcpyDeviceToHost, c->stream), "copy gemm flag");
    PM_CUDA(cudaStreamSynchronize(c->stream), "surrogate");
    if (e) return fail(PM_ETIMEOUT, "a tensor-core GEMM wait timed out");
    return PM_OK;
}

// Copy a host or device FP32 matrix [rows][cols] into the padded parameter slice [rows_pad][cols_pad].
void put_matrix(float* host, int64_t off, const float* src, int rows, int cols, int cols_pad)
{
    for (int r = 0; r < rows; ++r) memcpy(host + off + (int64_t)r * cols_pad, src + (int64_t)r * cols, (size_t)cols * 4);
}

void get_matrix(const float* host, int64_t off, float* dst, int rows, int cols, int cols_pad)
{
    for (int r = 0; r < rows; ++r) memcpy(dst + (int64_t)r * cols, host + off + (int64_t)r * cols_pad, (size_t)cols * 4);
}

uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int pm_surrogate_create(pm_ctx* c, pm_mlp** out, int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed)
{
    if (!c || !out) return fail(PM_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_in < 1 || n_out < 1 || n_hidden < 128 || n_hidden % 128 || n_in > 8192 || n_out > 8192 || n_hidden > 8192)
        return fail(PM_EINVAL, "need 1 <= n_in, n_out <= 8192 and n_hidden a multiple of 128 in [128, 8192]");
    int rc = set_device(c);
    if (rc) return rc;
    pm_mlp* n = new (std::nothrow) pm_mlp;
    if (!n) return fail(PM_ENOMEM, "surrogate object");
    n->n_in = n_in; n->H = n_hidden; n->n_out = n_out; n->Kin = pad64(n_in); n->Nout = pad128(n_out);
    n->device = c->device;
    n->oW1 = 0; n->ob1 = n->oW1 + (int64_t)n->H * n->Kin; n->oW2 = n->ob1 + n->H;
    n->ob2 = n->oW2 + (int64_t)n->H * n->H; n->oW3 = n->ob2 + n->H; n->ob3 = n->oW3 + (int64_t)n->Nout * n->H;
    n->P = n->ob3 + n->Nout;
    const size_t fbytes = (size_t)n->P * 4;
    const size_t wbytes = ((size_t)n->H * n->Kin + (size_t)n->H * n->H + (size_t)n->Nout * n->H) * 2;
    void* buf = nullptr;
    if (cudaMalloc(&buf, 4 * fbytes + 2 * wbytes + 4096) != cudaSuccess) {
        cudaGetLastError();
        delete n;
        return fail(PM_ENOMEM, "surrogate parameters");
    }
    Bump b(buf);
    n->params = b.take<float>((size_t)n->P); n->grads = b.take<float>((size_t)n->P);
    n->m = b.take<float>((size_t)n->P); n->v = b.take<float>((size_t)n->P);
    n->W1b = b.take<bf16>((size_t)n->H * n->Kin); n->W1t = b.take<bf16>((size_t)n->H * n->Kin);
    n->W2b = b.take<bf16>((size_t)n->H * n->H); n->W2t = b.take<bf16>((size_t)n->H * n->H);
    n->W3b = b.take<bf16>((size_t)n->Nout * n->H); n->W3t = b.take<bf16>((size_t)n->Nout * n->H);
    // He-normal initial weights from a seeded generator (SplitMix64 + Box-Muller), zero biases and padding.
    std::vector<float> h((size_t)n->P, 0.0f);
    uint64_t st = seed;
    auto normal = [&]() {
        const double u1 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        const double u2 = ((splitmix(st) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    for (int r = 0; r < n->H; ++r)
        for (int q = 0; q < n_in; ++q) h[(size_t)(n->oW1 + (int64_t)r * n->Kin + q)] = (float)(normal() * std::sqrt(2.0 / n_in));
    for (int r = 0; r < n->H; ++r)
        for (int q = 0; q < n->H; ++q) h[(size_t)(n->oW2 + (int64_t)r * n->H + q)] = (float)(normal() * std::sqrt(2.0 / n->H));
    for (int r = 0; r < n_out; ++r)
        for (int q = 0; q < n->H; ++q) h[(size_t)(n->oW3 + (int64_t)r * n->H + q)] = (float)(normal() * std::sqrt(1.0 / n->H));
    cudaError_t e = cudaMemcpyAsync(n->params, h.data(), fbytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->grads, 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(buf);
        delete n;
        return cuda_fail(e, "surrogate init");
    }
    if ((rc = mlp_cast_weights(c, n))) { cudaFree(buf); delete n; return rc; }
    *out = n;
    return PM_OK;
}

void pm_surrogate_destroy(pm_mlp* n)
{
    if (!n) return;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    mlp_free_act(n);
    if (n->params) cudaFree(n->params);
    delete n;
}

int pm_surrogate_set_params(pm_ctx* c, pm_mlp* n, const float* W1, const float* b1, const float* W2, const float* b2,
                            const float* W3, const float* b3)
{
    if (!c || !n || !W1 || !b1 || !W2 || !b2 || !W3 || !b3) return fail(PM_EINVAL, "NULL argument");
    int rc = set_device(c);
    if (rc) return rc;
    std::vector<float> h((size_t)n->P, 0.0f);
    put_matrix(h.data(), n->oW1, W1, n->H, n->n_in, n->Kin);
    memcpy(h.data() + n->ob1, b1, (size_t)n->H * 4);
    put_matrix(h.data(), n->oW2, W2, n->H, n->H, n->H);
    memcpy(h.data() + n->ob2, b2, (size_t)n->H * 4);
    put_matrix(h.data(), n->oW3, W3, n->n_out, n->H, n->H);
    memcpy(h.data() + n->ob3, b3, (size_t)n->n_out * 4);
    PM_CUDA(cudaMemcpyAsync(n->params, h.data(), (size_t)n->P * 4, cudaMemcpyHostToDevice, c->stream), "set params");
    PM_CUDA(cudaMemsetAsync(n->m, 0, (size_t)n->P * 4, c->stream), "reset moments");
    PM_CUDA(cudaMemsetAsync(n->v, 0, (size_t)n->P * 4, c->stream), "reset moments");
    n->step = 0;
    if ((rc = mlp_cast_weights(c, n))) return rc;
    PM_CUDA(cudaStreamSynchronize(c->stream), "set params");
    return PM_OK;
}

static int copy_params_out(pm_ctx* c, const pm_mlp* n, const float* dev, float* W1, float* b1, float* W2, float* b2,
                           float* W3, float* b3)
{
    std::vector<float> h((size_t)n->P);
    PM_CUDA(cudaMemcpyAsync(h.data(), dev, (size_t)n->P * 4, cudaMemcpyDeviceToHost, c->stream), "get params");
    PM_CUDA(cudaStreamSynchronize(c->stream), "get params");
    if (W1) get_matrix(h.data(), n->oW1, W1, n->H, n->n_in, n->Kin);
    if (b1) memcpy(b1, h.data() + n->ob1, (size_t)n->H * 4);
    if (W2) get_matrix(h.data(), n->oW2, W2, n->H, n->H, n->H);
    if (b2) memcpy(b2, h.data() + n->ob2, (size_t)n->H * 4);
    if (W3) get_matrix(h.data(), n->oW3, W3, n->n_out, n->H, n->H);
    if (b3) memcpy(b3, h.data() + n->ob3, (size_t)n->n_out * 4);
    return PM_OK;
}

int pm_surrogate_get_params(pm_ctx* c, const pm_mlp* n, float* W1, float* b1, float* W2, float* b2, float* W3,
                            float* b3)
{
    if (!c || !n) return fail(PM_EINVAL, "NULL argument");
    int rc = set_device(c);
    if (rc) return rc;
    return copy_params_out(c, n, n->params, W1, b1, W2, b2, W3, b3);
}

int pm_surrogate_gradients(pm_ctx* c, pm_mlp* n, const float* U, const float* T, int64_t B, float* loss, float* gW1,
                           float* gb1, float* gW2, float* gb2, float* gW3, float* gb3)
{
    if (!c || !n || !U || !T) return fail(PM_EINVAL, "NULL argument");
    if (B < 1 || B > (1 << 20)) return fail(PM_EINVAL, "batch size out of range");
    int rc = set_device(c);
    if (rc) return rc;
    const int Bp = (int)((B + 127) / 128 * 128);
    if ((rc = mlp_reserve(c, n, Bp))) return rc;
    // stage the batch through the workspace
    const size_t ub = (size_t)B * n->n_in * 4, tb = (size_t)B * n->n_out * 4;
    if ((rc = ensure_workspace(c, ub + tb + 1024))) return rc;
    float* dU = (float*)c->ws;
    float* dT = (float*)((char*)c->ws + ((ub + 255) & ~(size_t)255));
    PM_CUDA(cudaMemcpyAsync(dU, U, ub, cudaMemcpyHostToDevice, c->stream), "copy U");
    PM_CUDA(cudaMemcpyAsync(dT, T, tb, cudaMemcpyHostToDevice, c->stream), "copy T");
    PM_CUDA(cudaMemsetAsync(n->err, 0, 4, c->stream), "clear flag");
    gather_batch_kernel<<<Bp, 128, 0, c->stream>>>(dU, dT, nullptr, 0, (int)B, Bp, n->n_in, n->Kin, n->n_out, n->Nout,
                                                   n->Ub, n->Ut, n->Tb);
    PM_CUDA(cudaGetLastError(), "gather batch");
    count_launch(c);
    if ((rc = mlp_forward(c, n, (int)B, Bp))) return rc;
    if ((rc = mlp_backward(c, n, (int)B, Bp))) return rc;
    if ((rc = check_err(c, n))) return rc;
    if (loss) PM_CUDA(cudaMemcpy(loss, n->loss, 4, cudaMemcpyDeviceToHost), "copy loss");
    return copy_params_out(c, n, n->grads, gW1, gb1, gW2, gb2, gW3, gb3);
}

int pm_surrogate_train(pm_ctx* c, pm_mlp* n, const float* U, const float* Y, int64_t N, const pm_train_opts* o,
                       uint32_t flags, float* loss_history)
{
    if (!c || !n || !U || !Y || !o) return fail(PM_EINVAL, "NULL argument");
    if (N < 1) return fail(PM_EINVAL, "N < 1");
    if (o->epochs < 1 || o->batch < 1 || o->batch > (1 << 16)) return fail(PM_EINVAL, "bad epochs or batch");
    if (!(o->lr > 0) || !(o->beta1 >= 0 && o->beta1 < 1) || !(o->beta2 >= 0 && o->beta2 < 1) || !(o->eps > 0) ||
        !(o->weight_decay >= 0) || !(o->lr_decay > 0 && o->lr_decay <= 1))
        return fail(PM_EINVAL, "bad Adam settings");
    int rc = set_device(c);
    if (rc) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    if ((rc = check_ptrs(c, flags, {U, Y}))) return rc;
    const int64_t nb = (N + o->batch - 1) / o->batch;
    const int B = (int)std::min<int64_t>(o->batch, N);
    const int Bp = (B + 127) / 128 * 128;
    if ((rc = mlp_reserve(c, n, Bp))) return rc;
    // Device copies of the data (when given on the host) and the permutation.
    const size_t ub = (size_t)N * n->n_in * 4, yb = (size_t)N * n->n_out * 4, pb = (size_t)N * 8;
    Bump probe(nullptr);
    probe.take<char>(dev ? 0 : ub); probe.take<char>(dev ? 0 : yb); probe.take<int64_t>((size_t)N);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    Bump bw(c->ws);
    const float* dU = dev ? U : (float*)bw.take<char>(ub);
    const float* dY = dev ? Y : (float*)bw.take<char>(yb);
    int64_t* dperm = bw.take<int64_t>((size_t)N);
    if (!dev) {
        PM_CUDA(cudaMemcpyAsync((void*)dU, U, ub, cudaMemcpyHostToDevice, c->stream), "copy U");
        PM_CUDA(cudaMemcpyAsync((void*)dY, Y, yb, cudaMemcpyHostToDevice, c->stream), "copy Y");
    }
    std::vector<int64_t> perm((size_t)N);
    for (int64_t i = 0; i < N; ++i) perm[(size_t)i] = i;
    uint64_t st = o->shuffle_seed;
    std::vector<float> step_loss((size_t)nb);
    PM_CUDA(cudaMemsetAsync(n->err, 0, 4, c->stream), "clear flag");
    const BiasRanges br{{n->ob1, n->ob2, n->ob3}, {n->H, n->H, n->Nout}};
    float lr = o->lr;
    for (int ep = 0; ep < o->epochs; ++ep, lr *= o->lr_decay) {
        for (int64_t i = N - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(splitmix(st) % (uint64_t)(i + 1))]);
        PM_CUDA(cudaMemcpyAsync(dperm, perm.data(), pb, cudaMemcpyHostToDevice, c->stream), "copy permutation");
        double ep_loss = 0.0;
        for (int64_t s = 0; s < nb; ++s) {
            const int64_t off = s * o->batch;
            const int Bs = (int)std::min<int64_t>(o->batch, N - off);
            gather_batch_kernel<<<Bp, 128, 0, c->stream>>>(dU, dY, dperm, off, Bs, Bp, n->n_in, n->Kin, n->n_out,
                                                           n->Nout, n->Ub, n->Ut, n->Tb);
            PM_CUDA(cudaGetLastError(), "gather batch");
            count_launch(c);
            if ((rc = mlp_forward(c, n, Bs, Bp))) return rc;
            if ((rc = mlp_backward(c, n, Bs, Bp))) return rc;
            n->step += 1;
            const float c1 = 1.0f - std::pow(o->beta1, (float)n->step), c2 = 1.0f - std::pow(o->beta2, (float)n->step);
            adam_kernel<<<(unsigned)((n->P + 255) / 256), 256, 0, c->stream>>>(n->params, n->grads, n->m, n->v, n->P,
                                                                               lr, o->beta1, o->beta2, o->eps, c1, c2,
                                                                               o->weight_decay, br);
            PM_CUDA(cudaGetLastError(), "adam");
            count_launch(c);
            if ((rc = mlp_cast_weights(c, n))) return rc;
            if (loss_history) {
                PM_CUDA(cudaMemcpyAsync(&step_loss[(size_t)s], n->loss, 4, cudaMemcpyDeviceToHost, c->stream), "copy loss");
            }
        }
        if (loss_history) {
            PM_CUDA(cudaStreamSynchronize(c->stream), "epoch");
            for (int64_t s = 0; s < nb; ++s) ep_loss += step_loss[(size_t)s];
            loss_history[ep] = (float)(ep_loss / (double)nb);
        }
    }
    return check_err(c, n);
}

int pm_surrogate_input_gradient(pm_ctx* c, const pm_mlp* nc, const float* U, const float* dY, int64_t B, float* dU,
                                uint32_t flags)
{
    pm_mlp* n = const_cast<pm_mlp*>(nc);  // the activation workspace is scratch
    if (!c || !n || !U || !dY || !dU) return fail(PM_EINVAL, "NULL argument");
    if (B < 1 || B > (1 << 20)) return fail(PM_EINVAL, "batch size out of range");
    int rc = set_device(c);
    if (rc) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    if ((rc = check_ptrs(c, flags, {U, dY, dU}))) return rc;
    const int Bp = (int)((B + 127) / 128 * 128);
    if ((rc = mlp_reserve(c, n, Bp))) return rc;
    // workspace: the input and cotangent rows (host pointers only), then the FP32 product [Bp][Kin]
    const size_t ub = (size_t)B * n->n_in * 4, yb = (size_t)B * n->n_out * 4;
    Bump probe(nullptr);
    probe.take<char>(dev ? 0 : ub);
    probe.take<char>(dev ? 0 : yb);
    probe.take<float>((size_t)Bp * n->Kin);
    if ((rc = ensure_workspace(c, probe.off))) return rc;
    Bump bw(c->ws);
    const float* sU = dev ? U : (const float*)bw.take<char>(ub);
    const float* sY = dev ? dY : (const float*)bw.take<char>(yb);
    float* G = bw.take<float>((size_t)Bp * n->Kin);
    if (!dev) {
        PM_CUDA(cudaMemcpyAsync((void*)sU, U, ub, cudaMemcpyHostToDevice, c->stream), "copy U");
        PM_CUDA(cudaMemcpyAsync((void*)sY, dY, yb, cudaMemcpyHostToDevice, c->stream), "copy dY");
    }
    PM_CUDA(cudaMemsetAsync(n->err, 0, 4, c->stream), "clear flag");
    gather_batch_kernel<<<Bp, 128, 0, c->stream>>>(sU, nullptr, nullptr, 0, (int)B, Bp, n->n_in, n->Kin, n->n_out,
                                                   n->Nout, n->Ub, n->Ut, nullptr);
    set_cotangent_kernel<<<Bp, 128, 0, c->stream>>>(sY, (int)B, n->n_out, n->Nout, n->dYb);
    PM_CUDA(cudaGetLastError(), "stage rows");
    count_launch(c, 2);
    // the activations (their ReLU masks) at U
    if ((rc = mlp_forward(c, n, (int)B, Bp))) return rc;
    // dH2 = (dY W3) * [H2 > 0];  dH1 = (dH2 W2) * [H1 > 0];  dU = dH1 W1
    tc::Epilogue e = no_epilogue((int)B, n->H);
    e.mask = n->H2; e.ld_mask = n->H;
    e.out_bf16 = n->dH2b; e.ld_out = n->H;
    if ((rc = gemm(c, n->dYb, n->Nout, n->W3t, n->Nout, Bp, n->H, n->Nout, e, n->err))) return rc;
    e = no_epilogue((int)B, n->H);
    e.mask = n->H1; e.ld_mask = n->H;
    e.out_bf16 = n->dH1b; e.ld_out = n->H;
    if ((rc = gemm(c, n->dH2b, n->H, n->W2t, n->H, Bp, n->H, n->H, e, n->err))) return rc;
    e = no_epilogue((int)B, n->Kin);
    e.out_f32 = G; e.ld_f32 = n->Kin;
    if ((rc = gemm(c, n->dH1b, n->H, n->W1t, n->H, Bp, n->Kin, n->H, e, n->err))) return rc;
    PM_CUDA(cudaMemcpy2DAsync(dU, (size_t)n->n_in * 4, G, (size_t)n->Kin * 4, (size_t)n->n_in * 4, (size_t)B,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
            "copy dU");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    return check_err(c, n);
}

int pm_surrogate_infer(pm_ctx* c, const pm_mlp* nc, const float* U, int64_t B, float* Yout, uint32_t flags)
{
    pm_mlp* n = const_cast<pm_mlp*>(nc);  // the activation workspace is scratch
    if (!c || !n || !U || !Yout) return fail(PM_EINVAL, "NULL argument");
    if (B < 1 || B > (1 << 20)) return fail(PM_EINVAL, "batch size out of range");
    int rc = set_device(c);
    if (rc) return rc;
    const bool dev = flags & PM_DEVICE_PTRS;
    if ((rc = check_ptrs(c, flags, {U, Yout}))) return rc;
    const int Bp = (int)((B + 127) / 128 * 128);
    if ((rc = mlp_reserve(c, n, Bp))) return rc;
    const float* dU = U;
    if (!dev) {
        if ((rc = ensure_workspace(c, (size_t)B * n->n_in * 4 + 256))) return rc;
        PM_CUDA(cudaMemcpyAsync(c->ws, U, (size_t)B * n->n_in * 4, cudaMemcpyHostToDevice, c->stream), "copy U");
        dU = (const float*)c->ws;
    }
    PM_CUDA(cudaMemsetAsync(n->err, 0, 4, c->stream), "clear flag");
    gather_batch_kernel<<<Bp, 128, 0, c->stream>>>(dU, nullptr, nullptr, 0, (int)B, Bp, n->n_in, n->Kin, n->n_out,
                                                   n->Nout, n->Ub, n->Ut, nullptr);
    PM_CUDA(cudaGetLastError(), "gather batch");
    count_launch(c);
    if ((rc = mlp_forward(c, n, (int)B, Bp))) return rc;
    PM_CUDA(cudaMemcpy2DAsync(Yout, (size_t)n->n_out * 4, n->Y, (size_t)n->Nout * 4, (size_t)n->n_out * 4, (size_t)B,
                              dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
            "copy Y");
    if (dev && (flags & PM_ASYNC)) return PM_OK;
    return check_err(c, n);
}

int pm_gemm_bf16(pm_ctx* c, const void* A, int32_t lda, const void* B, int32_t ldb, int32_t M, int32_t N, int32_t K,
                 float* C, int32_t ldc)
{
    if (!c || !A || !B || !C) return fail(PM_EINVAL, "NULL argument");
    int rc = set_device(c);
    if (rc) return rc;
    if ((rc = check_ptrs(c, PM_DEVICE_PTRS, {A, B, C}))) return rc;
    if (ldc % 4 || ((uintptr_t)C % 16)) return fail(PM_EINVAL, "C must be 16-byte aligned with ldc a multiple of 4");
    if ((rc = ensure_workspace(c, 256))) return rc;
    unsigned* err = (unsigned*)c->ws;
    PM_CUDA(cudaMemsetAsync(err, 0, 4, c->stream), "clear flag");
    tc::Epilogue e = no_epilogue(M, N);
    e.out_f32 = C;
    e.ld_f32 = ldc;
    if ((rc = gemm(c, (const bf16*)A, lda, (const bf16*)B, ldb, M, N, K, e, err, take_wait_limit(c)))) return rc;
    unsigned flag = 0;
    PM_CUDA(cudaMemcpyAsync(&flag, err, 4, cudaMemcpyDeviceToHost, c->stream), "copy flag");
    PM_CUDA(cudaStreamSynchronize(c->stream), "gemm");
    if (flag) return fail(PM_ETIMEOUT, "a tensor-core GEMM wait timed out");
    return PM_OK;
}

int pm_surrogate_save(pm_ctx* c, const pm_mlp* n, const char* path)
{
    if (!c || !n || !path) return fail(PM_EINVAL, "NULL argument");
    int rc = set_device(c);
    if (rc) return rc;
    std::vector<float> h((size_t)n->P * 3);
    PM_CUDA(cudaMemcpyAsync(h.data(), n->params, (size_t)n->P * 4, cudaMemcpyDeviceToHost, c->stream), "save");
    PM_CUDA(cudaMemcpyAsync(h.data() + n->P, n->m, (size_t)n->P * 4, cudaMemcpyDeviceToHost, c->stream), "save");
    PM_CUDA(cudaMemcpyAsync(h.data() + 2 * n->P, n->v, (size_t)n->P * 4, cudaMemcpyDeviceToHost, c->stream), "save");
    PM_CUDA(cudaStreamSynchronize(c->stream), "save");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(PM_EINVAL, "cannot open %s", path);
    const int64_t hdr[6] = {0x504d4d4c50303031ll, n->n_in, n->H, n->n_out, n->step, n->P};
    bool ok = fwrite(hdr, sizeof hdr, 1, f) == 1 && fwrite(h.data(), 4, h.size(), f) == h.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? PM_OK : fail(PM_EINVAL, "write to %s failed", path);
}

int pm_surrogate_load(pm_ctx* c, pm_mlp** out, const char* path)
{
    if (!c || !out || !path) return fail(PM_EINVAL, "NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(PM_EINVAL, "cannot open %s", path);
    int64_t hdr[6];
    if (fread(hdr, sizeof hdr, 1, f) != 1 || hdr[0] != 0x504d4d4c50303031ll) { fclose(f); return fail(PM_EINVAL, "not a surrogate file"); }
    pm_mlp* n = nullptr;
    int rc = pm_surrogate_create(c, &n, (int32_t)hdr[1], (int32_t)hdr[2], (int32_t)hdr[3], 0);
    if (rc) { fclose(f); return rc; }
    if (hdr[5] != n->P) { fclose(f); pm_surrogate_destroy(n); return fail(PM_EINVAL, "size mismatch in %s", path); }
    std::vector<float> h((size_t)n->P * 3);
    const bool ok = fread(h.data(), 4, h.size(), f) == h.size();
    fclose(f);
    if (!ok) { pm_surrogate_destroy(n); return fail(PM_EINVAL, "truncated file %s", path); }
    n->step = hdr[4];
    cudaError_t e = cudaMemcpyAsync(n->params, h.data(), (size_t)n->P * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->m, h.data() + n->P, (size_t)n->P * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->v, h.data() + 2 * n->P, (size_t)n->P * 4, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) { pm_surrogate_destroy(n); return cuda_fail(e, "load"); }
    if ((rc = mlp_cast_weights(c, n))) { pm_surrogate_destroy(n); return rc; }
    PM_CUDA(cudaStreamSynchronize(c->stream), "load");
    *out = n;
    return PM_OK;
}

}  // extern "C"
