// Key switch of a large launch as a dense product on the tensor cores.
//
// For a launch of J ciphertexts the key switch is a matrix product: digits
// D[J][kN*l] (balanced, |d| <= B/2 = 4) times the key-switching key
// KSK[kN*l][n+1] (words mod 2^64).  Splitting every key word into its eight
// bytes makes it an exact BF16 product: digits and bytes are exact in bf16,
// each product is an integer of at most 4 * 255, and a partial sum over a
// chunk of 2560 rows stays below 2^22 in magnitude, exact in FP32 whatever the
// accumulation order.  So the key switch runs as cuBLAS bf16 x bf16 -> fp32
// GEMMs (4 chunks of the reduction dimension, one strided-batched call) and a
// small kernel recombines bytes and chunks mod 2^64, adds the body and
// modulus-switches -- the same integers as k_keyswitch, bit for bit.
//
//   kmat  [8 (n+1)][kN l] bf16   row c*8 + b = byte b of column c of the KSK
//   dig   [J][kN l] bf16         digits of the launch
//   acc   [4][J][8 (n+1)] fp32   per-chunk products
#include <algorithm>
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include "lvs_internal.hpp"

namespace lvs {

constexpr int kKsChunks = 4;
constexpr size_t kKsGemmBatch = 8192;   // jobs per GEMM (bounds the scratch)

struct KsGemm {
    cublasHandle_t h = nullptr;
    __nv_bfloat16 *kmat = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    __nv_bfloat16 *dig = nullptr;       // [kKsGemmBatch][kdim]
    float *acc = nullptr;               // [kKsChunks][kKsGemmBatch][M]
    uint32_t kdim = 0, M = 0;
};

namespace {

__global__ void k_ksk_bytes(const uint64_t *__restrict__ ksk, uint32_t rows, uint32_t n, __nv_bfloat16 *kmat)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over rows * (n+1)
    if (idx >= (size_t)rows * (n + 1)) return;
    const uint32_t r = (uint32_t)(idx / (n + 1)), c = (uint32_t)(idx % (n + 1));
    const uint64_t w = ksk[idx];
#pragma unroll
    for (int b = 0; b < 8; ++b)
        kmat[((size_t)c * 8 + b) * rows + r] = __float2bfloat16((float)((w >> (8 * b)) & 0xffu));
}

// digits of the jobs' input combinations: dig[j][u * l + lev - 1] = balanced
// digit of level lev (lev = 1 most significant), the decomposition of k_keyswitch
__global__ void k_ks_digits(const Job *__restrict__ jobs, uint32_t njobs, uint32_t big, uint32_t ks_level,
                            uint32_t ks_base_log, __nv_bfloat16 *__restrict__ dig)
{
    const uint32_t j = blockIdx.y;
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= njobs || u >= big) return;
    const Job &J = jobs[j];
    uint64_t a = 0;
#pragma unroll
    for (int s = 0; s < 3; ++s)
        if (J.src[s]) a += (uint64_t)(int64_t)J.coef[s] * __ldg(J.src[s] + u);
    const uint32_t beta = ks_level * ks_base_log;
    const uint64_t v = (a + (1ull << (63 - beta))) >> (64 - beta);
    const uint32_t Bk = 1u << ks_base_log, hBk = Bk >> 1;
    uint32_t carry = 0;
    __nv_bfloat16 *out = dig + (size_t)j * big * ks_level + (size_t)u * ks_level;
    for (int lev = (int)ks_level; lev >= 1; --lev) {
        const uint32_t uu = (uint32_t)(v >> ((ks_level - lev) * ks_base_log)) & (Bk - 1);
        const uint32_t r = uu + carry;
        carry = r >= hBk;
        out[lev - 1] = __float2bfloat16((float)((int)r - (int)(carry * Bk)));
    }
}

// recombination: sum over chunks and bytes mod 2^64, body, modulus switch
__global__ void k_ks_combine(const Job *__restrict__ jobs, uint32_t njobs, const float *__restrict__ acc, uint32_t M,
                             uint32_t n, uint32_t big, uint32_t log2_2N, uint32_t *__restrict__ ms)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)njobs * (n + 1)) return;
    const uint32_t j = (uint32_t)(idx / (n + 1)), c = (uint32_t)(idx % (n + 1));
    uint64_t sum = 0;
    for (int ch = 0; ch < kKsChunks; ++ch) {
        const float *a = acc + ((size_t)ch * njobs + j) * M + (size_t)c * 8;
#pragma unroll
        for (int b = 0; b < 8; ++b) sum += (uint64_t)(int64_t)a[b] << (8 * b);
    }
    uint64_t val = 0 - sum;
    if (c == n) {
        const Job &J = jobs[j];
        uint64_t bb = (uint64_t)(J.cst & 31) << kDeltaLog;
        for (int s = 0; s < 3; ++s)
            if (J.src[s]) bb += (uint64_t)(int64_t)J.coef[s] * J.src[s][big];
        val += bb;
    }
    ms[idx] = (uint32_t)((val + (1ull << (63 - log2_2N))) >> (64 - log2_2N)) & ((1u << log2_2N) - 1);
}

}  // namespace

void ks_gemm_free(lvs_ctx *ctx)
{
    KsGemm *g = ctx->ks_gemm;
    if (!g) return;
    if (g->h) cublasDestroy(g->h);
    cudaFree(g->kmat);
    cudaFree(g->ws);
    cudaFree(g->dig);
    cudaFree(g->acc);
    cudaGetLastError();
    delete g;
    ctx->ks_gemm = nullptr;
}

lvs_status ks_gemm_init(lvs_ctx *ctx)
{
    const auto &p = ctx->P.p;
    const uint32_t kdim = ctx->P.big() * p.ks_level, M = 8 * (p.n + 1);
    if (kdim % kKsChunks != 0) return LVS_OK;   // not available for this shape
    KsGemm *g = new (std::nothrow) KsGemm;
    if (!g) return set_error(LVS_ERR_OOM, "key-switch GEMM: host allocation failed");
    ctx->ks_gemm = g;
    g->kdim = kdim;
    g->M = M;
    g->ws_bytes = (size_t)32 << 20;
    if (cublasCreate(&g->h) != CUBLAS_STATUS_SUCCESS) {
        ks_gemm_free(ctx);
        return set_error(LVS_ERR_CUDA, "key-switch GEMM: cublasCreate failed");
    }
    if (cudaMalloc((void **)&g->kmat, (size_t)M * kdim * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&g->ws, g->ws_bytes) != cudaSuccess ||
        cudaMalloc((void **)&g->dig, kKsGemmBatch * kdim * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc((void **)&g->acc, (size_t)kKsChunks * kKsGemmBatch * M * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        ks_gemm_free(ctx);
        return set_error(LVS_ERR_OOM, "key-switch GEMM: device allocation failed");
    }
    if (cublasSetWorkspace(g->h, g->ws, g->ws_bytes) != CUBLAS_STATUS_SUCCESS) {
        ks_gemm_free(ctx);
        return set_error(LVS_ERR_CUDA, "key-switch GEMM: cublasSetWorkspace failed");
    }
    const size_t total = (size_t)kdim * (p.n + 1);
    k_ksk_bytes<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ctx->ksk, kdim, p.n, g->kmat);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ks_gemm_free(ctx);
        return cuda_error(e, "key-switch GEMM: key conversion");
    }
    return LVS_OK;
}

cudaError_t launch_keyswitch_gemm(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                                  int *nlaunch)
{
    KsGemm *g = ctx->ks_gemm;
    const auto &p = ctx->P.p;
    const uint32_t big = ctx->P.big(), kc = g->kdim / kKsChunks;
    const uint32_t log2_2N = ctx->P.log_n() + 1;
    int launches = 0;
    if (cublasSetStream(g->h, s) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    for (size_t j0 = 0; j0 < njobs; j0 += kKsGemmBatch) {
        const uint32_t nj = (uint32_t)std::min(kKsGemmBatch, njobs - j0);
        dim3 grid((big + 255) / 256, nj);
        k_ks_digits<<<grid, 256, 0, s>>>(jobs + j0, nj, big, p.ks_level, p.ks_base_log, g->dig);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const float alpha = 1.0f, beta = 0.0f;
        // acc[ch] (M x nj, column-major) = kmat[:, chunk]^T (M x kc) * dig[:, chunk] (kc x nj)
        const cublasStatus_t cs = cublasGemmStridedBatchedEx(
            g->h, CUBLAS_OP_T, CUBLAS_OP_N, (int)g->M, (int)nj, (int)kc, &alpha, g->kmat, CUDA_R_16BF, (int)g->kdim,
            (long long)kc, g->dig, CUDA_R_16BF, (int)g->kdim, (long long)kc, &beta, g->acc, CUDA_R_32F, (int)g->M,
            (long long)g->M * nj, kKsChunks, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
        if (cs != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
        const size_t total = (size_t)nj * (p.n + 1);
        k_ks_combine<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(jobs + j0, nj, g->acc, g->M, p.n, big, log2_2N,
                                                                     ms + j0 * (p.n + 1));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        launches += 2;
    }
    if (nlaunch) *nlaunch = launches;
    return cudaSuccess;
}

// key switch of a launch: the tensor-core form from ks_gemm_min PBS on, the
// kernel (k_keyswitch with its plan) below
cudaError_t launch_keyswitch_auto(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                                  int *nlaunch)
{
    if (ctx->ks_gemm && ctx->ks_gemm_min && njobs >= ctx->ks_gemm_min)
        return launch_keyswitch_gemm(ctx, jobs, njobs, ms, s, nlaunch);
    return launch_keyswitch(ctx, jobs, njobs, ms, s, nlaunch);
}

}  // namespace lvs
