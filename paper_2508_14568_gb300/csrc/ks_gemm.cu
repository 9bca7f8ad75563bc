// Key switch of a wide launch as a dense product on the tensor cores.
//
// For a launch of J ciphertexts the key switch (Section 2.2: PBS = key switch,
// modulus switch, blind rotation, sample extract) is a matrix product: the
// balanced digits D[J][kN*l] (|d| <= B/2 = 4) of the launch's inputs times
// the key-switching key KSK[kN*l][n+1] (words mod 2^64).  Splitting every key
// word into its eight bytes makes it an exact bf16 product: digits and bytes
// are exact in bf16, each product is an integer of magnitude at most 4 * 255,
// and every partial sum over the 10,240-long reduction stays below 2^24 in
// magnitude, so the fp32 accumulation is exact whatever its order.
//
// k_ks_digits writes the digits; k_ks_mma multiplies them with the key's byte
// planes on the tensor cores (mma.sync m16n8k16 bf16 -> fp32, 128 x 128 tiles
// staged through swizzled shared memory by cp.async, three stages) and, in the
// same kernel, rebuilds each output word mod 2^64 from its eight byte-plane
// sums (the eight columns of one 8-wide n-tile are the eight bytes of one key
// column, held by the four lanes of a quad), adds the body and
// modulus-switches: the same integers as k_keyswitch, bit for bit.
//
//   kmat  [ncols_pad][kN l] bf16   row 8c + b = byte b of column c of the KSK
//   dig   [batch][kN l] bf16       digits of the launch (row = job)
#include <algorithm>
#include <cuda_bf16.h>

#include "lvs_internal.hpp"

namespace lvs {

constexpr int KT_M = 128;        // jobs per CTA tile
constexpr int KT_N = 128;        // byte columns per CTA tile (16 key columns)
constexpr int KT_K = 64;         // reduction elements per stage (128 bytes per row)
constexpr int KT_STAGES = 3;
constexpr int KT_THREADS = 256;  // 8 warps: 2 along the jobs x 4 along the columns
constexpr size_t KT_STAGE_BYTES = (size_t)(KT_M + KT_N) * KT_K * 2;
constexpr size_t KT_SMEM = KT_STAGES * KT_STAGE_BYTES;   // 96 KB
constexpr size_t kKsGemmBatch = 8192;   // jobs per pass (bounds the digit scratch; a multiple of KT_M)

struct KsGemm {
    __nv_bfloat16 *kmat = nullptr;
    __nv_bfloat16 *dig = nullptr;       // [kKsGemmBatch][kdim]
    uint32_t kdim = 0, ncols = 0, nrows_pad = 0;
};

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of 16-byte chunk `ch` (0..7) of row `r` in a [rows][64] bf16 tile:
// rows of 128 bytes, chunks XOR-swizzled by the row's low three bits so that
// the eight rows one ldmatrix reads land on distinct banks
__device__ __forceinline__ uint32_t tile_off(uint32_t r, uint32_t ch) { return r * 128 + ((ch ^ (r & 7)) << 4); }

__global__ void k_ksk_bytes(const uint64_t *__restrict__ ksk, uint32_t rows, uint32_t n, uint32_t nrows_pad,
                            __nv_bfloat16 *kmat)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;   // over rows * nrows_pad / 8
    const size_t ncol_pad = nrows_pad / 8;
    if (idx >= (size_t)rows * ncol_pad) return;
    const uint32_t r = (uint32_t)(idx / ncol_pad), c = (uint32_t)(idx % ncol_pad);
    const uint64_t w = c <= n ? ksk[(size_t)r * (n + 1) + c] : 0;   // padding columns are zero
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

// One CTA: jobs [j0, j0 + 128) x byte columns [c0, c0 + 128) over the whole
// reduction.  Warp (wm, wn) owns 64 jobs x 32 byte columns = 4 x 4 m16n8 tiles;
// the n8 tile ni of a warp is key column (c0 + 32 wn + 8 ni) / 8.  The digit
// rows of the last tile past njobs hold stale values of earlier launches:
// rows of the product are independent and those rows are not written.
__global__ void __launch_bounds__(KT_THREADS, 2)
k_ks_mma(const __nv_bfloat16 *__restrict__ dig, const __nv_bfloat16 *__restrict__ kmat, uint32_t kdim,
         const Job *__restrict__ jobs, uint32_t njobs, uint32_t n, uint32_t big, uint32_t log2_2N,
         uint32_t *__restrict__ ms)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const uint32_t j0 = blockIdx.y * KT_M, c0 = blockIdx.x * KT_N;
    const uint32_t sbase = smem_u32(smem);
    const int nk = (int)(kdim / KT_K);

    auto load_stage = [&](int stage, int kt) {
        const uint32_t sa = sbase + stage * (uint32_t)KT_STAGE_BYTES, sb = sa + KT_M * KT_K * 2;
        const size_t k0 = (size_t)kt * KT_K;
#pragma unroll
        for (int i = 0; i < (KT_M * 8) / KT_THREADS; ++i) {
            const int id = tid + i * KT_THREADS, r = id >> 3, ch = id & 7;
            cp_async16(sa + tile_off(r, ch), dig + (size_t)(j0 + r) * kdim + k0 + ch * 8);
            cp_async16(sb + tile_off(r, ch), kmat + (size_t)(c0 + r) * kdim + k0 + ch * 8);
        }
    };

    float acc[4][4][4];
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][ni][q] = 0.f;

#pragma unroll
    for (int s = 0; s < KT_STAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<KT_STAGES - 2>();
        __syncthreads();   // stage kt is in place; everyone is done with stage kt - 1
        if (kt + KT_STAGES - 1 < nk) load_stage((kt + KT_STAGES - 1) % KT_STAGES, kt + KT_STAGES - 1);
        cp_async_commit();
        const uint32_t sa = sbase + (kt % KT_STAGES) * (uint32_t)KT_STAGE_BYTES, sb = sa + KT_M * KT_K * 2;
#pragma unroll
        for (int ks = 0; ks < KT_K / 16; ++ks) {
            uint32_t a[4][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const uint32_t r = wm * 64 + mi * 16 + (lane & 15);
                ldsm_x4(sa + tile_off(r, ks * 2 + (lane >> 4)), a[mi][0], a[mi][1], a[mi][2], a[mi][3]);
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const uint32_t r = wn * 32 + np * 16 + ((lane >> 4) << 3) + (lane & 7);
                ldsm_x4(sb + tile_off(r, ks * 2 + ((lane >> 3) & 1)), b[2 * np][0], b[2 * np][1], b[2 * np + 1][0],
                        b[2 * np + 1][1]);
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], a[mi], b[ni][0], b[ni][1]);
        }
    }
    cp_async_wait<0>();

    // epilogue: lane (g, t) holds byte planes 2t, 2t+1 of rows g and g + 8 of
    // each tile; the quad's four lanes together hold the eight bytes of the word
    const int g = lane >> 2, t = lane & 3;
    const uint32_t twoN_mask = (1u << log2_2N) - 1;
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
        const uint32_t c = (c0 + wn * 32 + ni * 8) >> 3;   // key column
#pragma unroll
        for (int mi = 0; mi < 4; ++mi) {
            uint64_t s[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t lo = __float2int_rn(acc[mi][ni][2 * h]), hi = __float2int_rn(acc[mi][ni][2 * h + 1]);
                s[h] = ((uint64_t)lo << (16 * t)) + ((uint64_t)hi << (16 * t + 8));
                s[h] += __shfl_xor_sync(0xffffffffu, s[h], 1);
                s[h] += __shfl_xor_sync(0xffffffffu, s[h], 2);
            }
            if (t < 2 && c <= n) {
                const uint32_t j = j0 + wm * 64 + mi * 16 + g + 8 * t;
                if (j < njobs) {
                    uint64_t val = 0 - (t == 0 ? s[0] : s[1]);   // (0, b) - sum_{u, lev} d * KSK
                    if (c == n) {
                        const Job &J = jobs[j];
                        uint64_t bb = (uint64_t)(J.cst & 31) << kDeltaLog;
                        for (int q = 0; q < 3; ++q)
                            if (J.src[q]) bb += (uint64_t)(int64_t)J.coef[q] * J.src[q][big];
                        val += bb;
                    }
                    ms[(size_t)j * (n + 1) + c] =
                        (uint32_t)((val + (1ull << (63 - log2_2N))) >> (64 - log2_2N)) & twoN_mask;
                }
            }
        }
    }
}

}  // namespace

void ks_gemm_free(lvs_ctx *ctx)
{
    KsGemm *g = ctx->ks_gemm;
    if (!g) return;
    cudaFree(g->kmat);
    cudaFree(g->dig);
    cudaGetLastError();
    delete g;
    ctx->ks_gemm = nullptr;
}

lvs_status ks_gemm_init(lvs_ctx *ctx)
{
    const auto &p = ctx->P.p;
    const uint32_t kdim = ctx->P.big() * p.ks_level;
    if (kdim % KT_K != 0) return LVS_OK;   // not available for this shape
    KsGemm *g = new (std::nothrow) KsGemm;
    if (!g) return set_error(LVS_ERR_OOM, "key-switch GEMM: host allocation failed");
    ctx->ks_gemm = g;
    g->kdim = kdim;
    g->ncols = p.n + 1;
    g->nrows_pad = (uint32_t)((8 * (size_t)(p.n + 1) + KT_N - 1) / KT_N * KT_N);
    if (cudaFuncSetAttribute(k_ks_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)KT_SMEM) != cudaSuccess) {
        cudaGetLastError();
        ks_gemm_free(ctx);
        return set_error(LVS_ERR_CUDA, "key-switch GEMM: kernel attribute");
    }
    if (cudaMalloc((void **)&g->kmat, (size_t)g->nrows_pad * kdim * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc((void **)&g->dig, kKsGemmBatch * kdim * sizeof(__nv_bfloat16)) != cudaSuccess) {
        cudaGetLastError();
        ks_gemm_free(ctx);
        return set_error(LVS_ERR_OOM, "key-switch GEMM: device allocation failed");
    }
    const size_t total = (size_t)kdim * (g->nrows_pad / 8);
    k_ksk_bytes<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(ctx->ksk, kdim, p.n, g->nrows_pad, g->kmat);
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
    const uint32_t big = ctx->P.big();
    const uint32_t log2_2N = ctx->P.log_n() + 1;
    int launches = 0;
    for (size_t j0 = 0; j0 < njobs; j0 += kKsGemmBatch) {
        const uint32_t nj = (uint32_t)std::min(kKsGemmBatch, njobs - j0);
        dim3 grid((big + 255) / 256, nj);
        k_ks_digits<<<grid, 256, 0, s>>>(jobs + j0, nj, big, p.ks_level, p.ks_base_log, g->dig);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        dim3 mgrid(g->nrows_pad / KT_N, (nj + KT_M - 1) / KT_M);
        k_ks_mma<<<mgrid, KT_THREADS, KT_SMEM, s>>>(g->dig, g->kmat, g->kdim, jobs + j0, nj, p.n, big, log2_2N,
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
