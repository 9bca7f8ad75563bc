// Autotuner of the key-switch launch shape (jobs per CTA and split of the
// input coefficients over CTAs), per launch-size bucket.
//
// Small launches (one pair's first anti-diagonals, a lone query) leave most
// SMs idle with one CTA column block per 16 jobs; splitting the 2048 input
// coefficients over gridDim.z and finishing with k_ks_finish fills the GPU,
// at the cost of writing and re-reading partial sums.  The best split depends
// on the launch size and the device, so it is measured: every candidate plan
// of a bucket runs on synthetic jobs (the kernel's work does not depend on the
// data) and the fastest is kept in the context.  Every plan computes the same
// values (sums mod 2^64 in any order), which the tests check bit for bit.
#include <algorithm>
#include <cstring>
#include <vector>

#include "lvs_internal.hpp"

namespace lvs {

static const size_t kBucketSize[kKsBuckets] = {4, 16, 64, 256, 1024, 4096};

static lvs_status time_plan(lvs_ctx *ctx, const Job *jobs, size_t nj, uint32_t *ms, uint64_t *part, KsPlan pl,
                            cudaEvent_t e0, cudaEvent_t e1, float *best)
{
    float t = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        LVS_CUDA(cudaEventRecord(e0, ctx->stream));
        LVS_CUDA(launch_keyswitch_plan(ctx, jobs, nj, ms, part, pl, ctx->stream));
        LVS_CUDA(cudaEventRecord(e1, ctx->stream));
        LVS_CUDA(cudaEventSynchronize(e1));
        float ms_ = 0;
        LVS_CUDA(cudaEventElapsedTime(&ms_, e0, e1));
        if (rep > 0) t = std::min(t, ms_);   // first run is a warm-up
    }
    *best = t;
    return LVS_OK;
}

}  // namespace lvs

using namespace lvs;

extern "C" {

lvs_status lvs_ctx_autotune(lvs_ctx *ctx)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_autotune: NULL context");
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaStreamSynchronize(ctx->stream));
    const auto &p = ctx->P.p;
    const size_t row = (size_t)ctx->P.big() + 2;
    const size_t max_nj = kBucketSize[kKsBuckets - 1];
    const size_t part_limit = (size_t)64 << 20 >> 3;   // 64 MB of partial sums at most
    uint64_t *src = nullptr, *part = nullptr;
    uint32_t *ms = nullptr;
    Job *djobs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lvs_status st = LVS_OK;
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(src); cudaFree(part); cudaFree(ms); cudaFree(djobs);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc((void **)&src, row * 8) != cudaSuccess || cudaMalloc((void **)&part, part_limit * 8) != cudaSuccess ||
        cudaMalloc((void **)&ms, max_nj * (p.n + 1) * 4) != cudaSuccess ||
        cudaMalloc((void **)&djobs, max_nj * sizeof(Job)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return set_error(LVS_ERR_OOM, "lvs_ctx_autotune: device allocation failed");
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return set_error(LVS_ERR_CUDA, "lvs_ctx_autotune: event creation failed");
    }
    std::vector<Job> jobs(max_nj);
    for (auto &J : jobs) {
        memset(&J, 0, sizeof(J));
        J.src[0] = src;
        J.coef[0] = 1;
    }
    cudaError_t e = cudaMemsetAsync(src, 0x5a, row * 8, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(djobs, jobs.data(), max_nj * sizeof(Job), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_error(e, "lvs_ctx_autotune: set-up");
    }
    const int splits[] = {1, 2, 4, 8, 16, 32};
    for (int b = 0; b < kKsBuckets && st == LVS_OK; ++b) {
        const size_t nj = kBucketSize[b];
        KsPlan best;
        float best_t = 1e30f;
        for (int tj : {4, 16}) {
            if (tj == 4 && nj > 64) continue;
            for (int sp : splits) {
                if ((size_t)sp * nj * (p.n + 1) > part_limit && sp > 1) continue;
                KsPlan pl;
                pl.tj = tj;
                pl.split = sp;
                float t = 0;
                st = time_plan(ctx, djobs, nj, ms, part, pl, e0, e1, &t);
                if (st != LVS_OK) break;
                if (t < best_t) { best_t = t; best = pl; }
            }
            if (st != LVS_OK) break;
        }
        if (st == LVS_OK) ctx->ks_tuned[b] = best;
    }
    cleanup();
    return st;
}

lvs_status lvs_ctx_ks_plan(lvs_ctx *ctx, size_t njobs, int32_t *jobs_per_cta, int32_t *split)
{
    if (!ctx || !jobs_per_cta || !split) return set_error(LVS_ERR_ARG, "lvs_ctx_ks_plan: NULL argument");
    const KsPlan pl = ks_plan(ctx, njobs);
    *jobs_per_cta = pl.tj;
    *split = pl.split;
    return LVS_OK;
}

lvs_status lvs_ctx_set_ks_plan(lvs_ctx *ctx, size_t njobs, int32_t jobs_per_cta, int32_t split)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_ks_plan: NULL context");
    if ((jobs_per_cta != 0 && jobs_per_cta != 4 && jobs_per_cta != 16) || split < 1 || split > 32)
        return set_error(LVS_ERR_ARG, "lvs_ctx_set_ks_plan: jobs_per_cta must be 4 or 16 (0: default), split 1..32");
    KsPlan pl;
    pl.tj = jobs_per_cta;
    pl.split = jobs_per_cta ? split : 1;
    ctx->ks_tuned[ks_bucket(njobs)] = pl;
    return LVS_OK;
}

}  // extern "C"
