// Autotuner of the launch shapes: the key switch's (jobs per CTA and split
// of the input coefficients over CTAs, per launch-size bucket, and from which
// launch size the tensor-core GEMM form takes over) and the blind
// rotation's (one CTA per ciphertext, or three -- one per prime -- for small
// launches).
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
    size_t gemm_min = 0;
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
        // the tensor-core key switch against the best kernel plan of the
        // bucket: the GEMM path serves every launch from the smallest
        // bucket size where it is faster
        if (st == LVS_OK && ctx->ks_gemm && nj >= 256) {
            float tg = 1e30f;
            for (int rep = 0; rep < 4 && st == LVS_OK; ++rep) {
                cudaError_t e3 = cudaEventRecord(e0, ctx->stream);
                if (e3 == cudaSuccess) e3 = launch_keyswitch_gemm(ctx, djobs, nj, ms, ctx->stream, nullptr);
                if (e3 == cudaSuccess) e3 = cudaEventRecord(e1, ctx->stream);
                if (e3 == cudaSuccess) e3 = cudaEventSynchronize(e1);
                float ms_ = 0;
                if (e3 == cudaSuccess) e3 = cudaEventElapsedTime(&ms_, e0, e1);
                if (e3 != cudaSuccess) st = cuda_error(e3, "lvs_ctx_autotune: key-switch GEMM timing");
                else if (rep > 0) tg = std::min(tg, ms_);
            }
            if (st == LVS_OK && tg < best_t && gemm_min == 0) gemm_min = nj;
        }
    }
    if (st == LVS_OK && ctx->ks_gemm) ctx->ks_gemm_min = gemm_min;
    // blind rotation: one CTA per ciphertext vs three CTAs (one per prime) per
    // ciphertext, on synthetic jobs (rotation amounts from a byte pattern);
    // the three-CTA form is kept up to the largest tested launch size where it
    // is faster, scanning upwards
    if (st == LVS_OK && ctx->br_clusters > 0) {
        const size_t nmax = 2 * (size_t)ctx->num_sms;
        uint64_t *dst = nullptr;
        if (cudaMalloc((void **)&dst, nmax * row * 8) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return set_error(LVS_ERR_OOM, "lvs_ctx_autotune: device allocation failed");
        }
        std::vector<Job> bj(nmax);
        for (size_t k = 0; k < nmax; ++k) {
            memset(&bj[k], 0, sizeof(Job));
            bj[k].kind = JOB_STORE;
            bj[k].lut = LUT_MIN;
            bj[k].dst[0] = dst + k * row;
        }
        cudaError_t e2 = cudaMemcpyAsync(djobs, bj.data(), nmax * sizeof(Job), cudaMemcpyHostToDevice, ctx->stream);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(ms, 0x35, nmax * (p.n + 1) * 4, ctx->stream);
        if (e2 != cudaSuccess) st = cuda_error(e2, "lvs_ctx_autotune: blind-rotation set-up");
        const size_t keep = ctx->br_split_max;
        size_t best_max = 0;
        const size_t sizes[] = {1, 8, 24, (size_t)ctx->num_sms / 3, (size_t)ctx->num_sms / 2,
                                (size_t)(2 * ctx->num_sms) / 3, (size_t)ctx->num_sms};
        for (size_t nj : sizes) {
            if (st != LVS_OK || nj == 0 || nj > nmax) break;
            float t[2] = {0, 0};
            for (int form = 0; form < 2 && st == LVS_OK; ++form) {
                ctx->br_split_max = form == 1 ? nj : 0;
                float best_t = 1e30f;
                for (int rep = 0; rep < 3 && st == LVS_OK; ++rep) {
                    cudaError_t e3 = cudaEventRecord(e0, ctx->stream);
                    if (e3 == cudaSuccess) e3 = launch_blind_rotate(ctx, djobs, nj, ms, ctx->luts, 0, ctx->stream);
                    if (e3 == cudaSuccess) e3 = cudaEventRecord(e1, ctx->stream);
                    if (e3 == cudaSuccess) e3 = cudaEventSynchronize(e1);
                    float ms_ = 0;
                    if (e3 == cudaSuccess) e3 = cudaEventElapsedTime(&ms_, e0, e1);
                    if (e3 != cudaSuccess) st = cuda_error(e3, "lvs_ctx_autotune: blind-rotation timing");
                    else if (rep > 0) best_t = std::min(best_t, ms_);
                }
                t[form] = best_t;
            }
            if (st != LVS_OK || t[1] >= t[0]) break;
            best_max = nj;
        }
        ctx->br_split_max = st == LVS_OK ? best_max : keep;
        cudaStreamSynchronize(ctx->stream);
        cudaFree(dst);
    }
    cleanup();
    return st;
}

lvs_status lvs_ctx_ks_plan(lvs_ctx *ctx, size_t njobs, int32_t *jobs_per_cta, int32_t *split)
{
    if (!ctx || !jobs_per_cta || !split) return set_error(LVS_ERR_ARG, "lvs_ctx_ks_plan: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    const KsPlan pl = ks_plan(ctx, njobs);
    *jobs_per_cta = pl.tj;
    *split = pl.split;
    return LVS_OK;
}

lvs_status lvs_ctx_ks_gemm_min(lvs_ctx *ctx, size_t *min_jobs)
{
    if (!ctx || !min_jobs) return set_error(LVS_ERR_ARG, "lvs_ctx_ks_gemm_min: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *min_jobs = ctx->ks_gemm ? ctx->ks_gemm_min : 0;
    return LVS_OK;
}

lvs_status lvs_ctx_set_ks_gemm_min(lvs_ctx *ctx, size_t min_jobs)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_ks_gemm_min: NULL context");
    if (min_jobs > 0 && !ctx->ks_gemm)
        return set_error(LVS_ERR_STATE, "lvs_ctx_set_ks_gemm_min: the tensor-core key switch is unavailable");
    std::lock_guard<std::mutex> lock(ctx->mu);   // batch calls read it under the lock
    ctx->ks_gemm_min = min_jobs;
    return LVS_OK;
}

lvs_status lvs_ctx_max_launch_jobs(lvs_ctx *ctx, size_t *max_jobs)
{
    if (!ctx || !max_jobs) return set_error(LVS_ERR_ARG, "lvs_ctx_max_launch_jobs: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *max_jobs = ctx->max_launch_jobs;
    return LVS_OK;
}

lvs_status lvs_ctx_set_max_launch_jobs(lvs_ctx *ctx, size_t max_jobs)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_max_launch_jobs: NULL context");
    if (max_jobs == 0) max_jobs = (size_t)1 << 16;
    if (max_jobs < 2 || max_jobs > ((size_t)1 << 20))
        return set_error(LVS_ERR_ARG, "lvs_ctx_set_max_launch_jobs: max_jobs must be in [2, 2^20]");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->max_launch_jobs = max_jobs;
    return LVS_OK;
}

lvs_status lvs_ctx_set_wave_fill(lvs_ctx *ctx, int32_t enable)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_wave_fill: NULL context");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->wave_fill = enable != 0;
    return LVS_OK;
}

lvs_status lvs_ctx_wave_fill(lvs_ctx *ctx, int32_t *enabled)
{
    if (!ctx || !enabled) return set_error(LVS_ERR_ARG, "lvs_ctx_wave_fill: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *enabled = ctx->wave_fill ? 1 : 0;
    return LVS_OK;
}

lvs_status lvs_ctx_set_key_staging(lvs_ctx *ctx, int32_t enable)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_key_staging: NULL context");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->key_staging = enable != 0 ? 1 : 0;
    return LVS_OK;
}

lvs_status lvs_ctx_key_staging(lvs_ctx *ctx, int32_t *enabled)
{
    if (!ctx || !enabled) return set_error(LVS_ERR_ARG, "lvs_ctx_key_staging: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *enabled = ctx->key_staging;
    return LVS_OK;
}

lvs_status lvs_debug_drop_key_copy(lvs_ctx *ctx, int32_t enable)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_debug_drop_key_copy: NULL context");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->debug_drop_key_copy = enable != 0;
    return LVS_OK;
}

lvs_status lvs_ctx_br_split(lvs_ctx *ctx, size_t *max_jobs)
{
    if (!ctx || !max_jobs) return set_error(LVS_ERR_ARG, "lvs_ctx_br_split: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *max_jobs = ctx->br_clusters > 0 ? ctx->br_split_max : 0;
    return LVS_OK;
}

lvs_status lvs_ctx_set_br_split(lvs_ctx *ctx, size_t max_jobs)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_br_split: NULL context");
    if (max_jobs > 0 && ctx->br_clusters <= 0)
        return set_error(LVS_ERR_STATE, "lvs_ctx_set_br_split: the device cannot run the three-CTA form");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->br_split_max = max_jobs;
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
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->ks_tuned[ks_bucket(njobs)] = pl;
    return LVS_OK;
}

}  // extern "C"
