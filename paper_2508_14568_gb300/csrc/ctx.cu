// Device context: key upload and conversion, scratch memory, launch runner
// (direct launches or one CUDA graph per run), kernel timing, and the
// low-level device-pointer entry points.
#include <algorithm>
#include <cstring>

#include <nvtx3/nvToolsExt.h>

#include "lvs_internal.hpp"
#include "ntt.cuh"

namespace lvs {

int br_blocks_per_sm(uint32_t N);   // kernels.cu

static lvs_status device_ok(int device)
{
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return set_error(LVS_ERR_CUDA, std::string("no CUDA device available: ") +
                                           (e != cudaSuccess ? cudaGetErrorString(e) : "0 devices"));
    if (device < 0 || device >= ndev) return set_error(LVS_ERR_ARG, "device index out of range");
    return LVS_OK;
}

lvs_status ensure_scratch(lvs_ctx *ctx, size_t njobs_total, size_t njobs_step)
{
    const size_t row = (size_t)ctx->P.p.n + 1;
    if (njobs_total > ctx->jobs_cap) {
        if (ctx->jobs) LVS_CUDA(cudaFreeAsync(ctx->jobs, ctx->stream));
        ctx->jobs = nullptr;
        ctx->jobs_cap = 0;
        const size_t cap = std::max(njobs_total, ctx->jobs_cap + ctx->jobs_cap / 2);
        if (cudaMallocAsync((void **)&ctx->jobs, cap * sizeof(Job), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LVS_ERR_OOM, "device allocation of the job list failed");
        }
        ctx->jobs_cap = cap;
    }
    // split key-switch scratch: the largest need over launch sizes up to njobs_step
    // (the plan is constant within a bucket, so bucket ends and njobs_step suffice)
    size_t part = 0;
    for (size_t lim = 4; lim < njobs_step; lim *= 4) part = std::max(part, ks_part_words(ctx, lim));
    if (njobs_step) part = std::max(part, ks_part_words(ctx, njobs_step));
    if (part > ctx->ks_part_cap) {
        if (ctx->ks_part) LVS_CUDA(cudaFreeAsync(ctx->ks_part, ctx->stream));
        ctx->ks_part = nullptr;
        ctx->ks_part_cap = 0;
        if (cudaMallocAsync((void **)&ctx->ks_part, part * sizeof(uint64_t), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LVS_ERR_OOM, "device allocation of the key-switch partial sums failed");
        }
        ctx->ks_part_cap = part;
    }
    if (njobs_step > ctx->ms_cap) {
        if (ctx->ms) LVS_CUDA(cudaFreeAsync(ctx->ms, ctx->stream));
        ctx->ms = nullptr;
        ctx->ms_cap = 0;
        const size_t cap = std::max(njobs_step, ctx->ms_cap + ctx->ms_cap / 2);
        if (cudaMallocAsync((void **)&ctx->ms, cap * row * sizeof(uint32_t), ctx->stream) != cudaSuccess) {
            cudaGetLastError();
            return set_error(LVS_ERR_OOM, "device allocation of the modulus-switch buffer failed");
        }
        ctx->ms_cap = cap;
    }
    return LVS_OK;
}

namespace {
std::mutex g_fault_mu;
uint32_t *g_fault_host[64];
uint32_t *g_fault_dev[64];
}  // namespace

uint32_t *device_fault_word(int device)
{
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_fault_mu);
    if (!g_fault_dev[device]) {
        uint32_t *h = nullptr, *d = nullptr;
        if (cudaHostAlloc((void **)&h, sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        *h = 0;
        if (cudaHostGetDevicePointer((void **)&d, h, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeHost(h);
            return nullptr;
        }
        g_fault_host[device] = h;
        g_fault_dev[device] = d;
    }
    return g_fault_dev[device];
}

lvs_status device_fault_check(int device)
{
    if (device < 0 || device >= 64) return LVS_OK;
    volatile uint32_t *h;
    {
        std::lock_guard<std::mutex> lock(g_fault_mu);
        h = g_fault_host[device];
    }
    if (h && *h) {
        *h = 0;
        return set_error(LVS_ERR_TIMEOUT, "blind rotation: a key-chunk copy did not land within about one second; "
                                          "the results of the work since the last check are void");
    }
    return LVS_OK;
}

cudaEvent_t pool_event(lvs_ctx *ctx)
{
    if (!ctx->timing.pool.empty()) {
        cudaEvent_t e = ctx->timing.pool.back();
        ctx->timing.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void timing_collect(lvs_ctx *ctx)
{
    auto &T = ctx->timing;
    if (T.pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : T.pending) {
        float ks = 0.f, br = 0.f;
        if (cudaEventElapsedTime(&ks, p.a, p.b) == cudaSuccess &&
            cudaEventElapsedTime(&br, p.b, p.c) == cudaSuccess) {
            T.stats[1].launches += 1;
            T.stats[1].items += p.items;
            T.stats[1].total_ms += ks;
            T.stats[0].launches += 1;
            T.stats[0].items += p.items;
            T.stats[0].total_ms += br;
        }
        cudaGetLastError();
        T.pool.push_back(p.a);
        T.pool.push_back(p.b);
        T.pool.push_back(p.c);
    }
    T.pending.clear();
}

static void reap_graphs(lvs_ctx *ctx, bool wait)
{
    for (size_t i = 0; i < ctx->graphs.size();) {
        auto &g = ctx->graphs[i];
        if (wait) cudaEventSynchronize(g.done);
        if (cudaEventQuery(g.done) == cudaSuccess) {
            cudaGraphExecDestroy(g.exec);
            cudaEventDestroy(g.done);
            ctx->graphs.erase(ctx->graphs.begin() + i);
        } else {
            cudaGetLastError();
            ++i;
        }
    }
}

// One launch step: the key switch (with the a2 gather) and the blind rotation.
// timed: CUDA events around both kernels; captured: the step is being
// captured into a graph, where the events become event-record nodes (external
// records) that the graph executes in place.
static lvs_status launch_step(lvs_ctx *ctx, const Job *d_jobs, size_t nj, bool timed, bool captured)
{
    nvtxMarkA(("lvs step: " + std::to_string(nj) + " PBS").c_str());
    cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
    auto rec = [&](cudaEvent_t e) {
        return captured ? cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal)
                        : cudaEventRecord(e, ctx->stream);
    };
    if (timed) {
        a = pool_event(ctx); b = pool_event(ctx); c = pool_event(ctx);
        if (!a || !b || !c) return set_error(LVS_ERR_CUDA, "event creation failed");
        LVS_CUDA(rec(a));
    }
    int nks = 0;
    LVS_CUDA(launch_keyswitch_auto(ctx, d_jobs, nj, ctx->ms, ctx->stream, &nks));
    if (timed) LVS_CUDA(rec(b));
    LVS_CUDA(launch_blind_rotate(ctx, d_jobs, nj, ctx->ms, ctx->luts, 0, ctx->stream));
    if (timed) {
        LVS_CUDA(rec(c));
        ctx->timing.pending.push_back({a, b, c, nj});
    }
    ctx->launches += nks + 1;
    return LVS_OK;
}

// A step wider than ctx->max_launch_jobs runs as several launches: bounded
// launch time and modulus-switch scratch.
constexpr size_t kMaxLaunchJobs = 1u << 16;

// End of the launch that starts at job c0 of a step ending at e.  The jobs of
// a step are independent except the two lookups of a refreshed cell (v through
// LUT_V, then h through LUT_V from the swapped key): the second reads the v row
// the first one writes, so both must share a launch, whose key switch gathers
// every input before its blind rotation writes.
static size_t chunk_end(const lvs_ctx *ctx, const std::vector<Job> &jobs, size_t c0, size_t e)
{
    size_t c1 = std::min(e, c0 + ctx->max_launch_jobs);
    if (c1 < e && c1 - c0 > 1) {
        const Job &a = jobs[c1 - 1], &b = jobs[c1];
        if (a.lut == LUT_V && b.lut == LUT_V && a.dst[0] == a.src[0] && a.src[0] == b.src[0] && a.src[1] == b.src[1])
            --c1;
    }
    return c1;
}

lvs_status run_steps(lvs_ctx *ctx, const std::vector<Job> &jobs, const std::vector<size_t> &off, bool use_graph)
{
    size_t widest = 0;
    for (size_t s = 0; s + 1 < off.size(); ++s) widest = std::max(widest, off[s + 1] - off[s]);
    widest = std::min(widest, ctx->max_launch_jobs);
    if (jobs.empty()) return LVS_OK;
    // NVTX range around the whole run (visible to nsys / ncu when attached; a
    // no-op otherwise)
    struct Range {
        Range(size_t steps) { nvtxRangePushA(("lvs wavefront: " + std::to_string(steps) + " steps").c_str()); }
        ~Range() { nvtxRangePop(); }
    } range(off.size() - 1);
    reap_graphs(ctx, false);
    lvs_status st = ensure_scratch(ctx, jobs.size(), widest);
    if (st != LVS_OK) return st;
    LVS_CUDA(cudaMemcpyAsync(ctx->jobs, jobs.data(), jobs.size() * sizeof(Job), cudaMemcpyHostToDevice,
                             ctx->stream));
    const bool timed = ctx->timing.enabled;
    // graphs need a capturable stream (not the legacy default stream)
    if (use_graph && ctx->stream != nullptr && off.size() > 2) {
        if (timed) {
            // every event the capture records exists before the capture starts
            size_t nl = 0;
            for (size_t s = 0; s + 1 < off.size(); ++s)
                for (size_t c0 = off[s]; c0 < off[s + 1]; c0 = chunk_end(ctx, jobs, c0, off[s + 1])) ++nl;
            while (ctx->timing.pool.size() < 3 * nl) {
                cudaEvent_t e = nullptr;
                if (cudaEventCreate(&e) != cudaSuccess) return set_error(LVS_ERR_CUDA, "event creation failed");
                ctx->timing.pool.push_back(e);
            }
        }
        cudaGraph_t graph = nullptr;
        LVS_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        lvs_status lst = LVS_OK;
        for (size_t s = 0; s + 1 < off.size() && lst == LVS_OK; ++s)
            for (size_t c0 = off[s], c1; c0 < off[s + 1] && lst == LVS_OK; c0 = c1) {
                c1 = chunk_end(ctx, jobs, c0, off[s + 1]);
                lst = launch_step(ctx, ctx->jobs + c0, c1 - c0, timed, true);
            }
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
        if (lst != LVS_OK) { if (graph) cudaGraphDestroy(graph); return lst; }
        if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return cuda_error(ce, "cudaGraphInstantiate");
        ce = cudaGraphLaunch(exec, ctx->stream);
        if (ce != cudaSuccess) { cudaGraphExecDestroy(exec); return cuda_error(ce, "cudaGraphLaunch"); }
        cudaEvent_t done = nullptr;
        LVS_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        LVS_CUDA(cudaEventRecord(done, ctx->stream));
        ctx->graphs.push_back({exec, done});
    } else {
        for (size_t s = 0; s + 1 < off.size(); ++s)
            for (size_t c0 = off[s], c1; c0 < off[s + 1]; c0 = c1) {
                c1 = chunk_end(ctx, jobs, c0, off[s + 1]);
                st = launch_step(ctx, ctx->jobs + c0, c1 - c0, timed, false);
                if (st != LVS_OK) return st;
            }
    }
    ctx->pbs_done += jobs.size();
    return LVS_OK;
}

}  // namespace lvs

using namespace lvs;

extern "C" {

lvs_status lvs_ctx_create(const lvs_server_key *sk, int device, void *stream, lvs_ctx **out)
{
    if (!sk || !out) return set_error(LVS_ERR_ARG, "lvs_ctx_create: NULL argument");
    lvs_status st = device_ok(device);
    if (st != LVS_OK) return st;
    LVS_CUDA(cudaSetDevice(device));
    lvs_ctx *ctx = new (std::nothrow) lvs_ctx;
    if (!ctx) return set_error(LVS_ERR_OOM, "lvs_ctx_create: host allocation failed");
    ctx->P = sk->P;
    ctx->device = device;
    auto fail = [&](lvs_status s) { lvs_ctx_free(ctx); return s; };
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(set_error(LVS_ERR_CUDA, "stream creation failed"));
        ctx->own_stream = true;
    }
    const uint32_t N = ctx->P.p.N, n = ctx->P.p.n;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    dev::PrimeConsts pc;
    make_prime_consts(pc);
    cudaError_t e = upload_prime_consts(pc);
    if (e == cudaSuccess) e = prepare_kernels(N);
    if (e != cudaSuccess) return fail(cuda_error(e, "kernel setup"));
    ctx->br_grid = std::max(1, ctx->num_sms * std::max(1, br_blocks_per_sm(N)));
    ctx->fault_dev = device_fault_word(device);
    // three-CTA blind rotation for launches that leave SMs idle: by default up
    // to one ciphertext per three SMs (lvs_ctx_autotune measures the crossover)
    ctx->br_clusters = br_cluster_capacity(N);
    ctx->br_split_max = ctx->br_clusters > 0 ? (size_t)(ctx->num_sms / 3) : 0;
    ctx->max_launch_jobs = kMaxLaunchJobs;

    std::vector<uint32_t> tw;
    make_twiddles(N, tw);
    std::vector<uint8_t> luts;
    make_luts(luts);
    const size_t bsk_ntt = bsk_ntt_words(n, N);
    if (cudaMalloc((void **)&ctx->tw, tw.size() * 4) != cudaSuccess ||
        cudaMalloc((void **)&ctx->luts, luts.size()) != cudaSuccess ||
        cudaMalloc((void **)&ctx->ksk, sk->ksk.size() * 8) != cudaSuccess ||
        cudaMalloc((void **)&ctx->ksk_colsum, ((size_t)n + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&ctx->bsk_ntt, bsk_ntt * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(LVS_ERR_OOM, "device allocation of the server key failed"));
    }
    uint64_t *coef = nullptr;
    if (cudaMalloc((void **)&coef, sk->bsk.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        return fail(set_error(LVS_ERR_OOM, "device allocation of the key staging buffer failed"));
    }
    e = cudaMemcpyAsync(ctx->tw, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->luts, luts.data(), luts.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->ksk, sk->ksk.data(), sk->ksk.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_ksk_colsum(ctx, ctx->stream);
    if (e == cudaSuccess) {
        // tensor-core key switch for large launches (optional: without it the
        // kernel path serves every launch size)
        if (ks_gemm_init(ctx) == LVS_OK && ctx->ks_gemm) ctx->ks_gemm_min = 1024;
        else cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(coef, sk->bsk.data(), sk->bsk.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    uint32_t mont[3][2];
    make_mont(N, mont);
    if (e == cudaSuccess) e = launch_bsk_to_ntt_count(N, coef, n, ctx->bsk_ntt, ctx->tw, mont, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(coef);
    if (e != cudaSuccess) return fail(cuda_error(e, "server key upload / conversion"));
    *out = ctx;
    return LVS_OK;
}

void lvs_ctx_free(lvs_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream || ctx->own_stream) cudaStreamSynchronize(ctx->stream);
    reap_graphs(ctx, true);
    timing_collect(ctx);
    for (auto e : ctx->timing.pool) cudaEventDestroy(e);
    cudaFree(ctx->bsk_ntt);
    cudaFree(ctx->ksk);
    cudaFree(ctx->ksk_colsum);
    ks_gemm_free(ctx);
    cudaFree(ctx->tw);
    cudaFree(ctx->luts);
    cudaFree(ctx->bsk_fft);
    cudaFree(ctx->fft_tw);
    if (ctx->ms) cudaFree(ctx->ms);
    if (ctx->jobs) cudaFree(ctx->jobs);
    if (ctx->ks_part) cudaFree(ctx->ks_part);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

lvs_status lvs_ctx_synchronize(lvs_ctx *ctx)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_synchronize: NULL context");
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    LVS_CUDA(cudaStreamSynchronize(ctx->stream));
    reap_graphs(ctx, true);
    return device_fault_check(ctx->device);
}

lvs_status lvs_ctx_set_timing(lvs_ctx *ctx, int enable)
{
    if (!ctx) return set_error(LVS_ERR_ARG, "lvs_ctx_set_timing: NULL context");
    std::lock_guard<std::mutex> lock(ctx->mu);
    timing_collect(ctx);
    ctx->timing.enabled = enable != 0;
    if (enable) {
        ctx->timing.stats[0] = lvs_kernel_stats{};
        ctx->timing.stats[1] = lvs_kernel_stats{};
        // events for the calls that create none themselves (the allocation-free entry point)
        while (ctx->timing.pool.size() < kTimingPoolEvents) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return set_error(LVS_ERR_CUDA, "lvs_ctx_set_timing: event creation failed");
            ctx->timing.pool.push_back(e);
        }
    }
    return LVS_OK;
}

lvs_status lvs_ctx_kernel_stats(lvs_ctx *ctx, int kind, lvs_kernel_stats *out)
{
    if (!ctx || !out || kind < 0 || kind > 1) return set_error(LVS_ERR_ARG, "lvs_ctx_kernel_stats: bad argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    timing_collect(ctx);
    *out = ctx->timing.stats[kind];
    return LVS_OK;
}

lvs_status lvs_ctx_pbs_count(lvs_ctx *ctx, uint64_t *out)
{
    if (!ctx || !out) return set_error(LVS_ERR_ARG, "lvs_ctx_pbs_count: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *out = ctx->pbs_done;
    return LVS_OK;
}

lvs_status lvs_ctx_launch_count(lvs_ctx *ctx, uint64_t *out)
{
    if (!ctx || !out) return set_error(LVS_ERR_ARG, "lvs_ctx_launch_count: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    *out = ctx->launches;
    return LVS_OK;
}

lvs_status lvs_pbs_batch_device(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride, const uint8_t *d_lut,
                                uint64_t *d_out, size_t out_stride, size_t count)
{
    if (!ctx || (count && (!d_in || !d_lut || !d_out)))
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device: NULL argument");
    const size_t big = ctx->P.big();
    if (in_stride < big + 1 || out_stride < big + 1)
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device: stride smaller than k*N+1");
    if (count == 0) return LVS_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    const size_t chunk = 1u << 16;
    for (size_t c0 = 0; c0 < count; c0 += chunk) {
        const size_t nc = std::min(chunk, count - c0);
        std::vector<Job> jobs(nc);
        for (size_t i = 0; i < nc; ++i) {
            Job &J = jobs[i];
            memset(&J, 0, sizeof(J));
            J.src[0] = d_in + (c0 + i) * in_stride;
            J.coef[0] = 1;
            J.kind = JOB_STORE;
            J.dst[0] = d_out + (c0 + i) * out_stride;
        }
        lvs_status st = ensure_scratch(ctx, nc, nc);
        if (st != LVS_OK) return st;
        LVS_CUDA(cudaMemcpyAsync(ctx->jobs, jobs.data(), nc * sizeof(Job), cudaMemcpyHostToDevice, ctx->stream));
        cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
        const bool timed = ctx->timing.enabled;
        if (timed) {
            a = pool_event(ctx); b = pool_event(ctx); c = pool_event(ctx);
            if (!a || !b || !c) return set_error(LVS_ERR_CUDA, "event creation failed");
            LVS_CUDA(cudaEventRecord(a, ctx->stream));
        }
        int nks = 0;
        LVS_CUDA(launch_keyswitch_auto(ctx, ctx->jobs, nc, ctx->ms, ctx->stream, &nks));
        if (timed) LVS_CUDA(cudaEventRecord(b, ctx->stream));
        LVS_CUDA(launch_blind_rotate(ctx, ctx->jobs, nc, ctx->ms, d_lut + c0 * 16, 1, ctx->stream));
        if (timed) {
            LVS_CUDA(cudaEventRecord(c, ctx->stream));
            ctx->timing.pending.push_back({a, b, c, nc});
        }
        ctx->pbs_done += nc;
        ctx->launches += nks + 1;
    }
    return LVS_OK;
}

lvs_status lvs_keyswitch_batch_device(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride, uint32_t *d_out,
                                      size_t count)
{
    if (!ctx || (count && (!d_in || !d_out))) return set_error(LVS_ERR_ARG, "lvs_keyswitch_batch_device: NULL argument");
    if (in_stride < (size_t)ctx->P.big() + 1) return set_error(LVS_ERR_ARG, "lvs_keyswitch_batch_device: bad stride");
    if (count == 0) return LVS_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::vector<Job> jobs(count);
    for (size_t i = 0; i < count; ++i) {
        memset(&jobs[i], 0, sizeof(Job));
        jobs[i].src[0] = d_in + i * in_stride;
        jobs[i].coef[0] = 1;
    }
    lvs_status st = ensure_scratch(ctx, count, count);
    if (st != LVS_OK) return st;
    LVS_CUDA(cudaMemcpyAsync(ctx->jobs, jobs.data(), count * sizeof(Job), cudaMemcpyHostToDevice, ctx->stream));
    int nks = 0;
    LVS_CUDA(launch_keyswitch_auto(ctx, ctx->jobs, count, d_out, ctx->stream, &nks));
    ctx->launches += nks;
    return LVS_OK;
}

lvs_status lvs_poly_mul_device(lvs_ctx *ctx, const int32_t *d_dig, const uint64_t *d_poly, uint64_t *d_out,
                               size_t count)
{
    if (!ctx || (count && (!d_dig || !d_poly || !d_out))) return set_error(LVS_ERR_ARG, "lvs_poly_mul_device: NULL argument");
    if (count == 0) return LVS_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    const uint32_t N = ctx->P.p.N;
    uint32_t *tmp = nullptr;
    if (cudaMallocAsync((void **)&tmp, bsk_ntt_words((uint32_t)count, N) * 4, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LVS_ERR_OOM, "lvs_poly_mul_device: scratch allocation failed");
    }
    uint32_t mont[3][2];
    make_mont(N, mont);
    cudaError_t e = launch_bsk_to_ntt_count(N, d_poly, (uint32_t)count, tmp, ctx->tw, mont, ctx->stream);
    if (e == cudaSuccess) e = launch_poly_mul(ctx, d_dig, tmp, d_out, count, ctx->stream);
    cudaFreeAsync(tmp, ctx->stream);
    ctx->launches += 2;
    if (e != cudaSuccess) return cuda_error(e, "lvs_poly_mul_device");
    return LVS_OK;
}

}  // extern "C"
