// Allocation-free variant of the device-pointer PBS entry point.
//
// Some callers cannot allocate device memory at call time: code that runs
// under a memory budget fixed up front (a server that reserves all of its
// device memory at start-up and must not fail mid-request), real-time paths
// where cudaMalloc's implicit synchronisation and latency are not acceptable,
// and hosts whose allocator is owned by another framework.  For them,
// lvs_pbs_batch_device_noalloc keeps its scratch -- the job descriptors and
// the modulus-switched masks that pass from the key-switch kernel to the
// blind-rotation kernel -- in one fixed-size array in device memory that the
// library declares at file scope.  Every GPU that loads the library holds that
// array (LVS_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// The host code never uses the array's name as a device address: the address
// is looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <mutex>

#include "lvs_internal.hpp"

namespace lvs {

static __device__ __align__(256) unsigned char g_noalloc_scratch[LVS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// one job per input row: PBS of row i of `in`, written to row i of `out`
__global__ void k_fill_raw_jobs(Job *jobs, const uint64_t *in, size_t in_stride, uint64_t *out, size_t out_stride,
                                uint32_t count)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Job J;
    memset(&J, 0, sizeof(J));
    J.src[0] = in + (size_t)i * in_stride;
    J.coef[0] = 1;
    J.kind = JOB_STORE;
    J.dst[0] = out + (size_t)i * out_stride;
    jobs[i] = J;
}

lvs_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return set_error(LVS_ERR_ARG, "noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_error(e, "noalloc: cudaGetSymbolAddress of the static scratch");
        g_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[device];
    return LVS_OK;
}

}  // namespace
}  // namespace lvs

using namespace lvs;

extern "C" lvs_status lvs_pbs_batch_device_noalloc(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride,
                                                   const uint8_t *d_lut, uint64_t *d_out, size_t out_stride,
                                                   size_t count)
{
    if (!ctx || (count && (!d_in || !d_lut || !d_out)))
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device_noalloc: NULL argument");
    const size_t big = ctx->P.big();
    if (in_stride < big + 1 || out_stride < big + 1)
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device_noalloc: stride smaller than k*N+1");
    // scratch layout: [count jobs][pad to 256][count * (n+1) u32 masks]
    const size_t jobs_bytes = (count * sizeof(Job) + 255) & ~(size_t)255;
    const size_t ms_bytes = count * ((size_t)ctx->P.p.n + 1) * sizeof(uint32_t);
    if (jobs_bytes + ms_bytes > (size_t)LVS_NOALLOC_SCRATCH_BYTES) {
        const size_t per = sizeof(Job) + ((size_t)ctx->P.p.n + 1) * sizeof(uint32_t);
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device_noalloc: " + std::to_string(count) +
                                          " PBS need more than the static scratch of " +
                                          std::to_string(LVS_NOALLOC_SCRATCH_BYTES) + " bytes (at most about " +
                                          std::to_string((LVS_NOALLOC_SCRATCH_BYTES - 256) / per) +
                                          " per call for n = " + std::to_string(ctx->P.p.n) + ")");
    }
    if (count == 0) return LVS_OK;
    std::lock_guard<std::mutex> lock(ctx->mu);   // the settings and counters the batch calls share
    LVS_CUDA(cudaSetDevice(ctx->device));
    unsigned char *base = nullptr;
    lvs_status st = scratch_address(ctx->device, &base);
    if (st != LVS_OK) return st;
    Job *jobs = reinterpret_cast<Job *>(base);
    uint32_t *ms = reinterpret_cast<uint32_t *>(base + jobs_bytes);
    k_fill_raw_jobs<<<(unsigned)((count + 127) / 128), 128, 0, ctx->stream>>>(jobs, d_in, in_stride, d_out, out_stride,
                                                                            (uint32_t)count);
    LVS_CUDA(cudaGetLastError());
    // timing (lvs_ctx_set_timing): only events the context created up front,
    // so that this call creates nothing; with the pool empty the call is not timed
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    const bool timed = ctx->timing.enabled && ctx->timing.pool.size() >= 3;
    if (timed) {
        for (auto &e : ev) { e = ctx->timing.pool.back(); ctx->timing.pool.pop_back(); }
        LVS_CUDA(cudaEventRecord(ev[0], ctx->stream));
    }
    // the key switch without its split form (whose partial sums would need scratch)
    LVS_CUDA(launch_keyswitch_plan(ctx, jobs, count, ms, nullptr, ks_plan(ctx, count), ctx->stream));
    if (timed) LVS_CUDA(cudaEventRecord(ev[1], ctx->stream));
    LVS_CUDA(launch_blind_rotate(ctx, jobs, count, ms, d_lut, 1, ctx->stream));
    if (timed) {
        LVS_CUDA(cudaEventRecord(ev[2], ctx->stream));
        ctx->timing.pending.push_back({ev[0], ev[1], ev[2], count});
    }
    ctx->pbs_done += count;
    ctx->launches += 3;   // kernels launched: job fill, key switch, blind rotation
    return LVS_OK;
}
