// Issue rate of 32-bit integer multiplies per SM per clock, measured on the
// device (the denominator of the blind rotation's roofline: its work is
// word-size modular multiplications, each a Shoup product of two low-half and
// one high-half 32-bit multiplies).
//
// One CTA of 1024 threads per SM (its unused dynamic shared memory keeps a
// second CTA off the SM) runs 16 or 32 independent multiply chains per thread
// (the faster of the two is kept, so that latency does not hide the issue
// rate);
// thread 0 reads the SM clock counter around the loop (after a barrier on both
// sides), so the rate is in multiplies per SM clock and does not depend on the
// clock frequency the GPU runs at.
#include <algorithm>
#include <vector>

#include "lvs_internal.hpp"

namespace lvs {

constexpr int kProbeThreads = 1024;
constexpr int kProbeIters = 2048;
constexpr int kProbeSmem = 160 << 10;   // more than half an SM's shared memory

template <int MODE, int kChains>
__global__ void __launch_bounds__(kProbeThreads) k_probe_mul(uint32_t *out, long long *cycles, uint32_t seed)
{
    uint32_t a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = seed + threadIdx.x * 7u + i * 13u;
    const uint32_t b = seed | 1u, c = seed ^ 0x9e37u;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            if (MODE == 0) a[i] = a[i] * b + c;                // low half
            else a[i] = __umulhi(a[i], b) + c;                 // high half
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = s;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace lvs

using namespace lvs;

extern "C" lvs_status lvs_probe_int_mul(int device, double *lo_per_sm_clk, double *hi_per_sm_clk)
{
    if (!lo_per_sm_clk || !hi_per_sm_clk) return set_error(LVS_ERR_ARG, "lvs_probe_int_mul: NULL argument");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return set_error(LVS_ERR_CUDA, "lvs_probe_int_mul: no such CUDA device");
    }
    LVS_CUDA(cudaSetDevice(device));
    int sms = 0;
    LVS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc((void **)&out, (size_t)sms * kProbeThreads * 4) != cudaSuccess ||
        cudaMalloc((void **)&cyc, (size_t)sms * sizeof(long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(out);
        return set_error(LVS_ERR_OOM, "lvs_probe_int_mul: device allocation failed");
    }
    double rate[2] = {0, 0};
    cudaError_t e = cudaSuccess;
    std::vector<long long> h(sms);
    // (mode, chains) variants; each runs twice, the first run warms up
    void (*kern[4])(uint32_t *, long long *, uint32_t) = {k_probe_mul<0, 16>, k_probe_mul<0, 32>,
                                                          k_probe_mul<1, 16>, k_probe_mul<1, 32>};
    const int chains[4] = {16, 32, 16, 32};
    for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
        e = cudaFuncSetAttribute(kern[v], cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            kern[v]<<<sms, kProbeThreads, kProbeSmem>>>(out, cyc, 3u + rep);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sms * sizeof(long long), cudaMemcpyDeviceToHost);
        }
        if (e == cudaSuccess) {
            std::sort(h.begin(), h.end());
            const double ops = (double)kProbeThreads * kProbeIters * chains[v];
            rate[v / 2] = std::max(rate[v / 2], ops / (double)h[sms / 2]);
        }
    }
    cudaFree(out);
    cudaFree(cyc);
    if (e != cudaSuccess) return cuda_error(e, "lvs_probe_int_mul");
    *lo_per_sm_clk = rate[0];
    *hi_per_sm_clk = rate[1];
    return LVS_OK;
}
