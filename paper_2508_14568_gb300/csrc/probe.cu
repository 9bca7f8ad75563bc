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
#include "ntt.cuh"

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

// Achievable rates of the blind rotation's arithmetic, in the form the NTT
// runs it: a stream of Shoup products (MODE 0) and a stream of complete lazy
// forward butterflies (MODE 1: reduction, product, two additions, with the run-time
// zero of the kernel's butterflies).  Each thread holds 32 independent values and
// 16 twiddle pairs in registers and runs radix-2 stages of 16 butterflies, so no
// address arithmetic enters the loop.  768 threads, one CTA per SM.
constexpr int kModThreads = 768;
constexpr int kModIters = 256;

template <int MODE>
__global__ void __launch_bounds__(kModThreads) k_probe_modmul(uint32_t *out, long long *cycles, const uint2 *tw,
                                                              uint32_t p, uint32_t z)
{
    uint32_t v[32], w[16], ws[16];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = (threadIdx.x * 32u + i) % (2 * p);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint2 t = tw[(threadIdx.x + i) & 1023];
        w[i] = t.x;
        ws[i] = t.y;
    }
    const uint32_t p2 = 2 * p, p2z = p2 + z;
    __syncthreads();
    const long long t0 = clock64();
#pragma unroll 1
    for (int it = 0; it < kModIters; ++it) {
#pragma unroll
        for (int s = 0; s < 5; ++s) {
            const int h = 16 >> s;
#pragma unroll
            for (int g = 0; g < (1 << s); ++g) {
                const int ti = ((1 << s) + g) & 15;
#pragma unroll
                for (int j = 0; j < h; ++j) {
                    uint32_t &a = v[g * 2 * h + j], &b = v[g * 2 * h + j + h];
                    if (MODE == 0) {
                        b = dev::opaque(dev::mul_shoup(w[ti], ws[ti], b, p));
                        a = a + z;
                    } else {
                        const uint32_t x = dev::csubz(a, p2, z);
                        const uint32_t t = dev::opaque(dev::mul_shoup(w[ti], ws[ti], b, p));
                        a = x + t + z;
                        b = x + p2z - t;
                    }
                }
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 32; ++i) acc += v[i];
    out[(size_t)blockIdx.x * kModThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Ceilings of the blind rotation's key product.  MODE 0: 32x32 -> 64-bit
// multiply-accumulates (the Montgomery sums of the key product), 16 independent
// accumulators per thread.  MODE 1: L2 -> SM reads in the key product's shape:
// 384 threads, each reading its 32 bytes (two 16-byte loads) of each of the 16
// chunks of a 192 KB row, all CTAs on the same row at the same time, rows in
// order through a buffer that stays in L2.  One CTA per SM; thread 0 times the
// loop with the SM clock counter between barriers.
constexpr int kKpThreads = 384;
constexpr int kKpWideIters = 2048;
constexpr int kKpRows = 500;                             // 500 x 192 KB = 96 MB < L2
constexpr int kKpRowU4 = 16 * kKpThreads * 2;            // uint4 per row
constexpr int kKpRowReads = 1000;

template <int MODE>
__global__ void __launch_bounds__(kKpThreads, 1)
k_probe_keyprod(const uint4 *__restrict__ rows, uint32_t *out, long long *cycles, uint32_t seed)
{
    const int tid = threadIdx.x;
    uint32_t s = 0;
    __syncthreads();
    const long long t0 = clock64();
    if (MODE == 0) {
        uint64_t acc[16];
        uint32_t a[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) { acc[i] = tid + i; a[i] = seed + tid * 7u + i * 13u; }
        const uint32_t b = seed | 1u;
#pragma unroll 1
        for (int it = 0; it < kKpWideIters; ++it) {
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] += (uint64_t)a[i] * b;
#pragma unroll
            for (int i = 0; i < 16; ++i) a[i] = dev::opaque(a[i]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) s ^= (uint32_t)acc[i] ^ (uint32_t)(acc[i] >> 32);
    } else {
#pragma unroll 1
        for (int it = 0; it < kKpRowReads; ++it) {
            const uint4 *kp = rows + (size_t)(it % kKpRows) * kKpRowU4 + tid * 2;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint4 x = __ldg(kp + q * kKpThreads * 2), y = __ldg(kp + q * kKpThreads * 2 + 1);
                s += x.x ^ x.y ^ x.z ^ x.w ^ y.x ^ y.y ^ y.z ^ y.w;
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    out[(size_t)blockIdx.x * kKpThreads + tid] = s;
    if (tid == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace lvs

using namespace lvs;

extern "C" lvs_status lvs_probe_modmul(int device, double *shoup_per_sm_clk, double *butterfly_per_sm_clk)
{
    if (!shoup_per_sm_clk || !butterfly_per_sm_clk) return set_error(LVS_ERR_ARG, "lvs_probe_modmul: NULL argument");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return set_error(LVS_ERR_CUDA, "lvs_probe_modmul: no such CUDA device");
    }
    LVS_CUDA(cudaSetDevice(device));
    int sms = 0;
    LVS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const uint32_t p = kPrime[0];
    std::vector<uint2> htw(1024);
    for (uint32_t i = 0; i < 1024; ++i) {
        const uint32_t w = (uint32_t)((1234567ull * (i + 1)) % p);
        htw[i] = make_uint2(w, (uint32_t)(((uint64_t)w << 32) / p));
    }
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    uint2 *tw = nullptr;
    if (cudaMalloc((void **)&out, (size_t)sms * kModThreads * 4) != cudaSuccess ||
        cudaMalloc((void **)&cyc, (size_t)sms * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void **)&tw, htw.size() * sizeof(uint2)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(out);
        cudaFree(cyc);
        return set_error(LVS_ERR_OOM, "lvs_probe_modmul: device allocation failed");
    }
    cudaError_t e = cudaMemcpy(tw, htw.data(), htw.size() * sizeof(uint2), cudaMemcpyHostToDevice);
    double rate[2] = {0, 0};
    std::vector<long long> h(sms);
    void (*kern[2])(uint32_t *, long long *, const uint2 *, uint32_t, uint32_t) = {k_probe_modmul<0>,
                                                                                   k_probe_modmul<1>};
    for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
        e = cudaFuncSetAttribute(kern[v], cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
            kern[v]<<<sms, kModThreads, kProbeSmem>>>(out, cyc, tw, p, 0u);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sms * sizeof(long long), cudaMemcpyDeviceToHost);
        }
        if (e == cudaSuccess) {
            std::sort(h.begin(), h.end());
            const double ops = (double)kModThreads * kModIters * 5 * 16;   // products or butterflies
            rate[v] = ops / (double)h[sms / 2];
        }
    }
    cudaFree(out);
    cudaFree(cyc);
    cudaFree(tw);
    if (e != cudaSuccess) return cuda_error(e, "lvs_probe_modmul");
    *shoup_per_sm_clk = rate[0];
    *butterfly_per_sm_clk = rate[1];
    return LVS_OK;
}

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

extern "C" lvs_status lvs_probe_key_product(int device, double *wide_per_sm_clk, double *l2_bytes_per_sm_clk)
{
    if (!wide_per_sm_clk || !l2_bytes_per_sm_clk) return set_error(LVS_ERR_ARG, "lvs_probe_key_product: NULL argument");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return set_error(LVS_ERR_CUDA, "lvs_probe_key_product: no such CUDA device");
    }
    LVS_CUDA(cudaSetDevice(device));
    int sms = 0;
    LVS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    uint32_t *out = nullptr;
    long long *cyc = nullptr;
    uint4 *rows = nullptr;
    const size_t row_bytes = (size_t)kKpRows * kKpRowU4 * sizeof(uint4);
    if (cudaMalloc((void **)&out, (size_t)sms * kKpThreads * 4) != cudaSuccess ||
        cudaMalloc((void **)&cyc, (size_t)sms * sizeof(long long)) != cudaSuccess ||
        cudaMalloc((void **)&rows, row_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(out);
        cudaFree(cyc);
        return set_error(LVS_ERR_OOM, "lvs_probe_key_product: device allocation failed");
    }
    cudaError_t e = cudaMemset(rows, 0x5a, row_bytes);
    double rate[2] = {0, 0};
    std::vector<long long> h(sms);
    void (*kern[2])(const uint4 *, uint32_t *, long long *, uint32_t) = {k_probe_keyprod<0>, k_probe_keyprod<1>};
    for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up (and fills L2)
            kern[v]<<<sms, kKpThreads>>>(rows, out, cyc, 5u + rep);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpy(h.data(), cyc, sms * sizeof(long long), cudaMemcpyDeviceToHost);
        }
        if (e == cudaSuccess) {
            std::sort(h.begin(), h.end());
            const double work = v == 0 ? (double)kKpThreads * kKpWideIters * 16       // multiply-accumulates
                                       : (double)kKpRowReads * kKpRowU4 * sizeof(uint4);   // bytes
            rate[v] = work / (double)h[sms / 2];
        }
    }
    cudaFree(out);
    cudaFree(cyc);
    cudaFree(rows);
    if (e != cudaSuccess) return cuda_error(e, "lvs_probe_key_product");
    *wide_per_sm_clk = rate[0];
    *l2_bytes_per_sm_clk = rate[1];
    return LVS_OK;
}
