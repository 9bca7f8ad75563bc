// FP64-FFT variant of the blind rotation, kept beside the exact NTT path as a
// measured alternative (it is not bit-exact: the key and the products are
// rounded to double precision, which adds a small error in the low bits of
// the torus, far below the bootstrap noise).
//
// Negacyclic products through a complex FFT of size M = N/2 ("folding"): a real
// polynomial a of Z[X]/(X^N + 1) is evaluated at the M roots w^(4k+1) of
// X^N + 1 (w = exp(i pi / N)); with c_j = (a_j + i a_{j+M}) w^j,
// a(w^(4k+1)) = sum_j c_j exp(2 pi i j k / M), a size-M DFT.  The other N/2
// roots are the conjugates, so for real polynomials these M values determine
// the product, and the inverse is a_j + i a_{j+M} = w^(-j) (1/M) sum_k A_k
// exp(-2 pi i j k / M).
//
// Forward: decimation in frequency (natural order in, bit-reversed out);
// inverse: decimation in time (bit-reversed in, natural out); the pointwise
// products do not depend on the order, and the key goes through the same
// forward transform.
//
// Kernel layout: one CTA of 256 threads per ciphertext, two CTAs per SM
// (shared memory: accumulator 32 KB + 4 x M complex = 64 KB).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "lvs_internal.hpp"

namespace lvs {
namespace fft {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csubd(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// tables: tw[t] = exp(2 pi i t / M), t < M/2; tws[j] = w^j = exp(i pi j / N), j < M
template <int LOGN>
__device__ __forceinline__ void fft_forward(double2 *x, const double2 *__restrict__ tw, int npoly)
{
    constexpr int M = (1 << LOGN) / 2;
    for (int span = M / 2, step = 1; span >= 1; span >>= 1, step <<= 1) {
        for (int b = threadIdx.x; b < npoly * (M / 2); b += kThreads) {
            const int poly = b / (M / 2), r = b % (M / 2);
            const int blk = r / span, j = r % span;
            double2 *p = x + poly * M + blk * 2 * span + j;
            const double2 u = p[0], v = p[span];
            p[0] = cadd(u, v);
            p[span] = cmul(csubd(u, v), tw[j * step]);
        }
        __syncthreads();
    }
}

template <int LOGN>
__device__ __forceinline__ void fft_inverse(double2 *x, const double2 *__restrict__ tw, int npoly)
{
    constexpr int M = (1 << LOGN) / 2;
    for (int span = 1, step = M / 2; span <= M / 2; span <<= 1, step >>= 1) {
        for (int b = threadIdx.x; b < npoly * (M / 2); b += kThreads) {
            const int poly = b / (M / 2), r = b % (M / 2);
            const int blk = r / span, j = r % span;
            double2 *p = x + poly * M + blk * 2 * span + j;
            double2 w = tw[j * step];
            w.y = -w.y;   // conjugate: exp(-2 pi i t / M)
            const double2 u = p[0], v = cmul(p[span], w);
            p[0] = cadd(u, v);
            p[span] = csubd(u, v);
        }
        __syncthreads();
    }
}

// a (real, exact integers < 2^87 in magnitude) -> a mod 2^64
__device__ __forceinline__ uint64_t torus_of(double v)
{
    const double q = rint(v * 0x1p-64);
    double r = v - q * 0x1p64;          // exact: a multiple of ulp(v) with |r| <= 2^63
    if (r >= 0x1p63) r -= 0x1p64;
    return (uint64_t)(long long)rint(r);
}

// fold + twist a real polynomial (given by its coefficient function) into M complex values
template <int LOGN, class F>
__device__ __forceinline__ void fold(double2 *x, const double2 *__restrict__ tws, F coef)
{
    constexpr int M = (1 << LOGN) / 2;
    for (int j = threadIdx.x; j < M; j += kThreads) x[j] = cmul(make_double2(coef(j), coef(j + M)), tws[j]);
}

// BSK (coefficient domain, [i][slot][N] u64, slot = row * 2 + column) -> FFT domain [i][slot][M]
template <int LOGN>
__global__ void __launch_bounds__(kThreads)
k_bsk_to_fft(const uint64_t *__restrict__ coef, uint32_t count, double2 *__restrict__ out,
             const double2 *__restrict__ tw, const double2 *__restrict__ tws)
{
    constexpr int N = 1 << LOGN, M = N / 2;
    __shared__ double2 x[M];
    const uint32_t i = blockIdx.x, slot = blockIdx.y;
    if (i >= count) return;
    const uint64_t *src = coef + ((size_t)i * 8 + slot) * N;
    fold<LOGN>(x, tws, [&](int t) { return (double)(int64_t)src[t]; });
    __syncthreads();
    fft_forward<LOGN>(x, tw, 1);
    for (int k = threadIdx.x; k < M; k += kThreads) out[((size_t)i * 8 + slot) * M + k] = x[k];
}

template <int LOGN>
struct FftSmem {
    static constexpr int N = 1 << LOGN, M = N / 2;
    static constexpr size_t total = 2 * N * sizeof(uint64_t) + 4 * M * sizeof(double2);
};

// Blind rotation with FP64 FFT products; same jobs, LUT encoding, sample
// extract and epilogue as k_blind_rotate.
template <int LOGN>
__global__ void __launch_bounds__(kThreads, 2)
k_blind_rotate_fft(const Job *__restrict__ jobs, uint32_t njobs, const uint32_t *__restrict__ ms, uint32_t n,
                   const double2 *__restrict__ bsk, const double2 *__restrict__ tw, const double2 *__restrict__ tws,
                   const uint8_t *__restrict__ luts, int lut_per_job, uint32_t base_log)
{
    constexpr int N = 1 << LOGN, M = N / 2;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *acc = reinterpret_cast<uint64_t *>(smem_raw);            // [2][N]
    double2 *F = reinterpret_cast<double2 *>(smem_raw + 2 * N * sizeof(uint64_t));   // [4][M]
    const int tid = threadIdx.x;
    const uint32_t B = 1u << base_log, hB = B >> 1;
    const uint32_t shift = 64 - 2 * base_log;
    const double invM = 1.0 / M;

    for (uint32_t job = blockIdx.x; job < njobs; job += gridDim.x) {
        const Job J = jobs[job];
        const uint32_t *msj = ms + (size_t)job * (n + 1);
        const uint8_t *lp = luts + (lut_per_job ? (size_t)job * 16 : (size_t)J.lut * 16);
        const uint32_t b = __ldg(msj + n);
        for (int e = tid; e < N; e += kThreads) {
            // X^{-b} v' at e: index (e + b) mod 2N of the negacyclic extension of v'
            const uint32_t idx = (e + b) & (2 * N - 1), t = idx & (N - 1), box = N / 16;
            uint64_t v = t < N - box / 2 ? (uint64_t)(lp[(t + box / 2) / box] & 31u) << kDeltaLog
                                         : 0 - ((uint64_t)(lp[0] & 31u) << kDeltaLog);
            acc[e] = 0;
            acc[N + e] = idx >= (uint32_t)N ? 0 - v : v;
        }
        __syncthreads();
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t a = __ldg(msj + i);
            if (a == 0) continue;
            // balanced digits of X^a ACC - ACC, folded and twisted: F[2j + lev-1]
            for (int jj = tid; jj < 2 * M; jj += kThreads) {
                const int j = jj / M, t = jj % M;
                double dv[2][2];
                for (int h = 0; h < 2; ++h) {
                    const uint32_t e = t + h * M;
                    const uint32_t idx = (e - a) & (2 * N - 1);
                    uint64_t rv = acc[j * N + (idx & (N - 1))];
                    if (idx >= (uint32_t)N) rv = 0 - rv;
                    const uint64_t x = rv - acc[j * N + e];
                    const uint64_t vv = (x + (1ull << (shift - 1))) >> shift;
                    const uint32_t u2 = (uint32_t)vv & (B - 1), u1 = (uint32_t)(vv >> base_log) & (B - 1);
                    const uint32_t c2 = u2 >= hB;
                    const uint32_t r1 = u1 + c2;
                    dv[0][h] = (double)((int32_t)r1 - (int32_t)((r1 >= hB) * B));
                    dv[1][h] = (double)((int32_t)u2 - (int32_t)(c2 * B));
                }
                F[(2 * j + 0) * M + t] = cmul(make_double2(dv[0][0], dv[0][1]), tws[t]);
                F[(2 * j + 1) * M + t] = cmul(make_double2(dv[1][0], dv[1][1]), tws[t]);
            }
            __syncthreads();
            fft_forward<LOGN>(F, tw, 4);
            // pointwise: out_c = sum_r F_r * G[i][r*2+c]
            const double2 *G = bsk + (size_t)i * 8 * M;
            for (int k = tid; k < M; k += kThreads) {
                double2 o0 = make_double2(0, 0), o1 = make_double2(0, 0);
                for (int r = 0; r < 4; ++r) {
                    const double2 f = F[r * M + k];
                    o0 = cadd(o0, cmul(f, __ldg(G + (r * 2 + 0) * M + k)));
                    o1 = cadd(o1, cmul(f, __ldg(G + (r * 2 + 1) * M + k)));
                }
                F[0 * M + k] = o0;
                F[1 * M + k] = o1;
            }
            __syncthreads();
            fft_inverse<LOGN>(F, tw, 2);
            // untwist, unfold, round mod 2^64, accumulate
            for (int jj = tid; jj < 2 * M; jj += kThreads) {
                const int c = jj / M, t = jj % M;
                double2 w = tws[t];
                w.y = -w.y;
                const double2 z = cmul(F[c * M + t], w);
                acc[c * N + t] += torus_of(z.x * invM);
                acc[c * N + t + M] += torus_of(z.y * invM);
            }
            __syncthreads();
        }
        uint64_t *o0 = J.dst[0];
        uint64_t *o1 = J.dst[1];
        for (int u = tid; u <= N; u += kThreads) {
            const uint64_t val = u == N ? acc[N] : (u == 0 ? acc[0] : 0 - acc[N - u]);
            if (J.kind == JOB_CELL) {
                const uint64_t vold = o0[u], hold = o1[u];
                const uint64_t vn = val - hold, hn = val - vold;
                o0[u] = vn;
                o1[u] = hn;
                if (J.tapsel) J.tap[u] = J.tapsel == 1 ? vn : hn;
            } else {
                o0[u] = val;
                if (J.tapsel) J.tap[u] = val;
            }
        }
        __syncthreads();
    }
}


template <int LOGN>
static cudaError_t set_attrs()
{
    return cudaFuncSetAttribute(k_blind_rotate_fft<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FftSmem<LOGN>::total);
}

template <int LOGN>
static int blocks_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blind_rotate_fft<LOGN>, kThreads,
                                                      FftSmem<LOGN>::total) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, nb);
}

}  // namespace fft

// host tables: tw[t] = exp(2 pi i t / M) for t < M/2, then tws[j] = exp(i pi j / N) for j < M
static void make_fft_tables(uint32_t N, std::vector<double> &out)
{
    const uint32_t M = N / 2;
    const double pi = 3.14159265358979323846264338327950288;
    out.clear();
    for (uint32_t t = 0; t < M / 2; ++t) {
        out.push_back(std::cos(2.0 * pi * t / M));
        out.push_back(std::sin(2.0 * pi * t / M));
    }
    for (uint32_t j = 0; j < M; ++j) {
        out.push_back(std::cos(pi * j / N));
        out.push_back(std::sin(pi * j / N));
    }
}

}  // namespace lvs

using namespace lvs;

lvs_status lvs_ctx_prepare_fft64(lvs_ctx *ctx, const lvs_server_key *sk)
{
    if (!ctx || !sk) return set_error(LVS_ERR_ARG, "lvs_ctx_prepare_fft64: NULL argument");
    const auto &p = ctx->P.p;
    if (memcmp(&sk->P.p, &p, sizeof(p)) != 0)
        return set_error(LVS_ERR_ARG, "lvs_ctx_prepare_fft64: server key parameters differ from the context's");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->bsk_fft) return LVS_OK;
    LVS_CUDA(cudaSetDevice(ctx->device));
    const uint32_t N = p.N, M = N / 2, n = p.n;
    std::vector<double> tab;
    make_fft_tables(N, tab);
    const size_t fft_words = (size_t)n * 8 * M * 2;   // doubles
    double *tw = nullptr, *bsk = nullptr;
    uint64_t *coef = nullptr;
    if (cudaMalloc((void **)&tw, tab.size() * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&bsk, fft_words * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&coef, sk->bsk.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tw);
        cudaFree(bsk);
        cudaFree(coef);
        return set_error(LVS_ERR_OOM, "lvs_ctx_prepare_fft64: device allocation of the FFT key failed");
    }
    const double2 *t2 = reinterpret_cast<const double2 *>(tw);
    const double2 *ts2 = t2 + M / 2;
    cudaError_t e = cudaMemcpyAsync(tw, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(coef, sk->bsk.data(), sk->bsk.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        dim3 grid(n, 8);
        if (N == 2048)
            fft::k_bsk_to_fft<11><<<grid, fft::kThreads, 0, ctx->stream>>>(coef, n, reinterpret_cast<double2 *>(bsk), t2, ts2);
        else
            fft::k_bsk_to_fft<9><<<grid, fft::kThreads, 0, ctx->stream>>>(coef, n, reinterpret_cast<double2 *>(bsk), t2, ts2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = N == 2048 ? fft::set_attrs<11>() : fft::set_attrs<9>();
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(coef);
    if (e != cudaSuccess) {
        cudaFree(tw);
        cudaFree(bsk);
        return cuda_error(e, "lvs_ctx_prepare_fft64: key conversion");
    }
    ctx->fft_tw = tw;
    ctx->bsk_fft = bsk;
    ctx->fft_grid = ctx->num_sms * (N == 2048 ? fft::blocks_per_sm<11>() : fft::blocks_per_sm<9>());
    return LVS_OK;
}

lvs_status lvs_pbs_batch_device_fft64(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride, const uint8_t *d_lut,
                                      uint64_t *d_out, size_t out_stride, size_t count)
{
    if (!ctx || (count && (!d_in || !d_lut || !d_out)))
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device_fft64: NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->bsk_fft)
        return set_error(LVS_ERR_STATE, "lvs_pbs_batch_device_fft64: call lvs_ctx_prepare_fft64 first");
    const auto &p = ctx->P.p;
    const size_t big = ctx->P.big();
    if (in_stride < big + 1 || out_stride < big + 1)
        return set_error(LVS_ERR_ARG, "lvs_pbs_batch_device_fft64: stride smaller than k*N+1");
    if (count == 0) return LVS_OK;
    LVS_CUDA(cudaSetDevice(ctx->device));
    const uint32_t M = p.N / 2;
    const double2 *t2 = reinterpret_cast<const double2 *>(ctx->fft_tw);
    const double2 *ts2 = t2 + M / 2;
    const double2 *bsk = reinterpret_cast<const double2 *>(ctx->bsk_fft);
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
        int nks = 0;
        LVS_CUDA(launch_keyswitch_auto(ctx, ctx->jobs, nc, ctx->ms, ctx->stream, &nks));
        const unsigned grid = (unsigned)std::min<size_t>(nc, (size_t)ctx->fft_grid);
        if (p.N == 2048)
            fft::k_blind_rotate_fft<11><<<grid, fft::kThreads, fft::FftSmem<11>::total, ctx->stream>>>(
                ctx->jobs, (uint32_t)nc, ctx->ms, p.n, bsk, t2, ts2, d_lut + c0 * 16, 1, p.pbs_base_log);
        else
            fft::k_blind_rotate_fft<9><<<grid, fft::kThreads, fft::FftSmem<9>::total, ctx->stream>>>(
                ctx->jobs, (uint32_t)nc, ctx->ms, p.n, bsk, t2, ts2, d_lut + c0 * 16, 1, p.pbs_base_log);
        LVS_CUDA(cudaGetLastError());
        ctx->pbs_done += nc;
        ctx->launches += nks + 1;
    }
    return LVS_OK;
}
