// Homomorphic readout of a distance (the return of Algorithm algo_complete,
// m + the sum of the last row's horizontal differences, done on ciphertexts).
//
// A result item holds `count` big-LWE ciphertexts of differences in {-1, 0, 1}
// (Z_32 residues times Delta) and a plaintext offset `base`; the distance is
// base + their sum.  Adding the ciphertexts and the trivial encryption of base
// gives one ciphertext of the distance mod 32.  It is the distance itself, with
// the padding bit clear (a valid input of a further bootstrap), while the
// distance stays below 16, hence the limit max(m, n) <= 15.
#include <algorithm>
#include <vector>

#include "lvs_internal.hpp"

namespace lvs {
namespace {

struct SumItem {
    uint64_t first, count;
    int64_t base;
};

// out[q][c] = sum_{r < count_q} in[first_q + r][c] (+ base_q Delta on the body):
// one CTA per item, threads over the k N + 1 words of a row
__global__ void k_result_sum(const uint64_t *__restrict__ in, size_t in_stride, const SumItem *__restrict__ items,
                             uint32_t words, uint64_t *__restrict__ out, size_t out_stride)
{
    const SumItem it = items[blockIdx.x];
    uint64_t *o = out + (size_t)blockIdx.x * out_stride;
    for (uint32_t c = threadIdx.x; c < words; c += blockDim.x) {
        uint64_t s = c + 1 == words ? (uint64_t)it.base << kDeltaLog : 0;
        const uint64_t *p = in + it.first * in_stride + c;
        for (uint64_t r = 0; r < it.count; ++r) s += __ldg(p + r * in_stride);
        o[c] = s;
    }
}

}  // namespace
}  // namespace lvs

using namespace lvs;

extern "C" {

lvs_status lvs_result_sum(lvs_ctx *ctx, const lvs_result *r, lvs_result **out)
{
    if (!ctx || !r || !out) return set_error(LVS_ERR_ARG, "lvs_result_sum: NULL argument");
    if (r->is_eq) return set_error(LVS_ERR_ARG, "lvs_result_sum: an equality result holds no distance");
    if (r->device != ctx->device || r->P.big() != ctx->P.big())
        return set_error(LVS_ERR_ARG, "lvs_result_sum: the result belongs to another context");
    std::vector<SumItem> items(r->items.size());
    for (size_t q = 0; q < items.size(); ++q) {
        const auto &it = r->items[q];
        if (std::max(it.m, it.n) > 15)
            return set_error(LVS_ERR_ARG, "lvs_result_sum: a distance of strings longer than 15 does not fit "
                                          "the 5-bit plaintext with its padding bit");
        items[q] = {it.first, it.count, it.base};
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    LVS_CUDA(cudaSetDevice(ctx->device));
    lvs_result *s = nullptr;
    lvs_status st = make_result(ctx, items.size(), &s);
    if (st != LVS_OK) return st;
    for (size_t q = 0; q < items.size(); ++q) s->items.push_back({r->items[q].m, r->items[q].n, q, 1, 0});
    if (!items.empty()) {
        SumItem *d_items = nullptr;
        cudaError_t e = cudaStreamWaitEvent(ctx->stream, r->done, 0);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&d_items, items.size() * sizeof(SumItem), ctx->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            lvs_result_free(s);
            return e == cudaErrorMemoryAllocation ? set_error(LVS_ERR_OOM, "lvs_result_sum: device allocation failed")
                                                  : cuda_error(e, "lvs_result_sum");
        }
        // pageable source: the call returns once the host array is staged
        e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(SumItem), cudaMemcpyHostToDevice,
                            ctx->stream);
        if (e == cudaSuccess) {
            k_result_sum<<<(unsigned)items.size(), 256, 0, ctx->stream>>>(r->d, r->stride, d_items, ctx->P.big() + 1,
                                                                            s->d, s->stride);
            e = cudaGetLastError();
            ctx->launches += 1;
        }
        cudaFreeAsync(d_items, ctx->stream);
        if (e != cudaSuccess) { lvs_result_free(s); return cuda_error(e, "lvs_result_sum"); }
    }
    if ((st = finish_result(ctx, s)) != LVS_OK) { lvs_result_free(s); return st; }
    *out = s;
    return LVS_OK;
}

}  // extern "C"
