// Continuous-batching server: encrypted name-matching / sequence queries are
// admitted while device memory allows, keep their difference-matrix frontier
// on the device, and advance together -- every launch step bootstraps the
// union of the next anti-diagonal work of all admitted queries (Section 6.2:
// cells of one anti-diagonal and different pairs are independent).  Queries
// that arrive while others run join at the next step boundary.
//
// A query is an encrypted string against either an encrypted reference (two
// equality lookups per cell, Algorithm alg_ascii; one for DNA) or a plaintext
// reference held by the server.  For a plaintext reference the query first
// builds the preprocessing table of Section 5 restricted to the symbols that
// occur in the reference (T[sigma][i] = enc(9 EQ(a_i, sigma)), 2 |S| m lookups),
// then needs one lookup per cell.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>

#include "lvs_internal.hpp"

namespace lvs {
namespace {

struct Query {
    uint64_t ticket = 0;
    lvs_ct_string q;                 // copy of the query string (host)
    lvs_ct_string ref;               // copy of the encrypted reference (host), if any
    bool plain = false;
    std::vector<uint8_t> ref_plain;
    std::vector<uint8_t> subset;     // distinct reference symbols (plaintext path)
    std::vector<std::pair<uint32_t, uint32_t>> sym;
    int32_t row_of[256];
    size_t m = 0, n = 0;
    uint32_t C = 2;
    size_t bytes = 0;                // device footprint (arena + result)
    // device state
    Arena A;
    PairRows P;
    size_t tmp = 0, table = 0;       // arena rows of the plaintext-path tables
    long prologue = 0;               // table-building steps (plaintext path)
    long steps = 0;                  // total steps
    long step = 0;                   // next step to run
};

}  // namespace
}  // namespace lvs

struct lvs_server {
    lvs_ctx *ctx = nullptr;
    size_t budget = 0;
    size_t max_active = 0;           // 0: no slot limit
    size_t used = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<lvs::Query *> pending;
    std::vector<lvs::Query *> active;
    struct Done { lvs_status st; std::string msg; lvs_result *r; };
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> known;   // ticket -> 1 while pending/active
    lvs_server_stats stats{};
};

namespace lvs {
namespace {

size_t query_rows(const Query &q)
{
    if (q.plain) return q.m * q.C + q.m + q.n + (q.C == 2 ? 2 : 1) * q.subset.size() * q.m;
    return (q.m + q.n) * q.C + q.m + q.n + (q.C == 2 ? 4 : 2) * q.m;
}

// device setup of an admitted query: arena, uploads, OneMatrix boundary
lvs_status setup(lvs_ctx *ctx, Query &q)
{
    lvs_status st = arena_alloc(ctx, query_rows(q), q.A);
    if (st != LVS_OK) return st;
    PairRows &P = q.P;
    P.m = q.m;
    P.n = q.n;
    P.C = q.C;
    if ((st = plan_refresh(ctx, 0, P)) != LVS_OK) return st;
    size_t r = 0;
    P.x = r; r += q.m * q.C;
    if ((st = upload_string(ctx, &q.q, q.A, P.x)) != LVS_OK) return st;
    if (!q.plain) {
        P.y = r; r += q.n * q.C;
        if ((st = upload_string(ctx, &q.ref, q.A, P.y)) != LVS_OK) return st;
    }
    P.v = r; r += q.m;
    P.h = r; r += q.n;
    const cudaError_t e = launch_fill_trivial(q.A.d, q.A.stride, ctx->P.big(), P.v, q.m + q.n, 1ull << kDeltaLog,
                                              ctx->stream);
    if (e != cudaSuccess) return cuda_error(e, "server fill");
    ctx->launches += (q.m + q.n) ? 1 : 0;
    if (q.plain) {
        if (q.C == 2) { q.tmp = r; r += q.subset.size() * q.m; }
        q.table = r; r += q.subset.size() * q.m;
        P.table = q.A.row(q.table);
        P.table_stride = q.A.stride;
        P.row_of = q.row_of;
        P.plain = q.ref_plain.data();
        q.prologue = (q.m && q.n) ? (long)q.C : 0;
    } else {
        if (q.C == 2) { P.eq1 = r; r += 2 * q.m; }
        P.eq9 = r; r += 2 * q.m;
    }
    q.steps = q.prologue + pair_steps(P);
    q.step = 0;
    return LVS_OK;
}

// jobs of the query's current step
void plan_query(const Query &q, std::vector<Job> &jobs)
{
    if (q.step < q.prologue) {
        // preprocessing table of the reference symbols (Section 5)
        const size_t m = q.m;
        table_step_jobs(
            (int)q.step, q.C, m, q.sym, [&](size_t i, int s) { return q.A.row(q.P.x + i * q.C + s); },
            [&](size_t r, size_t i) { return q.A.row(q.tmp + r * m + i); },
            [&](size_t r, size_t i) { return q.A.row(q.table + r * m + i); }, jobs);
        return;
    }
    plan_pair_step(q.P, q.A, q.step - q.prologue, jobs);
}

lvs_status finish(lvs_server *S, Query &q, lvs_result **out)
{
    lvs_ctx *ctx = S->ctx;
    lvs_result *r = nullptr;
    lvs_status st = make_result(ctx, q.n, &r);
    if (st != LVS_OK) return st;
    r->items.push_back({q.m, q.n, 0, q.n, (long)q.m});
    if (q.n) {
        const cudaError_t e = cudaMemcpy2DAsync(r->d, r->stride * 8, q.A.row(q.P.h), q.A.stride * 8,
                                                ((size_t)ctx->P.big() + 1) * 8, q.n, cudaMemcpyDeviceToDevice,
                                                ctx->stream);
        if (e != cudaSuccess) { lvs_result_free(r); return cuda_error(e, "server result copy"); }
    }
    if ((st = finish_result(ctx, r)) != LVS_OK) { lvs_result_free(r); return st; }
    *out = r;
    return LVS_OK;
}

void release(lvs_server *S, Query *q)
{
    arena_free(S->ctx, q->A);
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= q->bytes;
    S->known.erase(q->ticket);
    delete q;
}

void complete(lvs_server *S, Query *q, lvs_status st, const std::string &msg, lvs_result *r)
{
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->done[q->ticket] = {st, msg, r};
        S->stats.completed += 1;
    }
    release(S, q);
}

void worker_loop(lvs_server *S)
{
    lvs_ctx *ctx = S->ctx;
    cudaSetDevice(ctx->device);
    std::vector<Job> jobs;
    for (;;) {
        std::vector<Query *> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
            if (S->stop) return;
            // admission by device memory: always admit one query when idle
            while (!S->pending.empty()) {
                Query *q = S->pending.front();
                const size_t running = S->active.size() + admitted.size();
                if (S->max_active && running >= S->max_active) break;
                if (running > 0 && S->used + q->bytes > S->budget) break;
                S->pending.pop_front();
                S->used += q->bytes;
                admitted.push_back(q);
                S->stats.admitted += 1;
            }
            S->stats.pending = S->pending.size();
        }
        std::vector<Query *> retry;
        for (Query *q : admitted) {
            lvs_status st;
            {
                std::lock_guard<std::mutex> lk(ctx->mu);
                st = setup(ctx, *q);
            }
            if (st == LVS_ERR_OOM && !S->active.empty()) {
                // memory is held by running queries: try again at a later step
                {
                    std::lock_guard<std::mutex> lk(ctx->mu);
                    arena_free(ctx, q->A);
                }
                retry.push_back(q);
                continue;
            }
            if (st != LVS_OK) { complete(S, q, st, lvs_last_error(), nullptr); continue; }
            S->active.push_back(q);
        }
        if (!retry.empty()) {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto it = retry.rbegin(); it != retry.rend(); ++it) {
                S->used -= (*it)->bytes;
                S->pending.push_front(*it);
                S->stats.admitted -= 1;
                S->stats.requeued += 1;
            }
            S->stats.pending = S->pending.size();
        }
        jobs.clear();
        for (Query *q : S->active) plan_query(*q, jobs);
        const auto t0 = std::chrono::steady_clock::now();
        lvs_status st = LVS_OK;
        if (!jobs.empty()) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            st = run_steps(ctx, jobs, std::vector<size_t>{0, jobs.size()}, false);
            if (st == LVS_OK) {
                const cudaError_t e = cudaStreamSynchronize(ctx->stream);
                if (e != cudaSuccess) st = cuda_error(e, "server step");
                else st = device_fault_check(ctx->device);
            }
        }
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.steps += jobs.empty() ? 0 : 1;
            S->stats.pbs += jobs.size();
            S->stats.max_step_pbs = std::max<uint64_t>(S->stats.max_step_pbs, jobs.size());
            S->stats.busy_ms += ms;
        }
        const std::string err = st == LVS_OK ? std::string() : std::string(lvs_last_error());
        std::vector<Query *> still;
        for (Query *q : S->active) {
            if (st != LVS_OK) { complete(S, q, st, err, nullptr); continue; }
            q->step += 1;
            if (q->step >= q->steps) {
                lvs_result *r = nullptr;
                lvs_status fs;
                {
                    std::lock_guard<std::mutex> lk(ctx->mu);
                    fs = finish(S, *q, &r);
                }
                complete(S, q, fs, fs == LVS_OK ? std::string() : std::string(lvs_last_error()), r);
            } else {
                still.push_back(q);
            }
        }
        S->active.swap(still);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.active = S->active.size();
            S->stats.mem_in_use = S->used;
        }
    }
}

}  // namespace
}  // namespace lvs

using namespace lvs;

extern "C" {

lvs_status lvs_server_create(lvs_ctx *ctx, size_t mem_budget_bytes, size_t max_active, lvs_server **out)
{
    if (!ctx || !out) return set_error(LVS_ERR_ARG, "lvs_server_create: NULL argument");
    if (mem_budget_bytes == 0) return set_error(LVS_ERR_ARG, "lvs_server_create: zero memory budget");
    lvs_server *S = new (std::nothrow) lvs_server;
    if (!S) return set_error(LVS_ERR_OOM, "lvs_server_create: host allocation failed");
    S->ctx = ctx;
    S->budget = mem_budget_bytes;
    S->max_active = max_active;
    try {
        S->worker = std::thread(worker_loop, S);
    } catch (...) {
        delete S;
        return set_error(LVS_ERR_OOM, "lvs_server_create: cannot start the worker thread");
    }
    *out = S;
    return LVS_OK;
}

lvs_status lvs_server_submit(lvs_server *S, const lvs_query *qq, uint64_t *ticket)
{
    if (!S || !qq || !ticket || !qq->query) return set_error(LVS_ERR_ARG, "lvs_server_submit: NULL argument");
    lvs_status st = check_ctx_string(S->ctx, qq->query);
    if (st != LVS_OK) return st;
    Query *q = new (std::nothrow) Query;
    if (!q) return set_error(LVS_ERR_OOM, "lvs_server_submit: host allocation failed");
    try {
        q->q = *qq->query;
        q->q.d = nullptr;            // the copy never owns device memory
        q->m = q->q.len;
        q->C = q->q.symbols;
        for (int c = 0; c < 256; ++c) q->row_of[c] = -1;
        if (qq->ref_enc) {
            if ((st = check_ctx_string(S->ctx, qq->ref_enc)) != LVS_OK) { delete q; return st; }
            if ((qq->ref_enc->alphabet == LVS_ALPHA_DNA4) != (q->q.alphabet == LVS_ALPHA_DNA4)) {
                delete q;
                return set_error(LVS_ERR_ARG, "lvs_server_submit: query and reference alphabets differ");
            }
            q->ref = *qq->ref_enc;
            q->ref.d = nullptr;
            q->n = q->ref.len;
        } else {
            if (qq->ref_plain_len && !qq->ref_plain) { delete q; return set_error(LVS_ERR_ARG, "lvs_server_submit: NULL reference"); }
            q->plain = true;
            q->ref_plain.assign(qq->ref_plain, qq->ref_plain + qq->ref_plain_len);
            q->n = qq->ref_plain_len;
            for (uint8_t c : q->ref_plain) {
                uint32_t v[2] = {0, 0};
                if (!encode_char(q->q.alphabet, c, v)) {
                    delete q;
                    return set_error(LVS_ERR_ARG, "lvs_server_submit: reference character outside the alphabet");
                }
                if (q->row_of[c] < 0) {
                    q->row_of[c] = (int32_t)q->subset.size();
                    q->subset.push_back(c);
                    q->sym.push_back({v[0], v[1]});
                }
            }
        }
    } catch (const std::bad_alloc &) {
        delete q;
        return set_error(LVS_ERR_OOM, "lvs_server_submit: host allocation failed");
    }
    const size_t stride = (size_t)S->ctx->P.big() + 2;
    q->bytes = (query_rows(*q) + q->n) * stride * 8;
    if (q->bytes > S->budget) {
        delete q;
        return set_error(LVS_ERR_ARG, "lvs_server_submit: the query needs more device memory than the budget");
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->ticket = S->next_ticket++;
        S->pending.push_back(q);
        S->known[q->ticket] = 1;
        S->stats.submitted += 1;
        S->stats.pending = S->pending.size();
        *ticket = q->ticket;
    }
    S->cv.notify_one();
    return LVS_OK;
}

lvs_status lvs_server_poll(lvs_server *S, uint64_t ticket, lvs_result **out)
{
    if (!S || !out) return set_error(LVS_ERR_ARG, "lvs_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (S->known.count(ticket)) return LVS_ERR_STATE;   // not ready (no message)
        return set_error(LVS_ERR_ARG, "lvs_server_poll: unknown ticket");
    }
    const auto d = it->second;
    S->done.erase(it);
    if (d.st != LVS_OK) return set_error(d.st, d.msg);
    *out = d.r;
    return LVS_OK;
}

lvs_status lvs_server_stats_get(lvs_server *S, lvs_server_stats *out)
{
    if (!S || !out) return set_error(LVS_ERR_ARG, "lvs_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    out->mem_in_use = S->used;
    out->pending = S->pending.size();
    return LVS_OK;
}

void lvs_server_free(lvs_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->ctx->device);
    for (Query *q : S->active) release(S, q);
    S->active.clear();
    for (Query *q : S->pending) delete q;
    S->pending.clear();
    for (auto &kv : S->done)
        if (kv.second.r) lvs_result_free(kv.second.r);
    delete S;
}

}  // extern "C"
