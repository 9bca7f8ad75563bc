// Wavefront scheduler and the server-side entry points.
//
// The cells of one anti-diagonal of the difference matrix are independent
// (Section 6.2, "Parallelisation over cells"), and so are different string
// pairs ("Batch inputs matching").  A batch therefore advances every pair one
// anti-diagonal per launch step, and each step bootstraps the union of
//   - the cell PBS of anti-diagonal d      (key of Eq. eq_keyeq2, LUT_min),
//   - the second equality PBS of d+1       (Algorithm alg_ascii, LUT_EQ9),
//   - the first equality PBS of d+2        (LUT_EQ)
// over all pairs (two-lookup equality; with the one-lookup DNA equality the
// pipeline is one step shorter).  Equality results live in two-slot rings
// indexed by the parity of the anti-diagonal.
//
// Device memory of a batch ("arena"): rows of k*N+2 words (16-byte aligned
// big LWE ciphertexts): string symbols, the frontier v[i] / h[j] and the rings.
// It is allocated stream-ordered and released when the batch has been copied
// into its result.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "lvs_internal.hpp"

namespace lvs {

// host-side fault injection (lvs_debug_fail_allocations)
static std::atomic<int> g_fail_allocs{0};

static bool injected_failure()
{
    int c = g_fail_allocs.load();
    while (c > 0)
        if (g_fail_allocs.compare_exchange_weak(c, c - 1)) return true;
    return false;
}

lvs_status arena_alloc(lvs_ctx *ctx, size_t rows, Arena &A)
{
    A.stride = (size_t)ctx->P.big() + 2;
    A.rows = rows;
    A.d = nullptr;
    if (rows == 0) return LVS_OK;
    if (injected_failure())
        return set_error(LVS_ERR_OOM, "device allocation of the batch arena failed (injected)");
    if (cudaMallocAsync((void **)&A.d, rows * A.stride * 8, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LVS_ERR_OOM, "device allocation of the batch arena failed (" +
                                          std::to_string(rows * A.stride * 8 >> 20) + " MiB)");
    }
    return LVS_OK;
}

void arena_free(lvs_ctx *ctx, Arena &A)
{
    if (A.d) cudaFreeAsync(A.d, ctx->stream);
    A.d = nullptr;
}

// host string -> consecutive arena rows
lvs_status upload_string(lvs_ctx *ctx, const lvs_ct_string *s, const Arena &A, size_t first)
{
    const size_t nrows = s->len * s->symbols;
    if (nrows == 0) return LVS_OK;
    const size_t w = (size_t)s->big + 1;
    LVS_CUDA(cudaMemcpy2DAsync(A.row(first), A.stride * 8, s->host(), w * 8, w * 8, nrows,
                               cudaMemcpyHostToDevice, ctx->stream));
    return LVS_OK;
}

Job make_job(const uint64_t *s0, int c0, const uint64_t *s1, int c1, const uint64_t *s2, int c2, int cst,
             uint8_t lut, uint8_t kind, uint64_t *d0, uint64_t *d1)
{
    Job J;
    memset(&J, 0, sizeof(J));
    J.src[0] = s0; J.src[1] = s1; J.src[2] = s2;
    J.coef[0] = (int8_t)c0; J.coef[1] = (int8_t)c1; J.coef[2] = (int8_t)c2;
    J.cst = (int8_t)(((cst % 32) + 32) % 32);
    J.lut = lut;
    J.kind = kind;
    J.dst[0] = d0; J.dst[1] = d1;
    return J;
}

lvs_status make_result(lvs_ctx *ctx, size_t rows, lvs_result **out)
{
    lvs_result *r = new (std::nothrow) lvs_result;
    if (!r) return set_error(LVS_ERR_OOM, "result allocation failed");
    r->P = ctx->P;
    r->device = ctx->device;
    r->stride = (size_t)ctx->P.big() + 2;
    if (rows && cudaMalloc((void **)&r->d, rows * r->stride * 8) != cudaSuccess) {
        cudaGetLastError();
        delete r;
        return set_error(LVS_ERR_OOM, "device allocation of the result failed");
    }
    *out = r;
    return LVS_OK;
}

lvs_status finish_result(lvs_ctx *ctx, lvs_result *r)
{
    LVS_CUDA(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
    LVS_CUDA(cudaEventRecord(r->done, ctx->stream));
    return LVS_OK;
}

static long floor_div2(long x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

// cells (i, j) with i + j - 2 = d, 1 <= i <= m, 1 <= j <= n, inside the band:
// diagonals k = j - i with min(0, n - m) - band <= k <= max(0, n - m) + band
// (|i - j| <= band for m = n, Algorithm alg_levenshtein; for m != n the cells
// where an edit path of cost <= |n - m| + 2 band can pass)
template <class F>
static void for_diag(const PairRows &P, long d, F f)
{
    if (d < 0 || P.m == 0 || P.n == 0) return;
    long lo = std::max<long>(1, d + 2 - (long)P.n), hi = std::min<long>((long)P.m, d + 1);
    if (P.band >= 0) {
        const long delta = (long)P.n - (long)P.m;
        const long klo = std::min(0L, delta) - P.band, khi = std::max(0L, delta) + P.band;
        // k = d + 2 - 2i in [klo, khi]  <=>  ceil((d + 2 - khi) / 2) <= i <= floor((d + 2 - klo) / 2)
        lo = std::max(lo, -floor_div2(-(d + 2 - khi)));
        hi = std::min(hi, floor_div2(d + 2 - klo));
    }
    for (long i = lo; i <= hi; ++i) f((size_t)i, (size_t)(d + 2 - i));
}

// band mode: the readout path from (0, 0) to (m, n) -- down the main diagonal
// (v[i][i-1], h[i][i]) for i <= min(m, n), then along row m (h[m][j]) or down
// column n (v[i][n]); the distance is the sum of its differences (Section 3.2).
// A cell on the path copies its new v (tapsel 1) or h (tapsel 2) to the tap
// row of its step.
static Job tapped(const PairRows &P, const Arena &A, size_t i, size_t j, Job J)
{
    if (P.band < 0) return J;
    const size_t r = std::min(P.m, P.n);
    if (i <= r && j + 1 == i) { J.tap = A.row(P.tap + 2 * (i - 1)); J.tapsel = 1; }
    else if (i <= r && j == i) { J.tap = A.row(P.tap + 2 * (i - 1) + 1); J.tapsel = 2; }
    else if (P.n > P.m && i == P.m && j > P.m) { J.tap = A.row(P.tap + 2 * r + (j - P.m - 1)); J.tapsel = 2; }
    else if (P.m > P.n && j == P.n && i > P.n) { J.tap = A.row(P.tap + 2 * r + (i - P.n - 1)); J.tapsel = 1; }
    return J;
}

// the cell PBS of (i, j): key = (1 - v[i][j-1]) + 3 (1 + h[i-1][j]) + EQ9 through
// LUT_min with the in-place update of v[i] and h[j]; on a refreshed
// anti-diagonal (Section 3.1.3) two PBS through LUT_V instead: v from the
// key, h from the key with v and h exchanged, both fresh bootstrap outputs.
static void cell_jobs(const PairRows &P, const Arena &A, size_t i, size_t j, const uint64_t *e9, uint64_t *Vi,
                      uint64_t *Hj, std::vector<Job> &jobs)
{
    if (!P.refresh.empty() && P.refresh[i + j]) {
        const Job t = tapped(P, A, i, j, Job{});
        Job jv = make_job(Vi, -1, Hj, 3, e9, 1, 4, LUT_V, JOB_STORE, Vi, nullptr);
        Job jh = make_job(Vi, 3, Hj, -1, e9, 1, 4, LUT_V, JOB_STORE, Hj, nullptr);
        if (t.tapsel == 1) { jv.tap = t.tap; jv.tapsel = 1; }
        if (t.tapsel == 2) { jh.tap = t.tap; jh.tapsel = 1; }
        jobs.push_back(jv);
        jobs.push_back(jh);
        return;
    }
    jobs.push_back(tapped(P, A, i, j, make_job(Vi, -1, Hj, 3, e9, 1, 4, LUT_MIN, JOB_CELL, Vi, Hj)));
}

void plan_pair_step(const PairRows &P, const Arena &A, long s, std::vector<Job> &jobs)
{
    auto X = [&](size_t i, int sym) {
        return P.xd ? P.xd + ((i - 1) * P.C + sym) * P.xs : A.row(P.x + (i - 1) * P.C + sym);
    };
    auto Y = [&](size_t j, int sym) {
        return P.yd ? P.yd + ((j - 1) * P.C + sym) * P.ys : A.row(P.y + (j - 1) * P.C + sym);
    };
    auto V = [&](size_t i) { return A.row(P.v + i - 1); };
    auto H = [&](size_t j) { return A.row(P.h + j - 1); };
    auto E1 = [&](long d, size_t i) { return A.row(P.eq1 + (size_t)(d & 1) * P.m + i - 1); };
    auto E9 = [&](long d, size_t i) { return A.row(P.eq9 + (size_t)(d & 1) * P.m + i - 1); };
    if (P.table) {
        // preprocessed: EQ9[i][j] = T[b_j][i], one cell PBS per cell
        for_diag(P, s, [&](size_t i, size_t j) {
            const uint64_t *t = P.table + ((size_t)P.row_of[P.plain[j - 1]] * P.m + (i - 1)) * P.table_stride;
            cell_jobs(P, A, i, j, t, V(i), H(j), jobs);
        });
        return;
    }
    if (P.C == 2) {
        // EQ1 of diagonal s: z1 = x1_i - y1_j
        for_diag(P, s, [&](size_t i, size_t j) {
            jobs.push_back(make_job(X(i, 0), 1, Y(j, 0), -1, nullptr, 0, 0, LUT_EQ, JOB_STORE, E1(s, i), nullptr));
        });
        // EQ9 of diagonal s-1: z2 = 2 (x2_i - y2_j) + (1 - EQ1)
        for_diag(P, s - 1, [&](size_t i, size_t j) {
            jobs.push_back(make_job(X(i, 1), 2, Y(j, 1), -2, E1(s - 1, i), -1, 1, LUT_EQ9, JOB_STORE, E9(s - 1, i),
                                    nullptr));
        });
        // cells of diagonal s-2: key = (1 - v[i][j-1]) + 3 (1 + h[i-1][j]) + EQ9
        for_diag(P, s - 2, [&](size_t i, size_t j) {
            cell_jobs(P, A, i, j, E9(s - 2, i), V(i), H(j), jobs);
        });
    } else {
        // DNA: EQ9 = PBS(x_i - y_j; LUT_EQ9), one lookup
        for_diag(P, s, [&](size_t i, size_t j) {
            jobs.push_back(make_job(X(i, 0), 1, Y(j, 0), -1, nullptr, 0, 0, LUT_EQ9, JOB_STORE, E9(s, i), nullptr));
        });
        for_diag(P, s - 1, [&](size_t i, size_t j) {
            cell_jobs(P, A, i, j, E9(s - 1, i), V(i), H(j), jobs);
        });
    }
}

long pair_steps(const PairRows &P)
{
    if (P.m == 0 || P.n == 0) return 0;
    const long depth = P.table ? 0 : (long)P.C;
    return (long)(P.m + P.n - 2) + depth + 1;
}

// Runs the wavefront over all pairs; rows already placed.
// Launch of every step of every pair.  All pairs start together; at each
// launch, when the PBS of the pairs' current steps exceed a multiple of `wave`
// (the jobs the blind-rotation grid runs at once) by a remainder r, pairs with
// slack -- whose remaining steps are fewer than the longest pair's -- are held
// back one launch, smallest current step first, until at least r PBS are held
// back: the launch then ends on a full wave and the held-back steps join later
// launches.  A pair's steps keep their order (each launch runs at most one step
// of a pair, after its earlier steps), and the number of launches stays the
// longest pair's step count.  wave == 0: no holding back.
void schedule_steps(const std::vector<std::vector<uint32_t>> &counts, size_t wave,
                    std::vector<std::vector<long>> &launch_of, long *nlaunch)
{
    const size_t np = counts.size();
    launch_of.assign(np, {});
    std::vector<size_t> cur(np, 0);
    for (size_t p = 0; p < np; ++p) launch_of[p].assign(counts[p].size(), -1);
    std::vector<size_t> act, cand;
    std::vector<char> held(np, 0);
    long t = 0;
    for (;; ++t) {
        act.clear();
        size_t rem_max = 0, tot = 0;
        for (size_t p = 0; p < np; ++p)
            if (cur[p] < counts[p].size()) {
                act.push_back(p);
                rem_max = std::max(rem_max, counts[p].size() - cur[p]);
                tot += counts[p][cur[p]];
            }
        if (act.empty()) break;
        const size_t r = wave ? tot % wave : 0;
        if (wave && tot > wave && r > 0) {
            cand.clear();
            for (size_t p : act)
                if (counts[p].size() - cur[p] < rem_max && counts[p][cur[p]] > 0) cand.push_back(p);
            std::stable_sort(cand.begin(), cand.end(),
                             [&](size_t x, size_t y) { return counts[x][cur[x]] < counts[y][cur[y]]; });
            size_t s = 0;
            for (size_t p : cand) {
                if (s >= r) break;
                held[p] = 1;
                s += counts[p][cur[p]];
            }
        }
        for (size_t p : act) {
            if (held[p]) { held[p] = 0; continue; }
            launch_of[p][cur[p]] = t;
            ++cur[p];
        }
    }
    *nlaunch = t;
}

static lvs_status run_wavefront(lvs_ctx *ctx, const std::vector<PairRows> &pairs, const Arena &A, bool use_graph)
{
    const size_t np = pairs.size();
    // every step of every pair, planned once
    std::vector<std::vector<Job>> pj(np);
    std::vector<std::vector<size_t>> poff(np);
    std::vector<std::vector<uint32_t>> counts(np);
    for (size_t p = 0; p < np; ++p) {
        const long steps = pair_steps(pairs[p]);
        poff[p].push_back(0);
        for (long s = 0; s < steps; ++s) {
            plan_pair_step(pairs[p], A, s, pj[p]);
            poff[p].push_back(pj[p].size());
            counts[p].push_back((uint32_t)(poff[p][s + 1] - poff[p][s]));
        }
    }
    std::vector<std::vector<long>> launch_of;
    long nl = 0;
    schedule_steps(counts, ctx->wave_fill ? (size_t)ctx->br_grid : 0, launch_of, &nl);
    // launch t = the steps scheduled at t, in pair order
    std::vector<std::vector<std::pair<size_t, size_t>>> at(nl);
    for (size_t p = 0; p < np; ++p)
        for (size_t s = 0; s < launch_of[p].size(); ++s) at[launch_of[p][s]].push_back({p, s});
    std::vector<Job> jobs;
    std::vector<size_t> off{0};
    for (long t = 0; t < nl; ++t) {
        for (const auto &ps : at[t])
            jobs.insert(jobs.end(), pj[ps.first].begin() + poff[ps.first][ps.second],
                        pj[ps.first].begin() + poff[ps.first][ps.second + 1]);
        off.push_back(jobs.size());
    }
    return run_steps(ctx, jobs, off, use_graph);
}

lvs_status check_ctx_string(const lvs_ctx *ctx, const lvs_ct_string *s)
{
    if (!s) return set_error(LVS_ERR_ARG, "NULL encrypted string");
    if (s->big != ctx->P.big()) return set_error(LVS_ERR_ARG, "encrypted string dimension does not match the context");
    return LVS_OK;
}

}  // namespace lvs

using namespace lvs;

extern "C" {

void lvs_debug_fail_allocations(int32_t count) { g_fail_allocs.store(count > 0 ? count : 0); }

lvs_status lvs_edit_distance_batch(lvs_ctx *ctx, const lvs_ct_string *const *a, const lvs_ct_string *const *b,
                                   size_t npairs, const lvs_opts *opts, lvs_result **out)
{
    if (!ctx || !out || (npairs && (!a || !b))) return set_error(LVS_ERR_ARG, "lvs_edit_distance_batch: NULL argument");
    lvs_opts o;
    lvs_opts_default(&o);
    if (opts) o = *opts;
    const bool banded = o.band >= 0;
    std::vector<PairRows> pairs(npairs);
    size_t rows = 0, xrows = 0, vrows = 0, hrows = 0, rrows = 0, trows = 0;
    for (size_t p = 0; p < npairs; ++p) {
        lvs_status st = check_ctx_string(ctx, a[p]);
        if (st == LVS_OK) st = check_ctx_string(ctx, b[p]);
        if (st != LVS_OK) return st;
        if (symbols_per_char(a[p]->alphabet) != symbols_per_char(b[p]->alphabet) ||
            (a[p]->alphabet == LVS_ALPHA_DNA4) != (b[p]->alphabet == LVS_ALPHA_DNA4))
            return set_error(LVS_ERR_ARG, "lvs_edit_distance_batch: pair " + std::to_string(p) +
                                              " mixes alphabets");
        PairRows &P = pairs[p];
        P.m = a[p]->len;
        P.n = b[p]->len;
        P.C = a[p]->symbols;
        if (banded) {
            P.band = o.band;
            trows += P.m + P.n;
        }
        if ((st = plan_refresh(ctx, o.refresh_budget, P)) != LVS_OK) return st;
        if (a[p]->d && a[p]->ddevice == ctx->device) { P.xd = a[p]->d; P.xs = a[p]->dstride; }
        else xrows += P.m * P.C;
        if (b[p]->d && b[p]->ddevice == ctx->device) { P.yd = b[p]->d; P.ys = b[p]->dstride; }
        else xrows += P.n * P.C;
        vrows += P.m;
        hrows += P.n;
        rrows += (P.C == 2 ? 4 : 2) * P.m;
    }
    // rows: [strings][v][h][band taps][rings]
    rows = xrows + vrows + hrows + trows + rrows;
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lock(ctx->mu);
    Arena A;
    lvs_status st = arena_alloc(ctx, rows, A);
    if (st != LVS_OK) return st;
    size_t cx = 0, cv = xrows, ch = xrows + vrows, ct = xrows + vrows + hrows, cr = ct + trows;
    for (size_t p = 0; p < npairs; ++p) {
        PairRows &P = pairs[p];
        if (banded) { P.tap = ct; ct += P.m + P.n; }
        if (!P.xd) { P.x = cx; cx += P.m * P.C; }
        if (!P.yd) { P.y = cx; cx += P.n * P.C; }
        P.v = cv; cv += P.m;
        P.h = ch; ch += P.n;
        if (P.C == 2) { P.eq1 = cr; cr += 2 * P.m; }
        P.eq9 = cr; cr += 2 * P.m;
        if ((!P.xd && (st = upload_string(ctx, a[p], A, P.x)) != LVS_OK) ||
            (!P.yd && (st = upload_string(ctx, b[p], A, P.y)) != LVS_OK)) {
            arena_free(ctx, A);
            return st;
        }
    }
    // OneMatrix boundary: v[i][0] = h[0][j] = 1 as noiseless ciphertexts (0, Delta);
    // band taps start at 1 too (out-of-band path values keep the OneMatrix value)
    cudaError_t e = launch_fill_trivial(A.d, A.stride, ctx->P.big(), xrows, vrows + hrows + trows, 1ull << kDeltaLog,
                                        ctx->stream);
    if (e != cudaSuccess) { arena_free(ctx, A); return cuda_error(e, "fill"); }
    ctx->launches += vrows + hrows ? 1 : 0;
    st = run_wavefront(ctx, pairs, A, o.use_graph != 0);
    if (st != LVS_OK) { arena_free(ctx, A); return st; }
    lvs_result *r = nullptr;
    // result rows: h[m][1..n] (distance m + sum), or the band's diagonal path (distance = sum)
    const size_t out_rows = banded ? trows : hrows;
    st = make_result(ctx, out_rows, &r);
    if (st != LVS_OK) { arena_free(ctx, A); return st; }
    size_t first = 0;
    for (size_t p = 0; p < npairs; ++p) {
        const size_t cnt = banded ? pairs[p].m + pairs[p].n : pairs[p].n;
        r->items.push_back({pairs[p].m, pairs[p].n, first, cnt, banded ? 0L : (long)pairs[p].m});
        first += cnt;
    }
    if (out_rows) {
        e = cudaMemcpy2DAsync(r->d, r->stride * 8, A.row(banded ? xrows + vrows + hrows : xrows + vrows), A.stride * 8,
                              (ctx->P.big() + 1) * 8, out_rows, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) { arena_free(ctx, A); lvs_result_free(r); return cuda_error(e, "result copy"); }
    }
    arena_free(ctx, A);
    st = finish_result(ctx, r);
    if (st != LVS_OK) { lvs_result_free(r); return st; }
    *out = r;
    return LVS_OK;
}

lvs_status lvs_eq(lvs_ctx *ctx, const lvs_ct_string *a, size_t i, const lvs_ct_string *b, size_t j, int times9,
                  lvs_result **out)
{
    if (!ctx || !out) return set_error(LVS_ERR_ARG, "lvs_eq: NULL argument");
    lvs_status st = check_ctx_string(ctx, a);
    if (st == LVS_OK) st = check_ctx_string(ctx, b);
    if (st != LVS_OK) return st;
    if (i >= a->len || j >= b->len) return set_error(LVS_ERR_ARG, "lvs_eq: character index out of range");
    if ((a->alphabet == LVS_ALPHA_DNA4) != (b->alphabet == LVS_ALPHA_DNA4))
        return set_error(LVS_ERR_ARG, "lvs_eq: alphabets differ");
    const uint32_t C = a->symbols;
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lock(ctx->mu);
    Arena A;
    // rows: x (C), y (C), eq1
    if ((st = arena_alloc(ctx, 2 * C + 1, A)) != LVS_OK) return st;
    const size_t w = (size_t)a->big + 1;
    cudaError_t e = cudaMemcpy2DAsync(A.row(0), A.stride * 8, a->host() + i * C * w, w * 8, w * 8, C,
                                      cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(A.row(C), A.stride * 8, b->host() + j * C * w, w * 8, w * 8, C,
                              cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) { arena_free(ctx, A); return cuda_error(e, "lvs_eq upload"); }
    lvs_result *r = nullptr;
    if ((st = make_result(ctx, 1, &r)) != LVS_OK) { arena_free(ctx, A); return st; }
    r->is_eq = true;
    r->items.push_back({1, 1, 0, 1, 0});
    const uint8_t last = times9 ? LUT_EQ9 : LUT_EQ;
    std::vector<Job> jobs;
    std::vector<size_t> off{0};
    if (C == 2) {
        jobs.push_back(make_job(A.row(0), 1, A.row(C), -1, nullptr, 0, 0, LUT_EQ, JOB_STORE, A.row(2 * C), nullptr));
        off.push_back(1);
        jobs.push_back(make_job(A.row(1), 2, A.row(C + 1), -2, A.row(2 * C), -1, 1, last, JOB_STORE, r->d, nullptr));
        off.push_back(2);
    } else {
        jobs.push_back(make_job(A.row(0), 1, A.row(C), -1, nullptr, 0, 0, last, JOB_STORE, r->d, nullptr));
        off.push_back(1);
    }
    st = run_steps(ctx, jobs, off, false);
    arena_free(ctx, A);
    if (st == LVS_OK) st = finish_result(ctx, r);
    if (st != LVS_OK) { lvs_result_free(r); return st; }
    *out = r;
    return LVS_OK;
}

lvs_status lvs_preprocess_batch(lvs_ctx *ctx, const lvs_ct_string *const *encs, size_t count, const uint8_t *subset,
                                size_t nsub, lvs_eq_table **outs)
{
    if (!ctx || !outs || (count && !encs)) return set_error(LVS_ERR_ARG, "lvs_preprocess: NULL argument");
    lvs_status st = LVS_OK;
    for (size_t k = 0; k < count; ++k)
        if ((st = check_ctx_string(ctx, encs[k])) != LVS_OK) return st;
    std::vector<lvs_eq_table *> tabs(count, nullptr);
    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> syms(count);
    auto free_all = [&]() {
        for (auto t : tabs) lvs_eq_table_free(t);
    };
    // host side of every table: subset rows and their symbol values
    for (size_t k = 0; k < count; ++k) {
        const lvs_ct_string *enc = encs[k];
        std::vector<uint8_t> sub;
        if (subset) sub.assign(subset, subset + nsub);
        else
            for (uint32_t s2 = 0; s2 < alphabet_size(enc->alphabet); ++s2) sub.push_back(alphabet_char(enc->alphabet, s2));
        lvs_eq_table *t = new (std::nothrow) lvs_eq_table;
        if (!t) { free_all(); return set_error(LVS_ERR_OOM, "lvs_preprocess: host allocation failed"); }
        tabs[k] = t;
        t->P = ctx->P;
        t->device = ctx->device;
        t->alphabet = enc->alphabet;
        t->len = enc->len;
        t->stride = (size_t)ctx->P.big() + 2;
        for (int c = 0; c < 256; ++c) t->row_of[c] = -1;
        syms[k].resize(sub.size());
        for (size_t r = 0; r < sub.size(); ++r) {
            uint32_t v[2] = {0, 0};
            if (!encode_char(enc->alphabet, sub[r], v) || t->row_of[sub[r]] >= 0) {
                free_all();
                return set_error(LVS_ERR_ARG, "lvs_preprocess: subset character " + std::to_string(sub[r]) +
                                                  " is outside the alphabet or repeated");
            }
            t->row_of[sub[r]] = (int32_t)r;
            syms[k][r] = {v[0], v[1]};
        }
        t->subset = sub;
    }
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lock(ctx->mu);
    // arena: per string x (m*C) and, for two lookups, EQ1 (R*m)
    size_t rows = 0;
    std::vector<size_t> base(count);
    for (size_t k = 0; k < count; ++k) {
        const size_t m = encs[k]->len, C = encs[k]->symbols, R = tabs[k]->subset.size();
        base[k] = rows;
        rows += m * C + (C == 2 ? R * m : 0);
        if (R * m != 0 && cudaMalloc((void **)&tabs[k]->d, R * m * tabs[k]->stride * 8) != cudaSuccess) {
            cudaGetLastError();
            free_all();
            return set_error(LVS_ERR_OOM, "lvs_preprocess: device allocation of the table failed");
        }
    }
    Arena A;
    if ((st = arena_alloc(ctx, rows, A)) != LVS_OK) { free_all(); return st; }
    for (size_t k = 0; k < count && st == LVS_OK; ++k) st = upload_string(ctx, encs[k], A, base[k]);
    if (st != LVS_OK) { arena_free(ctx, A); free_all(); return st; }
    // step 0: EQ1 = PBS(x1_i - sigma1; LUT_EQ) (DNA: EQ9 = PBS(x_i - sigma; LUT_EQ9));
    // step 1: EQ9 = PBS(2 (x2_i - sigma2) + 1 - EQ1; LUT_EQ9) -- all strings in the same launches
    std::vector<Job> jobs;
    std::vector<size_t> off{0};
    for (int step = 0; step < 2; ++step) {
        for (size_t k = 0; k < count; ++k) {
            lvs_eq_table *t = tabs[k];
            const size_t m = encs[k]->len, C = encs[k]->symbols, b0 = base[k];
            table_step_jobs(
                step, (uint32_t)C, m, syms[k], [&](size_t i, int s) { return A.row(b0 + i * C + s); },
                [&](size_t r, size_t i) { return A.row(b0 + m * C + r * m + i); },
                [&](size_t r, size_t i) { return t->d + (r * m + i) * t->stride; }, jobs);
        }
        off.push_back(jobs.size());
    }
    st = run_steps(ctx, jobs, off, false);
    arena_free(ctx, A);
    for (size_t k = 0; k < count && st == LVS_OK; ++k)
        if (cudaEventCreateWithFlags(&tabs[k]->done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(tabs[k]->done, ctx->stream) != cudaSuccess)
            st = set_error(LVS_ERR_CUDA, "lvs_preprocess: event");
    if (st != LVS_OK) { free_all(); return st; }
    for (size_t k = 0; k < count; ++k) outs[k] = tabs[k];
    return LVS_OK;
}

lvs_status lvs_preprocess(lvs_ctx *ctx, const lvs_ct_string *enc, const uint8_t *subset, size_t nsub,
                          lvs_eq_table **out)
{
    if (!ctx || !out || !enc) return set_error(LVS_ERR_ARG, "lvs_preprocess: NULL argument");
    return lvs_preprocess_batch(ctx, &enc, 1, subset, nsub, out);
}

void lvs_eq_table_free(lvs_eq_table *t)
{
    if (!t) return;
    cudaSetDevice(t->device);
    if (t->done) { cudaEventSynchronize(t->done); cudaEventDestroy(t->done); }
    if (t->d) cudaFree(t->d);
    cudaGetLastError();
    delete t;
}

// plan jobs -> exported rows (offsets from the base of a one-word-per-row array)
static void export_jobs(const std::vector<Job> &J, const std::vector<int64_t> &step_of, const uint64_t *base,
                        lvs_plan_job *jobs)
{
    auto row = [&](const uint64_t *q) -> int64_t { return q ? (int64_t)(q - base) : -1; };
    for (size_t k = 0; k < J.size(); ++k) {
        lvs_plan_job &o = jobs[k];
        o.step = step_of[k];
        for (int t = 0; t < 3; ++t) {
            o.src[t] = row(J[k].src[t]);
            o.coef[t] = J[k].src[t] ? J[k].coef[t] : 0;
        }
        o.cst = J[k].cst;
        o.dst[0] = row(J[k].dst[0]);
        o.dst[1] = row(J[k].dst[1]);
        o.tap = J[k].tapsel ? row(J[k].tap) : -1;
        o.lut = J[k].lut;
        o.kind = J[k].kind;
        o.tapsel = J[k].tapsel;
        o.pad = 0;
    }
}

lvs_status lvs_plan_pair(size_t m, size_t n, uint32_t eq_lookups, int32_t band, const uint8_t *refresh,
                         const uint8_t *plain, const uint8_t *subset, size_t nsub, lvs_plan_layout *layout,
                         lvs_plan_job *jobs, size_t *count)
{
    if (!count) return set_error(LVS_ERR_ARG, "lvs_plan_pair: NULL count");
    if (eq_lookups > 2) return set_error(LVS_ERR_ARG, "lvs_plan_pair: eq_lookups must be 0, 1 or 2");
    const bool pre = eq_lookups == 0;
    if (pre && n && (!plain || !subset || nsub == 0))
        return set_error(LVS_ERR_ARG, "lvs_plan_pair: the plaintext reference needs plain and subset");
    PairRows P;
    P.m = m;
    P.n = n;
    P.C = pre ? 1 : eq_lookups;
    P.band = band >= 0 ? band : -1;
    if (refresh) P.refresh.assign(refresh, refresh + m + n + 1);
    int32_t row_of[256];
    std::fill(row_of, row_of + 256, -1);
    if (pre)
        for (size_t k = 0; k < nsub; ++k) {
            if (row_of[subset[k]] >= 0) return set_error(LVS_ERR_ARG, "lvs_plan_pair: repeated subset symbol");
            row_of[subset[k]] = (int32_t)k;
        }
    if (pre)
        for (size_t j = 0; j < n; ++j)
            if (row_of[plain[j]] < 0) return set_error(LVS_ERR_ARG, "lvs_plan_pair: plain symbol outside the subset");
    lvs_plan_layout L;
    L.a = L.b = L.path = L.eq1 = L.eq9 = L.table = -1;
    size_t r = 0;
    if (pre) { L.table = 0; r += nsub * m; }
    else { L.a = (int64_t)r; r += m * P.C; L.b = (int64_t)r; r += n * P.C; }
    L.v = (int64_t)r; r += m;
    L.h = (int64_t)r; r += n;
    if (P.band >= 0) { L.path = (int64_t)r; r += m + n; }
    if (!pre) {
        if (P.C == 2) { L.eq1 = (int64_t)r; r += 2 * m; }
        L.eq9 = (int64_t)r; r += 2 * m;
    }
    L.rows = (int64_t)r;
    // one word per row: a row's index is its offset from the base
    std::vector<uint64_t> base(r + 1);
    Arena A;
    A.d = base.data();
    A.stride = 1;
    A.rows = r;
    if (!pre) { P.x = (size_t)L.a; P.y = (size_t)L.b; }
    P.v = (size_t)L.v;
    P.h = (size_t)L.h;
    if (P.band >= 0) P.tap = (size_t)L.path;
    if (!pre) {
        if (P.C == 2) P.eq1 = (size_t)L.eq1;
        P.eq9 = (size_t)L.eq9;
    } else {
        P.table = A.row(0);
        P.table_stride = 1;
        P.row_of = row_of;
        P.plain = plain;
    }
    const long steps = pair_steps(P);
    L.steps = steps;
    std::vector<Job> J;
    std::vector<int64_t> step_of;
    for (long st = 0; st < steps; ++st) {
        plan_pair_step(P, A, st, J);
        step_of.resize(J.size(), st);
    }
    if (layout) *layout = L;
    const size_t room = *count;
    *count = J.size();
    if (!jobs) return LVS_OK;
    if (room < J.size()) return set_error(LVS_ERR_ARG, "lvs_plan_pair: jobs has too little room");
    export_jobs(J, step_of, A.d, jobs);
    return LVS_OK;
}

lvs_status lvs_plan_batch(const size_t *m, const size_t *n, size_t npairs, uint32_t eq_lookups, int32_t band,
                          size_t wave, int64_t *launch_of, size_t *count, size_t *nlaunch)
{
    if (!count || !nlaunch || (npairs && (!m || !n))) return set_error(LVS_ERR_ARG, "lvs_plan_batch: NULL argument");
    if (eq_lookups < 1 || eq_lookups > 2) return set_error(LVS_ERR_ARG, "lvs_plan_batch: eq_lookups must be 1 or 2");
    std::vector<std::vector<uint32_t>> counts(npairs);
    size_t total = 0;
    for (size_t p = 0; p < npairs; ++p) {
        size_t cnt = 0;
        lvs_status st = lvs_plan_pair(m[p], n[p], eq_lookups, band, nullptr, nullptr, nullptr, 0, nullptr, nullptr, &cnt);
        if (st != LVS_OK) return st;
        std::vector<lvs_plan_job> J(std::max<size_t>(1, cnt));
        lvs_plan_layout L;
        st = lvs_plan_pair(m[p], n[p], eq_lookups, band, nullptr, nullptr, nullptr, 0, &L, J.data(), &cnt);
        if (st != LVS_OK) return st;
        counts[p].assign((size_t)L.steps, 0);
        for (size_t k = 0; k < cnt; ++k) counts[p][(size_t)J[k].step] += 1;
        total += (size_t)L.steps;
    }
    std::vector<std::vector<long>> lo;
    long nl = 0;
    schedule_steps(counts, wave, lo, &nl);
    const size_t room = *count;
    *count = total;
    *nlaunch = (size_t)nl;
    if (!launch_of) return LVS_OK;
    if (room < total) return set_error(LVS_ERR_ARG, "lvs_plan_batch: launch_of has too little room");
    size_t k = 0;
    for (size_t p = 0; p < npairs; ++p)
        for (long v : lo[p]) launch_of[k++] = v;
    return LVS_OK;
}

lvs_status lvs_plan_table(size_t m, lvs_alphabet alphabet, const uint8_t *subset, size_t nsub,
                          lvs_plan_layout *layout, lvs_plan_job *jobs, size_t *count)
{
    if (!count || (nsub && !subset)) return set_error(LVS_ERR_ARG, "lvs_plan_table: NULL argument");
    const uint32_t C = symbols_per_char(alphabet);
    if (alphabet_size(alphabet) == 0) return set_error(LVS_ERR_ARG, "lvs_plan_table: unknown alphabet");
    std::vector<std::pair<uint32_t, uint32_t>> sym(nsub);
    bool seen[256] = {};
    for (size_t r = 0; r < nsub; ++r) {
        uint32_t v[2] = {0, 0};
        if (!encode_char(alphabet, subset[r], v) || seen[subset[r]])
            return set_error(LVS_ERR_ARG, "lvs_plan_table: subset symbol outside the alphabet or repeated");
        seen[subset[r]] = true;
        sym[r] = {v[0], v[1]};
    }
    lvs_plan_layout L;
    L.a = 0;
    L.b = L.v = L.h = L.path = L.eq9 = -1;
    size_t r = m * C;
    L.eq1 = C == 2 ? (int64_t)r : -1;
    if (C == 2) r += nsub * m;
    L.table = (int64_t)r;
    r += nsub * m;
    L.rows = (int64_t)r;
    L.steps = (m && nsub) ? (int64_t)C : 0;
    std::vector<uint64_t> base(r + 1);
    uint64_t *b0 = base.data();
    std::vector<Job> J;
    std::vector<int64_t> step_of;
    for (int st = 0; st < (int)L.steps; ++st) {
        table_step_jobs(
            st, C, m, sym, [&](size_t i, int s) { return b0 + i * C + s; },
            [&](size_t k, size_t i) { return b0 + L.eq1 + k * m + i; },
            [&](size_t k, size_t i) { return b0 + L.table + k * m + i; }, J);
        step_of.resize(J.size(), st);
    }
    if (layout) *layout = L;
    const size_t room = *count;
    *count = J.size();
    if (!jobs) return LVS_OK;
    if (room < J.size()) return set_error(LVS_ERR_ARG, "lvs_plan_table: jobs has too little room");
    export_jobs(J, step_of, b0, jobs);
    return LVS_OK;
}

lvs_status lvs_edit_distance_preprocessed_batch(lvs_ctx *ctx, const lvs_eq_table *const *t, const uint8_t *const *plain,
                                                const size_t *plain_len, size_t nq, const lvs_opts *opts,
                                                lvs_result **out)
{
    if (!ctx || !out || (nq && (!t || !plain || !plain_len)))
        return set_error(LVS_ERR_ARG, "lvs_edit_distance_preprocessed_batch: NULL argument");
    lvs_opts o;
    lvs_opts_default(&o);
    if (opts) o = *opts;
    const bool banded = o.band >= 0;
    std::vector<PairRows> pairs(nq);
    size_t vrows = 0, hrows = 0, trows = 0;
    for (size_t q = 0; q < nq; ++q) {
        if (!t[q] || (plain_len[q] && !plain[q])) return set_error(LVS_ERR_ARG, "NULL table or string");
        if (t[q]->P.p.N != ctx->P.p.N || t[q]->device != ctx->device)
            return set_error(LVS_ERR_ARG, "table does not belong to this context");
        for (size_t j = 0; j < plain_len[q]; ++j)
            if (t[q]->row_of[plain[q][j]] < 0)
                return set_error(LVS_ERR_ARG, "query " + std::to_string(q) + ": plaintext character " +
                                                  std::to_string(plain[q][j]) + " is not in the table subset");
        PairRows &P = pairs[q];
        P.m = t[q]->len;
        P.n = plain_len[q];
        P.table = t[q]->d;
        P.table_stride = t[q]->stride;
        P.row_of = t[q]->row_of;
        P.plain = plain[q];
        if (banded) {
            P.band = o.band;
            trows += P.m + P.n;
        }
        lvs_status st = plan_refresh(ctx, o.refresh_budget, P);
        if (st != LVS_OK) return st;
        vrows += P.m;
        hrows += P.n;
    }
    LVS_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lock(ctx->mu);
    for (size_t q = 0; q < nq; ++q)
        if (t[q]->done) LVS_CUDA(cudaStreamWaitEvent(ctx->stream, t[q]->done, 0));
    // rows: [v][h][band taps]
    Arena A;
    lvs_status st = arena_alloc(ctx, vrows + hrows + trows, A);
    if (st != LVS_OK) return st;
    size_t cv = 0, ch = vrows, ct = vrows + hrows;
    for (auto &P : pairs) {
        P.v = cv; cv += P.m;
        P.h = ch; ch += P.n;
        if (banded) { P.tap = ct; ct += P.m + P.n; }
    }
    // OneMatrix boundary (and the band's path, whose out-of-band steps keep it)
    cudaError_t e = launch_fill_trivial(A.d, A.stride, ctx->P.big(), 0, vrows + hrows + trows, 1ull << kDeltaLog,
                                        ctx->stream);
    if (e != cudaSuccess) { arena_free(ctx, A); return cuda_error(e, "fill"); }
    ctx->launches += vrows + hrows + trows ? 1 : 0;
    st = run_wavefront(ctx, pairs, A, o.use_graph != 0);
    if (st != LVS_OK) { arena_free(ctx, A); return st; }
    lvs_result *r = nullptr;
    const size_t out_rows = banded ? trows : hrows;
    if ((st = make_result(ctx, out_rows, &r)) != LVS_OK) { arena_free(ctx, A); return st; }
    size_t first = 0;
    for (auto &P : pairs) {
        const size_t cnt = banded ? P.m + P.n : P.n;
        r->items.push_back({P.m, P.n, first, cnt, banded ? 0L : (long)P.m});
        first += cnt;
    }
    if (out_rows) {
        e = cudaMemcpy2DAsync(r->d, r->stride * 8, A.row(banded ? vrows + hrows : vrows), A.stride * 8,
                              (ctx->P.big() + 1) * 8, out_rows, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) { arena_free(ctx, A); lvs_result_free(r); return cuda_error(e, "result copy"); }
    }
    arena_free(ctx, A);
    if ((st = finish_result(ctx, r)) != LVS_OK) { lvs_result_free(r); return st; }
    *out = r;
    return LVS_OK;
}

lvs_status lvs_ct_string_pin(lvs_ct_string *s)
{
    if (!s) return set_error(LVS_ERR_ARG, "lvs_ct_string_pin: NULL string");
    if (s->pinned || s->data.empty()) return LVS_OK;
    uint64_t *h = nullptr;
    if (cudaMallocHost((void **)&h, s->data.size() * 8) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LVS_ERR_OOM, "lvs_ct_string_pin: page-locked allocation failed");
    }
    memcpy(h, s->data.data(), s->data.size() * 8);
    s->pinned = h;
    return LVS_OK;
}

lvs_status lvs_ct_string_upload(lvs_ctx *ctx, lvs_ct_string *s)
{
    if (!ctx || !s) return set_error(LVS_ERR_ARG, "lvs_ct_string_upload: NULL argument");
    lvs_status st = check_ctx_string(ctx, s);
    if (st != LVS_OK) return st;
    if (s->d && s->ddevice == ctx->device) return LVS_OK;
    if (s->d) return set_error(LVS_ERR_STATE, "lvs_ct_string_upload: string already resident on another device");
    const size_t rows = s->len * s->symbols;
    if (rows == 0) return LVS_OK;
    LVS_CUDA(cudaSetDevice(ctx->device));
    const size_t stride = (size_t)s->big + 2, w = (size_t)s->big + 1;
    uint64_t *d = nullptr;
    if (cudaMalloc((void **)&d, rows * stride * 8) != cudaSuccess) {
        cudaGetLastError();
        return set_error(LVS_ERR_OOM, "lvs_ct_string_upload: device allocation failed");
    }
    cudaError_t e = cudaMemcpy2D(d, stride * 8, s->host(), w * 8, w * 8, rows, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_error(e, "lvs_ct_string_upload"); }
    s->d = d;
    s->dstride = stride;
    s->ddevice = ctx->device;
    return LVS_OK;
}

lvs_status lvs_result_info(const lvs_result *r, size_t *items, size_t pair, size_t *m, size_t *n)
{
    if (!r) return set_error(LVS_ERR_ARG, "lvs_result_info: NULL result");
    if (items) *items = r->items.size();
    if (m || n) {
        if (pair >= r->items.size()) return set_error(LVS_ERR_ARG, "lvs_result_info: item out of range");
        if (m) *m = r->items[pair].m;
        if (n) *n = r->items[pair].n;
    }
    return LVS_OK;
}

lvs_status lvs_result_export(const lvs_result *r, size_t pair, uint64_t *dst, size_t *words)
{
    if (!r || !words) return set_error(LVS_ERR_ARG, "lvs_result_export: NULL argument");
    if (pair >= r->items.size()) return set_error(LVS_ERR_ARG, "lvs_result_export: item out of range");
    const auto &it = r->items[pair];
    const size_t w = (size_t)r->P.big() + 1;
    if (dst) {
        if (*words < it.count * w) return set_error(LVS_ERR_ARG, "lvs_result_export: destination too small");
        LVS_CUDA(cudaSetDevice(r->device));
        LVS_CUDA(cudaEventSynchronize(r->done));
        if (lvs_status st = device_fault_check(r->device); st != LVS_OK) return st;
        if (it.count)
            LVS_CUDA(cudaMemcpy2D(dst, w * 8, r->d + it.first * r->stride, r->stride * 8, w * 8, it.count,
                                  cudaMemcpyDeviceToHost));
    }
    *words = it.count * w;
    return LVS_OK;
}

void lvs_result_free(lvs_result *r)
{
    if (!r) return;
    cudaSetDevice(r->device);
    if (r->done) { cudaEventSynchronize(r->done); cudaEventDestroy(r->done); }
    // cudaFree waits for the device, so work still reading r (lvs_result_sum) ends first
    if (r->d) cudaFree(r->d);
    cudaGetLastError();
    delete r;
}

static lvs_status decrypt_rows(const lvs_client_key *ck, const lvs_result *r, const uint64_t *host, size_t pair,
                               uint32_t *out)
{
    const auto &it = r->items[pair];
    const size_t w = (size_t)r->P.big() + 1;
    if (r->is_eq) {
        *out = decrypt_lwe(*ck, host);
        return LVS_OK;
    }
    // D[m][n] = base + sum of the path differences, each in {-1, 0, 1} (Z_32
    // residues): base m with the last row h[m][1..n], base 0 with the band path
    long d = it.base;
    for (size_t j = 0; j < it.count; ++j) {
        const uint32_t v = decrypt_lwe(*ck, host + j * w);
        d += v >= 16 ? (long)v - 32 : (long)v;
    }
    *out = (uint32_t)std::max(0L, d);
    return LVS_OK;
}

lvs_status lvs_decrypt(const lvs_client_key *ck, const lvs_result *r, size_t pair, uint32_t *dist)
{
    if (!ck || !r || !dist) return set_error(LVS_ERR_ARG, "lvs_decrypt: NULL argument");
    if (pair >= r->items.size()) return set_error(LVS_ERR_ARG, "lvs_decrypt: item out of range");
    if (ck->P.big() != r->P.big()) return set_error(LVS_ERR_ARG, "lvs_decrypt: key does not match the result");
    size_t words = 0;
    lvs_status st = lvs_result_export(r, pair, nullptr, &words);
    if (st != LVS_OK) return st;
    std::vector<uint64_t> host(words);
    if ((st = lvs_result_export(r, pair, host.data(), &words)) != LVS_OK) return st;
    return decrypt_rows(ck, r, host.data(), pair, dist);
}

lvs_status lvs_decrypt_distance(const lvs_client_key *ck, const uint64_t *rows, size_t count, int64_t base,
                                uint32_t *dist)
{
    if (!ck || !dist || (count && !rows)) return set_error(LVS_ERR_ARG, "lvs_decrypt_distance: NULL argument");
    const size_t w = (size_t)ck->P.big() + 1;
    long d = (long)base;
    for (size_t j = 0; j < count; ++j) {
        const uint32_t v = decrypt_lwe(*ck, rows + j * w);
        d += v >= 16 ? (long)v - 32 : (long)v;
    }
    *dist = (uint32_t)std::max(0L, d);
    return LVS_OK;
}

lvs_status lvs_decrypt_all(const lvs_client_key *ck, const lvs_result *r, uint32_t *dist)
{
    if (!ck || !r || (!dist && !r->items.empty())) return set_error(LVS_ERR_ARG, "lvs_decrypt_all: NULL argument");
    if (r->items.empty()) return LVS_OK;
    const size_t w = (size_t)r->P.big() + 1;
    size_t total = 0;
    for (const auto &it : r->items) total = std::max(total, it.first + it.count);
    std::vector<uint64_t> host(total * w);
    LVS_CUDA(cudaSetDevice(r->device));
    LVS_CUDA(cudaEventSynchronize(r->done));
    if (lvs_status st = device_fault_check(r->device); st != LVS_OK) return st;
    if (total)
        LVS_CUDA(cudaMemcpy2D(host.data(), w * 8, r->d, r->stride * 8, w * 8, total, cudaMemcpyDeviceToHost));
    for (size_t p = 0; p < r->items.size(); ++p) {
        lvs_status st = decrypt_rows(ck, r, host.data() + r->items[p].first * w, p, dist + p);
        if (st != LVS_OK) return st;
    }
    return LVS_OK;
}

}  // extern "C"
