// Internal declarations of the GB300 Leuvenshtein library (not part of the ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lvs.h"

namespace lvs {

// ----------------------------------------------------------------- errors
lvs_status set_error(lvs_status st, const std::string &msg);
lvs_status cuda_error(cudaError_t e, const char *what);
#define LVS_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e__ = (call);                                             \
        if (e__ != cudaSuccess) return ::lvs::cuda_error(e__, #call);         \
    } while (0)

// ----------------------------------------------------------------- constants
constexpr int kPrimes = 3;
// Three NTT primes p = c * 2^12 + 1 < 2^30 (2N-th roots of unity exist for
// N <= 2048; 4p < 2^32 allows lazy butterflies).  Their product M > 2^89
// bounds the exact integer external product (|coef| <= 4 * N * 2^12 * 2^63).
constexpr uint32_t kPrime[kPrimes] = {0x3fff4001u, 0x3ffee001u, 0x3ffeb001u};
constexpr int kDeltaLog = 59;      // q / 32
constexpr int kRows = 4;           // (k+1) * pbs_level with k = 1, level = 2
constexpr int kMaxJobsPerLaunch = 1 << 20;

// LUT ids in the context's LUT table
enum : uint8_t { LUT_EQ = 0, LUT_EQ9 = 1, LUT_MIN = 2, LUT_V = 3, LUT_USER0 = 8 };
// job kinds (epilogue of the blind-rotation kernel)
enum : uint8_t { JOB_STORE = 0, JOB_CELL = 1 };

// One PBS of a wavefront launch.  Input = sum_s coef[s] * (*src[s]) +
// cst * Delta, a linear combination of big ciphertexts (Section 2.2 linear
// operations); output written by the epilogue `kind`:
//   STORE: *dst[0] = PBS
//   CELL : M = PBS; *dst[0] (v) = M - *dst[1]_old (h),
//                   *dst[1] (h) = M - *dst[0]_old (v)      (Section 3.1.1)
//          and, for a cell on the readout path of a band, a copy of the new
//          v (tapsel 1) or h (tapsel 2) to *tap.
// All pointers are device rows of k*N+1 words.
struct alignas(16) Job {
    const uint64_t *src[3];
    uint64_t *dst[2];
    uint64_t *tap;
    int8_t coef[3];
    int8_t cst;
    uint8_t lut;
    uint8_t kind;
    uint8_t tapsel;
    uint8_t pad[9];
};
static_assert(sizeof(Job) == 64, "Job layout");

// ----------------------------------------------------------------- host keys
struct Params {
    lvs_params p;
    uint32_t big() const { return p.k * p.N; }
    uint32_t log_n() const { uint32_t l = 0; while ((1u << l) < p.N) ++l; return l; }
    size_t bsk_words() const { return (size_t)p.n * (p.k + 1) * p.pbs_level * (p.k + 1) * p.N; }
    size_t ksk_words() const { return (size_t)p.k * p.N * p.ks_level * (p.n + 1); }
};
lvs_status check_params(const lvs_params &p);

}  // namespace lvs

struct lvs_client_key {
    lvs::Params P;
    std::vector<uint64_t> lwe_key;   // n
    std::vector<uint64_t> glwe_key;  // k*N
};

struct lvs_server_key {
    lvs::Params P;
    std::vector<uint64_t> bsk;  // coefficient domain
    std::vector<uint64_t> ksk;
};

struct lvs_ct_string {
    lvs_alphabet alphabet;
    uint32_t symbols;   // per character
    uint32_t big;       // k*N
    size_t len;         // characters
    std::vector<uint64_t> data;  // [len][symbols][big+1]
    uint64_t *d = nullptr;       // optional device copy, rows of `dstride` words
    size_t dstride = 0;
    int ddevice = -1;
    uint64_t *pinned = nullptr;  // optional page-locked copy of `data` (lvs_ct_string_pin)
    const uint64_t *host() const { return pinned ? pinned : data.data(); }
};

namespace lvs {
uint32_t symbols_per_char(lvs_alphabet a);
// character -> (symbol values); returns false if outside the alphabet
bool encode_char(lvs_alphabet a, uint8_t c, uint32_t sym[2]);
uint32_t alphabet_size(lvs_alphabet a);
uint8_t alphabet_char(lvs_alphabet a, uint32_t idx);
void encrypt_lwe(const lvs_client_key &ck, uint32_t value, uint64_t seed, uint64_t i0, uint64_t i1,
                 uint64_t *ct);
uint32_t decrypt_lwe(const lvs_client_key &ck, const uint64_t *ct);

struct Timing {
    bool enabled = false;
    // one launch step: key switch between a and b, blind rotation between b and c
    struct Pending { cudaEvent_t a, b, c; uint64_t items; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    lvs_kernel_stats stats[2] = {};
};

}  // namespace lvs

namespace lvs {
struct KsGemm;   // tensor-core key switch (ks_gemm.cu)
// key-switch launch shape: jobs per CTA (4 or 16) and split of the input
// coefficients over gridDim.z; one plan per launch-size bucket
struct KsPlan { int tj = 0; int split = 1; };
constexpr int kKsBuckets = 6;   // launch sizes 1-4, 5-16, 17-64, 65-256, 257-1024, more
inline int ks_bucket(size_t njobs)
{
    int b = 0;
    for (size_t lim = 4; b < kKsBuckets - 1 && njobs > lim; lim *= 4) ++b;
    return b;
}
}  // namespace lvs

struct lvs_ctx {
    lvs::Params P;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int br_grid = 0;
    int br_clusters = 0;           // resident clusters of the three-CTA blind rotation
    size_t br_split_max = 0;       // launches of at most this many PBS use it (0: never)
    // device keys
    uint32_t *bsk_ntt = nullptr;   // [n][kPrimes][16][q][key_lane_word order] u32
    uint32_t *fault_dev = nullptr; // device view of this device's give-up word (device_fault_word)
    int key_staging = 0;           // 1: key-staged blind rotation (head of each BSK row by bulk copy)
    bool debug_drop_key_copy = false; // tests: the staged form never issues one warp's copies
    uint64_t *ksk = nullptr;       // [kN][ks_l][n+1]
    uint64_t *ksk_colsum = nullptr; // [n+1]: column sums of the KSK
    uint32_t *tw = nullptr;        // twiddles: uint2 {w, w_shoup} [prime][fwd, inv][N]
    uint8_t *luts = nullptr;       // [256][16]
    // optional FP64-FFT key (lvs_ctx_prepare_fft64)
    double *bsk_fft = nullptr;     // [n][8][N/2] complex
    double *fft_tw = nullptr;      // twiddles: [N/4] complex exp(2 pi i t/(N/2)), then [N/2] complex exp(i pi j/N)
    int fft_grid = 0;
    // scratch (grown on demand; owned by the context)
    uint32_t *ms = nullptr;        // [ms_cap][n+1] modulus-switched masks of one launch
    size_t ms_cap = 0;
    lvs::Job *jobs = nullptr;      // [jobs_cap] jobs of a whole run
    size_t jobs_cap = 0;
    uint64_t *ks_part = nullptr;   // split key-switch partial sums
    size_t ks_part_cap = 0;        // words
    lvs::KsPlan ks_tuned[lvs::kKsBuckets];   // autotuned plans (tj = 0: default heuristic)
    lvs::KsGemm *ks_gemm = nullptr;  // key switch on the tensor cores (null: unavailable)
    size_t ks_gemm_min = 0;          // launches of at least this many PBS use it (0: never)
    size_t max_launch_jobs = (size_t)1 << 16;   // wider wavefront steps run as several launches
    bool wave_fill = true;         // batch calls hold pairs back to end launches on full waves
    uint64_t pbs_done = 0;
    uint64_t launches = 0;
    lvs::Timing timing;
    struct GraphRun { cudaGraphExec_t exec; cudaEvent_t done; };
    std::vector<GraphRun> graphs;  // launched graphs, destroyed once complete
    std::mutex mu;
};

struct lvs_result {
    lvs::Params P;
    int device = 0;
    uint64_t *d = nullptr;            // device rows [total][stride], owned
    size_t stride = 0;                // words per row (>= k*N+1)
    // distance = base + sum of the decrypted rows [first, first + count)
    struct Item { size_t m, n, first, count; long base; };
    std::vector<Item> items;
    bool is_eq = false;
    cudaEvent_t done = nullptr;       // recorded after the producing launches
};

struct lvs_eq_table {
    lvs::Params P;
    int device = 0;
    lvs_alphabet alphabet = LVS_ALPHA_ASCII7;
    size_t len = 0;                   // characters of the encrypted string
    std::vector<uint8_t> subset;      // plaintext characters, one table row each
    int32_t row_of[256];              // character -> row, -1 if absent
    uint64_t *d = nullptr;            // device rows [nsub][len][stride], owned
    size_t stride = 0;
    cudaEvent_t done = nullptr;
};

namespace lvs {
namespace dev { struct PrimeConsts; }
// kernel launch wrappers (kernels.cu)
cudaError_t upload_prime_consts(const dev::PrimeConsts &pc);
cudaError_t prepare_kernels(uint32_t N);
cudaError_t launch_bsk_to_ntt_count(uint32_t N, const uint64_t *coef, uint32_t count, uint32_t *out,
                                    const uint32_t *tw, const uint32_t mont[3][2], cudaStream_t s);
// nlaunch (optional): kernels launched (2 with a split: the key switch and its finishing reduction)
cudaError_t launch_keyswitch(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                             int *nlaunch = nullptr);
cudaError_t launch_keyswitch_plan(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, uint64_t *part,
                                  KsPlan pl, cudaStream_t s);
// tensor-core key switch (ks_gemm.cu)
lvs_status ks_gemm_init(lvs_ctx *ctx);
void ks_gemm_free(lvs_ctx *ctx);
cudaError_t launch_keyswitch_gemm(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                                  int *nlaunch);
// the key switch of a launch, in the form its size calls for
cudaError_t launch_keyswitch_auto(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                                  int *nlaunch = nullptr);
KsPlan ks_plan(const lvs_ctx *ctx, size_t njobs);
size_t ks_part_words(const lvs_ctx *ctx, size_t njobs);
cudaError_t launch_ksk_colsum(const lvs_ctx *ctx, cudaStream_t s);
cudaError_t launch_blind_rotate(const lvs_ctx *ctx, const Job *jobs, size_t njobs, const uint32_t *ms,
                                const uint8_t *luts, int lut_per_job, cudaStream_t s);
cudaError_t launch_poly_mul(const lvs_ctx *ctx, const int32_t *dig, const uint32_t *keyntt, uint64_t *out,
                            size_t count, cudaStream_t s);
cudaError_t launch_fill_trivial(uint64_t *arena, size_t stride, uint32_t big, size_t first, size_t count,
                                uint64_t body, cudaStream_t s);
int br_smem_bytes(uint32_t N);
int br_cluster_capacity(uint32_t N);
int br_threads(uint32_t N);
size_t bsk_ntt_words(uint32_t n, uint32_t N);
// Per-device word in mapped pinned host memory that a kernel sets when one of
// its bounded device-side waits gives up (allocated once per device, kept for
// the life of the process); device_fault_check reads and clears it:
// LVS_ERR_TIMEOUT if it was set.  Call after the work has been synchronized.
uint32_t *device_fault_word(int device);
lvs_status device_fault_check(int device);

// host tables (tables.cu)
void make_twiddles(uint32_t N, std::vector<uint32_t> &out);
void make_prime_consts(dev::PrimeConsts &pc);
void make_mont(uint32_t N, uint32_t mont[3][2]);
void make_luts(std::vector<uint8_t> &table);   // [256][16]

// ----------------------------------------------------------------- planner (sched.cu)
struct Arena {
    uint64_t *d = nullptr;
    size_t stride = 0;
    size_t rows = 0;
    uint64_t *row(size_t r) const { return d + r * stride; }
};

// Per pair plan: the rows of its strings, frontier and rings.
struct PairRows {
    size_t m = 0, n = 0;
    uint32_t C = 2;          // equality lookups per cell (2 ASCII / 27, 1 DNA)
    size_t x = 0, y = 0;     // first arena row of a / b (row = first + char * C + symbol)
    const uint64_t *xd = nullptr, *yd = nullptr;   // device-resident strings (else arena rows)
    size_t xs = 0, ys = 0;                         // their row strides
    size_t v = 0, h = 0;     // v[i] at v + i - 1, h[j] at h + j - 1
    size_t eq1 = 0, eq9 = 0; // ring rows: + (d & 1) * m + i - 1
    const uint64_t *table = nullptr;   // preprocessed path: rows T[row][i]
    size_t table_stride = 0;
    const int32_t *row_of = nullptr;
    const uint8_t *plain = nullptr;
    long band = -1;          // >= 0: only cells with |i - j| <= band (square pairs)
    size_t tap = 0;          // band: m + n rows, the readout path [v[1][0], h[1][1], ..., v[r][r-1], h[r][r],
                             // then h[m][m+1..n] or v[r+1..m][n]], r = min(m, n)
    std::vector<uint8_t> refresh;   // empty, or [m + n + 1]: 1 if anti-diagonal i + j is refreshed
};

lvs_status arena_alloc(lvs_ctx *ctx, size_t rows, Arena &A);
void arena_free(lvs_ctx *ctx, Arena &A);
lvs_status upload_string(lvs_ctx *ctx, const lvs_ct_string *s, const Arena &A, size_t first);
Job make_job(const uint64_t *s0, int c0, const uint64_t *s1, int c1, const uint64_t *s2, int c2, int cst,
             uint8_t lut, uint8_t kind, uint64_t *d0, uint64_t *d1);
lvs_status make_result(lvs_ctx *ctx, size_t rows, lvs_result **out);
lvs_status finish_result(lvs_ctx *ctx, lvs_result *r);
// Jobs of step `step` of the Section 5 table build of one encrypted string of m
// characters against subset symbols sym (their two plaintext halves).  Two
// lookups (C = 2): step 0 EQ1[r][i] = PBS(x1_i - sigma1_r; LUT_EQ), step 1
// T[r][i] = PBS(2 (x2_i - sigma2_r) + 1 - EQ1[r][i]; LUT_EQ9).  DNA (C = 1):
// step 0 T[r][i] = PBS(x_i - sigma_r; LUT_EQ9).  X(i, s) is the row of symbol s
// of character i (from 0), E1(r, i) and T(r, i) the rows of EQ1 and of the table.
template <class FX, class FE, class FT>
void table_step_jobs(int step, uint32_t C, size_t m, const std::vector<std::pair<uint32_t, uint32_t>> &sym, FX X,
                     FE E1, FT T, std::vector<Job> &jobs)
{
    for (size_t r = 0; r < sym.size(); ++r)
        for (size_t i = 0; i < m; ++i) {
            if (C == 1) {
                if (step == 0)
                    jobs.push_back(make_job(X(i, 0), 1, nullptr, 0, nullptr, 0, -(int)sym[r].first, LUT_EQ9, JOB_STORE,
                                            T(r, i), nullptr));
            } else if (step == 0) {
                jobs.push_back(make_job(X(i, 0), 1, nullptr, 0, nullptr, 0, -(int)sym[r].first, LUT_EQ, JOB_STORE,
                                        E1(r, i), nullptr));
            } else {
                jobs.push_back(make_job(X(i, 1), 2, E1(r, i), -1, nullptr, 0, 1 - 2 * (int)sym[r].second, LUT_EQ9,
                                        JOB_STORE, T(r, i), nullptr));
            }
        }
}
// launch index of every step of every pair from the PBS count of each step: the
// launches fill the waves of a grid of `wave` concurrent jobs (0: all pairs step
// together); nlaunch = number of launches
void schedule_steps(const std::vector<std::vector<uint32_t>> &counts, size_t wave,
                    std::vector<std::vector<long>> &launch_of, long *nlaunch);
// jobs of wavefront step s of one pair (cells of anti-diagonal s - depth, etc.)
void plan_pair_step(const PairRows &P, const Arena &A, long s, std::vector<Job> &jobs);
// number of steps of one pair (0 if it has no cell)
long pair_steps(const PairRows &P);
lvs_status check_ctx_string(const lvs_ctx *ctx, const lvs_ct_string *s);

// noise budget and refresh plan (noise.cu)
double noise_budget(const lvs_params &p, double log2_pfail);
lvs_status noise_plan(size_t m, size_t n, long band, double budget, std::vector<uint8_t> *refresh, double *worst);
// refresh_budget: 0 = from the parameters (failure probability 2^-64), > 0 = explicit, < 0 = none
lvs_status plan_refresh(const lvs_ctx *ctx, int32_t refresh_budget, PairRows &P);

// scratch and timing (ctx.cu)
lvs_status ensure_scratch(lvs_ctx *ctx, size_t njobs_total, size_t njobs_step);
lvs_status run_steps(lvs_ctx *ctx, const std::vector<Job> &jobs, const std::vector<size_t> &step_off,
                     bool use_graph);
void timing_collect(lvs_ctx *ctx);
// a timing event from the context's pool (created if the pool is empty; null on failure)
cudaEvent_t pool_event(lvs_ctx *ctx);
// events created up front by lvs_ctx_set_timing(ctx, 1): one launch step uses three
constexpr size_t kTimingPoolEvents = 48;
}  // namespace lvs
