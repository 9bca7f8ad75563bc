// Host side of the library: parameters, errors, key generation, client-side
// encryption / decryption and the string / key handles.
//
// Randomness: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
// number generators", OOPSLA 2014) taken as a counter-based generator: the
// c-th word of the stream whose state is K is mix64(K + (c + 1) * gamma).
// A stream is named by (seed, tag, i0, i1): K = f(f(f(seed ^ tag) ^ i0) ^ i1)
// with f(x) = mix64(x + gamma).  Noise is TUniform(b): with r the low b+2 bits
// of one word, e = ceil(r / 2) - 2^b, uniform on [-2^b, 2^b] with half weight
// at both ends.  Keys are binary (each key bit = the top bit of one word).
#include <algorithm>
#include <cstring>
#include <functional>
#include <new>
#include <thread>

#include "lvs_internal.hpp"

namespace lvs {

static thread_local std::string g_last_error;

lvs_status set_error(lvs_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

lvs_status cuda_error(cudaError_t e, const char *what)
{
    return set_error(LVS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------- generator
namespace rng {
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
inline uint64_t mix64(uint64_t z)
{
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27; z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
inline uint64_t first(uint64_t state) { return mix64(state + kGamma); }
inline uint64_t word(uint64_t state, uint64_t c) { return mix64(state + (c + 1) * kGamma); }
inline uint64_t stream(uint64_t seed, uint64_t tag, uint64_t i0, uint64_t i1)
{
    return first(first(first(seed ^ tag) ^ i0) ^ i1);
}
inline int64_t tuniform(uint64_t w, uint32_t b)
{
    const uint64_t r = w & ((uint64_t(1) << (b + 2)) - 1);
    return int64_t((r + 1) >> 1) - (int64_t(1) << b);
}
enum : uint64_t { TAG_LWE_KEY = 1, TAG_GLWE_KEY = 2, TAG_BSK = 3, TAG_KSK = 4, TAG_ENC = 5 };
}  // namespace rng

lvs_status check_params(const lvs_params &p)
{
    if (p.k != 1) return set_error(LVS_ERR_ARG, "params: only k = 1 is supported");
    if (p.N != 512 && p.N != 2048) return set_error(LVS_ERR_ARG, "params: N must be 512 or 2048");
    if (p.n < 1 || p.n > 4096) return set_error(LVS_ERR_ARG, "params: n out of range [1, 4096]");
    if (p.pbs_level != 2 || p.pbs_base_log < 1 || p.pbs_level * p.pbs_base_log > 26)
        return set_error(LVS_ERR_ARG, "params: the NTT path needs pbs_level = 2 and level * base_log <= 26");
    if (p.ks_level < 1 || p.ks_base_log < 1 || p.ks_level * p.ks_base_log > 30 || p.ks_level > 8)
        return set_error(LVS_ERR_ARG, "params: ks gadget out of range");
    if (p.lwe_noise_log2 > 60 || p.glwe_noise_log2 > 60)
        return set_error(LVS_ERR_ARG, "params: noise bound too large");
    return LVS_OK;
}

// ---------------------------------------------------------------- alphabets
uint32_t symbols_per_char(lvs_alphabet a) { return a == LVS_ALPHA_DNA4 ? 1 : 2; }

uint32_t alphabet_size(lvs_alphabet a)
{
    switch (a) {
    case LVS_ALPHA_ASCII7: return 128;
    case LVS_ALPHA_27: return 27;
    case LVS_ALPHA_DNA4: return 4;
    }
    return 0;
}

uint8_t alphabet_char(lvs_alphabet a, uint32_t idx)
{
    switch (a) {
    case LVS_ALPHA_ASCII7: return (uint8_t)idx;
    case LVS_ALPHA_27: return idx == 26 ? ' ' : (uint8_t)('A' + idx);
    case LVS_ALPHA_DNA4: return (uint8_t)"ACGT"[idx & 3];
    }
    return 0;
}

bool encode_char(lvs_alphabet a, uint8_t c, uint32_t sym[2])
{
    uint32_t idx;
    switch (a) {
    case LVS_ALPHA_ASCII7:
        if (c >= 128) return false;
        idx = c;
        break;
    case LVS_ALPHA_27:
        if (c == ' ') idx = 26;
        else if (c >= 'A' && c <= 'Z') idx = c - 'A';
        else return false;
        break;
    case LVS_ALPHA_DNA4: {
        const char *p = (const char *)memchr("ACGT", c, 4);
        if (!p || c == 0) return false;
        sym[0] = (uint32_t)(p - "ACGT");
        return true;
    }
    default:
        return false;
    }
    sym[0] = idx & 15;   // 4-bit symbol x1
    sym[1] = idx >> 4;   // 3-bit (or 1-bit) symbol x2
    return true;
}

// ---------------------------------------------------------------- LWE
void encrypt_lwe(const lvs_client_key &ck, uint32_t value, uint64_t seed, uint64_t i0, uint64_t i1,
                 uint64_t *ct)
{
    const uint32_t d = ck.P.big();
    const uint64_t st = rng::stream(seed, rng::TAG_ENC, i0, i1);
    uint64_t b = 0;
    for (uint32_t c = 0; c < d; ++c) {
        const uint64_t a = rng::word(st, c);
        ct[c] = a;
        b += a & (0 - ck.glwe_key[c]);
    }
    b += (uint64_t)rng::tuniform(rng::word(st, d), ck.P.p.glwe_noise_log2);
    ct[d] = b + ((uint64_t)(value & 31u) << kDeltaLog);
}

uint32_t decrypt_lwe(const lvs_client_key &ck, const uint64_t *ct)
{
    const uint32_t d = ck.P.big();
    uint64_t s = 0;
    for (uint32_t c = 0; c < d; ++c) s += ct[c] & (0 - ck.glwe_key[c]);
    const uint64_t ph = ct[d] - s;
    return (uint32_t)(((ph + (uint64_t(1) << (kDeltaLog - 1))) >> kDeltaLog) & 31u);
}

// ---------------------------------------------------------------- keygen
// GLWE row (k = 1): mask A uniform, body = A * S + e (negacyclic, S binary:
// the product is the sum of the rotations X^u * A over the set bits u of S).
static void glwe_row(const Params &P, const std::vector<uint32_t> &ones, uint64_t key, uint64_t *row)
{
    const uint32_t N = P.p.N;
    uint64_t *A = row, *B = row + N;
    for (uint32_t t = 0; t < N; ++t) A[t] = rng::word(key, t);
    for (uint32_t t = 0; t < N; ++t) B[t] = (uint64_t)rng::tuniform(rng::word(key, N + t), P.p.glwe_noise_log2);
    for (uint32_t u : ones) {
        // B += X^u * A
        for (uint32_t t = u; t < N; ++t) B[t] += A[t - u];
        for (uint32_t t = 0; t < u; ++t) B[t] -= A[t + N - u];
    }
}

static void parallel_for(size_t n, const std::function<void(size_t)> &f)
{
    unsigned T = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
    if (n < 2 || T == 1) {
        for (size_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < T; ++t)
        th.emplace_back([&, t] { for (size_t i = t; i < n; i += T) f(i); });
    for (auto &x : th) x.join();
}

}  // namespace lvs

using namespace lvs;

extern "C" {

const char *lvs_last_error(void) { return g_last_error.c_str(); }
const char *lvs_version(void) { return "lvs-gb300 0.1 (sm_103a)"; }

void lvs_params_default(lvs_params *o)
{
    if (!o) return;
    *o = lvs_params{834, 1, 2048, 2, 13, 5, 3, 45, 17};
}

void lvs_params_test(lvs_params *o)
{
    if (!o) return;
    *o = lvs_params{64, 1, 512, 2, 13, 5, 3, 45, 17};
}

void lvs_opts_default(lvs_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->band = -1;
    o->use_graph = 1;
}

lvs_status lvs_keygen(const lvs_params *params, uint64_t seed, lvs_client_key **client,
                      lvs_server_key **server)
{
    if (!params || !client || !server) return set_error(LVS_ERR_ARG, "lvs_keygen: NULL argument");
    lvs_status st = check_params(*params);
    if (st != LVS_OK) return st;
    lvs_client_key *ck = nullptr;
    lvs_server_key *sk = nullptr;
    try {
        ck = new lvs_client_key;
        sk = new lvs_server_key;
        Params P{*params};
        ck->P = sk->P = P;
        const uint32_t n = P.p.n, N = P.p.N, k = P.p.k, L = P.p.pbs_level;
        ck->lwe_key.resize(n);
        ck->glwe_key.resize((size_t)k * N);
        const uint64_t kl = rng::stream(seed, rng::TAG_LWE_KEY, 0, 0);
        for (uint32_t i = 0; i < n; ++i) ck->lwe_key[i] = rng::word(kl, i) >> 63;
        const uint64_t kg = rng::stream(seed, rng::TAG_GLWE_KEY, 0, 0);
        for (uint32_t u = 0; u < k * N; ++u) ck->glwe_key[u] = rng::word(kg, u) >> 63;
        std::vector<uint32_t> ones;
        for (uint32_t u = 0; u < N; ++u)
            if (ck->glwe_key[u]) ones.push_back(u);

        // BSK_i: rows r = j * L + lev - 1, each a GLWE (mask, body) of 2N words
        sk->bsk.assign(P.bsk_words(), 0);
        const size_t row_words = (size_t)(k + 1) * N;
        const uint32_t rows = (k + 1) * L;
        parallel_for((size_t)n * rows, [&](size_t idx) {
            const uint32_t i = (uint32_t)(idx / rows), r = (uint32_t)(idx % rows);
            const uint32_t j = r / L, lev = r % L + 1;
            uint64_t *row = sk->bsk.data() + idx * row_words;
            glwe_row(P, ones, rng::stream(seed, rng::TAG_BSK, i, r), row);
            row[(size_t)j * N] += ck->lwe_key[i] << (64 - lev * P.p.pbs_base_log);
        });

        // KSK[u][lev]: LWE_s(S'_u * q / Bks^lev) of n+1 words
        const uint32_t ksl = P.p.ks_level;
        sk->ksk.assign(P.ksk_words(), 0);
        parallel_for((size_t)k * N, [&](size_t u) {
            for (uint32_t lev = 1; lev <= ksl; ++lev) {
                const uint64_t key = rng::stream(seed, rng::TAG_KSK, u, lev - 1);
                uint64_t *row = sk->ksk.data() + ((size_t)u * ksl + (lev - 1)) * (n + 1);
                uint64_t b = 0;
                for (uint32_t c = 0; c < n; ++c) {
                    row[c] = rng::word(key, c);
                    b += row[c] & (0 - ck->lwe_key[c]);
                }
                b += (uint64_t)rng::tuniform(rng::word(key, n), P.p.lwe_noise_log2);
                b += ck->glwe_key[u] << (64 - lev * P.p.ks_base_log);
                row[n] = b;
            }
        });
    } catch (const std::bad_alloc &) {
        delete ck;
        delete sk;
        return set_error(LVS_ERR_OOM, "lvs_keygen: host allocation failed");
    }
    *client = ck;
    *server = sk;
    return LVS_OK;
}

void lvs_client_key_free(lvs_client_key *ck) { delete ck; }
void lvs_server_key_free(lvs_server_key *sk) { delete sk; }

static lvs_status export_vec(const std::vector<uint64_t> &v, uint64_t *dst, size_t *words)
{
    if (!words) return set_error(LVS_ERR_ARG, "export: NULL size pointer");
    if (dst) {
        if (*words < v.size()) return set_error(LVS_ERR_ARG, "export: destination too small");
        memcpy(dst, v.data(), v.size() * sizeof(uint64_t));
    }
    *words = v.size();
    return LVS_OK;
}

lvs_status lvs_client_key_export(const lvs_client_key *ck, uint64_t *lwe_key, size_t *lwe_words,
                                 uint64_t *glwe_key, size_t *glwe_words)
{
    if (!ck) return set_error(LVS_ERR_ARG, "lvs_client_key_export: NULL key");
    lvs_status st = export_vec(ck->lwe_key, lwe_key, lwe_words);
    if (st != LVS_OK) return st;
    return export_vec(ck->glwe_key, glwe_key, glwe_words);
}

lvs_status lvs_server_key_export(const lvs_server_key *sk, uint64_t *bsk, size_t *bsk_words,
                                 uint64_t *ksk, size_t *ksk_words)
{
    if (!sk) return set_error(LVS_ERR_ARG, "lvs_server_key_export: NULL key");
    lvs_status st = export_vec(sk->bsk, bsk, bsk_words);
    if (st != LVS_OK) return st;
    return export_vec(sk->ksk, ksk, ksk_words);
}

lvs_status lvs_server_key_import(const lvs_params *params, const uint64_t *bsk, size_t bsk_words,
                                 const uint64_t *ksk, size_t ksk_words, lvs_server_key **out)
{
    if (!params || !bsk || !ksk || !out) return set_error(LVS_ERR_ARG, "lvs_server_key_import: NULL argument");
    lvs_status st = check_params(*params);
    if (st != LVS_OK) return st;
    Params P;
    P.p = *params;
    if (bsk_words != P.bsk_words() || ksk_words != P.ksk_words())
        return set_error(LVS_ERR_ARG, "lvs_server_key_import: key sizes do not match the parameters");
    lvs_server_key *sk = new (std::nothrow) lvs_server_key;
    if (!sk) return set_error(LVS_ERR_OOM, "lvs_server_key_import: host allocation failed");
    try {
        sk->P = P;
        sk->bsk.assign(bsk, bsk + bsk_words);
        sk->ksk.assign(ksk, ksk + ksk_words);
    } catch (const std::bad_alloc &) {
        delete sk;
        return set_error(LVS_ERR_OOM, "lvs_server_key_import: host allocation failed");
    }
    *out = sk;
    return LVS_OK;
}

lvs_status lvs_client_key_import(const lvs_params *params, const uint64_t *lwe_key, size_t lwe_words,
                                 const uint64_t *glwe_key, size_t glwe_words, lvs_client_key **out)
{
    if (!params || !lwe_key || !glwe_key || !out) return set_error(LVS_ERR_ARG, "lvs_client_key_import: NULL argument");
    lvs_status st = check_params(*params);
    if (st != LVS_OK) return st;
    Params P;
    P.p = *params;
    if (lwe_words != P.p.n || glwe_words != P.big())
        return set_error(LVS_ERR_ARG, "lvs_client_key_import: key sizes do not match the parameters");
    for (size_t i = 0; i < lwe_words; ++i)
        if (lwe_key[i] > 1) return set_error(LVS_ERR_ARG, "lvs_client_key_import: LWE key is not binary");
    for (size_t i = 0; i < glwe_words; ++i)
        if (glwe_key[i] > 1) return set_error(LVS_ERR_ARG, "lvs_client_key_import: GLWE key is not binary");
    lvs_client_key *ck = new (std::nothrow) lvs_client_key;
    if (!ck) return set_error(LVS_ERR_OOM, "lvs_client_key_import: host allocation failed");
    ck->P = P;
    ck->lwe_key.assign(lwe_key, lwe_key + lwe_words);
    ck->glwe_key.assign(glwe_key, glwe_key + glwe_words);
    *out = ck;
    return LVS_OK;
}

lvs_status lvs_server_key_params(const lvs_server_key *sk, lvs_params *out)
{
    if (!sk || !out) return set_error(LVS_ERR_ARG, "lvs_server_key_params: NULL argument");
    *out = sk->P.p;
    return LVS_OK;
}

lvs_status lvs_encrypt_string(const lvs_client_key *ck, const uint8_t *s, size_t len,
                              lvs_alphabet alphabet, uint64_t noise_seed, uint64_t string_id,
                              lvs_ct_string **out)
{
    if (!ck || !out || (len && !s)) return set_error(LVS_ERR_ARG, "lvs_encrypt_string: NULL argument");
    if (alphabet_size(alphabet) == 0) return set_error(LVS_ERR_ARG, "lvs_encrypt_string: unknown alphabet");
    const uint32_t sy = symbols_per_char(alphabet), big = ck->P.big();
    std::vector<uint32_t> syms(len * sy);
    for (size_t i = 0; i < len; ++i) {
        uint32_t v[2];
        if (!encode_char(alphabet, s[i], v))
            return set_error(LVS_ERR_ARG, "lvs_encrypt_string: character " + std::to_string(s[i]) +
                                              " at " + std::to_string(i) + " is outside the alphabet");
        for (uint32_t t = 0; t < sy; ++t) syms[i * sy + t] = v[t];
    }
    lvs_ct_string *r = nullptr;
    try {
        r = new lvs_ct_string;
        r->alphabet = alphabet;
        r->symbols = sy;
        r->big = big;
        r->len = len;
        r->data.assign(len * sy * (size_t)(big + 1), 0);
    } catch (const std::bad_alloc &) {
        delete r;
        return set_error(LVS_ERR_OOM, "lvs_encrypt_string: host allocation failed");
    }
    parallel_for(len * sy, [&](size_t idx) {
        const size_t ci = idx / sy, si = idx % sy;
        encrypt_lwe(*ck, syms[idx], noise_seed, string_id, 2 * ci + si, r->data.data() + idx * (big + 1));
    });
    *out = r;
    return LVS_OK;
}

void lvs_ct_string_free(lvs_ct_string *s)
{
    if (!s) return;
    if (s->pinned) {
        cudaFreeHost(s->pinned);
        cudaGetLastError();
    }
    if (s->d) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(s->ddevice);
        cudaFree(s->d);
        cudaSetDevice(cur);
        cudaGetLastError();
    }
    delete s;
}

lvs_status lvs_ct_string_info(const lvs_ct_string *s, size_t *len, uint32_t *symbols, uint32_t *big_dim,
                              lvs_alphabet *alphabet)
{
    if (!s) return set_error(LVS_ERR_ARG, "lvs_ct_string_info: NULL string");
    if (len) *len = s->len;
    if (symbols) *symbols = s->symbols;
    if (big_dim) *big_dim = s->big;
    if (alphabet) *alphabet = s->alphabet;
    return LVS_OK;
}

lvs_status lvs_ct_string_export(const lvs_ct_string *s, uint64_t *dst, size_t *words)
{
    if (!s) return set_error(LVS_ERR_ARG, "lvs_ct_string_export: NULL string");
    return export_vec(s->data, dst, words);
}

lvs_status lvs_ct_string_import(const uint64_t *src, size_t len, lvs_alphabet alphabet, uint32_t big_dim,
                                lvs_ct_string **out)
{
    if (!out || (len && !src)) return set_error(LVS_ERR_ARG, "lvs_ct_string_import: NULL argument");
    if (alphabet_size(alphabet) == 0) return set_error(LVS_ERR_ARG, "lvs_ct_string_import: unknown alphabet");
    if (big_dim != 512 && big_dim != 2048) return set_error(LVS_ERR_ARG, "lvs_ct_string_import: bad dimension");
    lvs_ct_string *r = nullptr;
    try {
        r = new lvs_ct_string;
        r->alphabet = alphabet;
        r->symbols = symbols_per_char(alphabet);
        r->big = big_dim;
        r->len = len;
        r->data.assign(src, src + len * r->symbols * (size_t)(big_dim + 1));
    } catch (const std::bad_alloc &) {
        delete r;
        return set_error(LVS_ERR_OOM, "lvs_ct_string_import: host allocation failed");
    }
    *out = r;
    return LVS_OK;
}

lvs_status lvs_decrypt_lwe(const lvs_client_key *ck, const uint64_t *ct, uint32_t *value)
{
    if (!ck || !ct || !value) return set_error(LVS_ERR_ARG, "lvs_decrypt_lwe: NULL argument");
    *value = decrypt_lwe(*ck, ct);
    return LVS_OK;
}

lvs_status lvs_encrypt_lwe(const lvs_client_key *ck, uint32_t value, uint64_t noise_seed, uint64_t i0,
                           uint64_t i1, uint64_t *ct)
{
    if (!ck || !ct) return set_error(LVS_ERR_ARG, "lvs_encrypt_lwe: NULL argument");
    encrypt_lwe(*ck, value, noise_seed, i0, i1, ct);
    return LVS_OK;
}

}  // extern "C"
