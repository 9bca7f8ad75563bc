/*
 * CPU TFHE oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct restatement of the TFHE primitives the
 * Leuvenshtein method runs on (paper, Section 2.2 "TFHE": LWE ciphertexts with a
 * 5-bit plaintext space of 1 padding bit + 4 message bits, linear operations,
 * and the programmable bootstrap whose lookup table is negacyclic, Table
 * table_lutrelu).  The paper defers the construction of TFHE itself to the
 * original TFHE papers; this file follows that standard construction:
 *   key switch -> modulus switch -> blind rotation (n CMux, each an external
 *   product of a GGSW row set with a GLWE accumulator) -> sample extract.
 *
 * Every polynomial product here is a SCHOOLBOOK negacyclic product computed
 * with wrapping uint64 arithmetic (exact mod 2^64).  There is no NTT, no FFT,
 * no blocking and no fusion: each function is one step of the definition.
 *
 * Conventions that the paper leaves open (see the "readings" list of the
 * design notes):  q = 2^64; Delta = 2^59 (5-bit plaintext);
 *   modulus switch  : round half up, wrap mod 2N;
 *   gadget decomposition: round to the top l*logB bits (half up), then
 *                     balanced digits in [-B/2, B/2) with carry, least
 *                     significant level processed first, final carry dropped;
 *   test polynomial : box = N/16 coefficients per value, rotated by -box/2;
 *   randomness      : SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 *                     counter-based generator; TUniform(b) noise, the uniform
 *                     integer distribution on [-2^b, 2^b] with half weight
 *                     at both ends.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this file.  It shares no code with the product library.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    uint32_t n;              /* LWE dimension after key switching          */
    uint32_t k;              /* GLWE dimension                             */
    uint32_t N;              /* polynomial size                            */
    uint32_t pbs_level;      /* gadget levels of the bootstrapping key     */
    uint32_t pbs_base_log;   /* log2 of the bootstrapping gadget base      */
    uint32_t ks_level;       /* gadget levels of the key-switching key     */
    uint32_t ks_base_log;    /* log2 of the key-switching gadget base      */
    uint32_t lwe_noise_log2; /* TUniform bound of key-switching-key noise  */
    uint32_t glwe_noise_log2;/* TUniform bound of GLWE / fresh noise       */
} orc_params;

/* ------------------------------------------------------------------ */
/* SplitMix64, taken as a counter-based generator.                     */
/* The c-th output (c = 0, 1, ...) of the generator started in state K */
/* is mix(K + (c+1) * GAMMA).                                          */
/* ------------------------------------------------------------------ */
#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t orc_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* first output of SplitMix64 from state x */
uint64_t orc_sm64(uint64_t x) { return orc_mix(x + ORC_GAMMA); }

/* c-th output from state key */
uint64_t orc_word(uint64_t key, uint64_t c) { return orc_mix(key + (c + 1) * ORC_GAMMA); }

/* state of the stream named (seed, tag, i0, i1) */
uint64_t orc_stream(uint64_t seed, uint64_t tag, uint64_t i0, uint64_t i1)
{
    return orc_sm64(orc_sm64(orc_sm64(seed ^ tag) ^ i0) ^ i1);
}

/* TUniform(b) from one random word: r = low (b+2) bits, e = ceil(r/2) - 2^b */
int64_t orc_tuniform(uint64_t w, uint32_t b)
{
    uint64_t r = w & ((1ULL << (b + 2)) - 1ULL);
    return (int64_t)((r + 1) >> 1) - (int64_t)(1ULL << b);
}

enum { ORC_TAG_LWE_KEY = 1, ORC_TAG_GLWE_KEY = 2, ORC_TAG_BSK = 3, ORC_TAG_KSK = 4, ORC_TAG_ENC = 5 };

/* ------------------------------------------------------------------ */
/* Polynomials in Z_{2^64}[X]/(X^N + 1)                                */
/* ------------------------------------------------------------------ */

/* out = a * b, schoolbook: X^i * X^j = X^{i+j} if i+j < N, else -X^{i+j-N} */
void orc_negacyclic_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t N)
{
    for (uint32_t t = 0; t < N; t++) out[t] = 0;
    for (uint32_t i = 0; i < N; i++) {
        for (uint32_t j = 0; j < N - i; j++) out[i + j] += a[i] * b[j];       /* i + j <  N */
        for (uint32_t j = N - i; j < N; j++) out[i + j - N] -= a[i] * b[j];   /* i + j >= N */
    }
}

/* out = X^r * in, r in [0, 2N) */
void orc_poly_rotate(const uint64_t *in, uint32_t r, uint64_t *out, uint32_t N)
{
    for (uint32_t s = 0; s < N; s++) {
        uint32_t d = s + r;
        int neg = 0;
        while (d >= N) { d -= N; neg = !neg; }
        out[d] = neg ? (uint64_t)0 - in[s] : in[s];
    }
}

/* ------------------------------------------------------------------ */
/* Key generation                                                     */
/* Layouts:                                                           */
/*   lwe_key [n]            (0/1)                                     */
/*   glwe_key[k*N]          (0/1), polynomial j at [j*N, (j+1)*N);     */
/*                          also the "big" LWE key of dimension kN    */
/*   bsk [n][(k+1)*l][(k+1)][N]: GGSW(s_i); row r = j*l + (lev-1)      */
/*        encrypts s_i * q / B^lev added to component j               */
/*   ksk [k*N][ks_l][n+1]: LWE_s(S'_u * q / Bks^lev), body at index n */
/* ------------------------------------------------------------------ */

static void glwe_encrypt_row(const orc_params *P, const uint64_t *glwe_key, uint64_t key,
                             uint64_t *row /* (k+1)*N */, uint64_t *tmp /* N */)
{
    uint32_t N = P->N, k = P->k;
    uint64_t *body = row + (size_t)k * N;
    for (uint32_t j = 0; j < k; j++)
        for (uint32_t t = 0; t < N; t++)
            row[(size_t)j * N + t] = orc_word(key, (uint64_t)j * N + t);
    for (uint32_t t = 0; t < N; t++)
        body[t] = (uint64_t)orc_tuniform(orc_word(key, (uint64_t)k * N + t), P->glwe_noise_log2);
    for (uint32_t j = 0; j < k; j++) {
        orc_negacyclic_mul(row + (size_t)j * N, glwe_key + (size_t)j * N, tmp, N);
        for (uint32_t t = 0; t < N; t++) body[t] += tmp[t];
    }
}

void orc_keygen(const orc_params *P, uint64_t seed, uint64_t *lwe_key, uint64_t *glwe_key,
                uint64_t *bsk, uint64_t *ksk)
{
    uint32_t n = P->n, k = P->k, N = P->N, l = P->pbs_level, lb = P->pbs_base_log;
    uint32_t ksl = P->ks_level, kslb = P->ks_base_log;
    uint64_t kl = orc_stream(seed, ORC_TAG_LWE_KEY, 0, 0);
    for (uint32_t i = 0; i < n; i++) lwe_key[i] = orc_word(kl, i) >> 63;
    uint64_t kg = orc_stream(seed, ORC_TAG_GLWE_KEY, 0, 0);
    for (uint32_t u = 0; u < k * N; u++) glwe_key[u] = orc_word(kg, u) >> 63;

    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * N);
    size_t row_words = (size_t)(k + 1) * N;
    for (uint32_t i = 0; i < n; i++) {
        for (uint32_t j = 0; j <= k; j++) {
            for (uint32_t lev = 1; lev <= l; lev++) {
                uint32_t r = j * l + (lev - 1);
                uint64_t *row = bsk + ((size_t)i * (k + 1) * l + r) * row_words;
                glwe_encrypt_row(P, glwe_key, orc_stream(seed, ORC_TAG_BSK, i, r), row, tmp);
                /* message s_i * q / B^lev on the constant coefficient of component j */
                uint64_t g = 1ULL << (64 - lev * lb);
                row[(size_t)j * N] += lwe_key[i] * g;
            }
        }
    }
    free(tmp);

    for (uint32_t u = 0; u < k * N; u++) {
        for (uint32_t lev = 1; lev <= ksl; lev++) {
            uint64_t key = orc_stream(seed, ORC_TAG_KSK, u, lev - 1);
            uint64_t *row = ksk + ((size_t)u * ksl + (lev - 1)) * (n + 1);
            uint64_t b = 0;
            for (uint32_t c = 0; c < n; c++) {
                row[c] = orc_word(key, c);
                b += row[c] * lwe_key[c];
            }
            b += (uint64_t)orc_tuniform(orc_word(key, n), P->lwe_noise_log2);
            b += glwe_key[u] * (1ULL << (64 - lev * kslb));
            row[n] = b;
        }
    }
}

/* ------------------------------------------------------------------ */
/* LWE encryption / decryption under a key of dimension dim           */
/* ------------------------------------------------------------------ */

/* ct = (a, <a,s> + mu + e), a uniform, e ~ TUniform(noise_log2);
   the stream is (noise_seed, ENC, i0, i1); words 0..dim-1 mask, word dim noise */
void orc_lwe_encrypt(const uint64_t *key, uint32_t dim, uint64_t mu, uint32_t noise_log2,
                     uint64_t noise_seed, uint64_t i0, uint64_t i1, uint64_t *ct)
{
    uint64_t st = orc_stream(noise_seed, ORC_TAG_ENC, i0, i1);
    uint64_t b = 0;
    for (uint32_t c = 0; c < dim; c++) {
        ct[c] = orc_word(st, c);
        b += ct[c] * key[c];
    }
    b += (uint64_t)orc_tuniform(orc_word(st, dim), noise_log2);
    ct[dim] = b + mu;
}

uint64_t orc_lwe_phase(const uint64_t *key, uint32_t dim, const uint64_t *ct)
{
    uint64_t s = 0;
    for (uint32_t c = 0; c < dim; c++) s += ct[c] * key[c];
    return ct[dim] - s;
}

/* decode a 5-bit plaintext: round(phase / 2^59) mod 32 */
uint32_t orc_lwe_decrypt(const uint64_t *key, uint32_t dim, const uint64_t *ct)
{
    uint64_t ph = orc_lwe_phase(key, dim, ct);
    return (uint32_t)(((ph + (1ULL << 58)) >> 59) & 31ULL);
}

/* ------------------------------------------------------------------ */
/* Gadget decomposition of one torus value into l balanced digits.    */
/* digit[lev-1] multiplies q / B^lev.                                  */
/* ------------------------------------------------------------------ */
void orc_decompose(uint64_t a, uint32_t l, uint32_t logB, int64_t *digit)
{
    uint32_t beta = l * logB;
    uint64_t v = (a + (1ULL << (63 - beta))) >> (64 - beta);
    uint64_t B = 1ULL << logB;
    uint64_t carry = 0;
    for (int lev = (int)l; lev >= 1; lev--) {
        uint64_t u = (v >> ((l - lev) * logB)) & (B - 1);
        uint64_t r = u + carry;
        if (r >= B / 2) { digit[lev - 1] = (int64_t)r - (int64_t)B; carry = 1; }
        else            { digit[lev - 1] = (int64_t)r;               carry = 0; }
    }
}

/* ------------------------------------------------------------------ */
/* Key switch: LWE under the big key (dim kN) -> LWE under s (dim n)  */
/* out = (0, b) - sum_{u, lev} d_{u,lev} * KSK[u][lev]                 */
/* ------------------------------------------------------------------ */
void orc_keyswitch(const orc_params *P, const uint64_t *ksk, const uint64_t *in, uint64_t *out)
{
    uint32_t n = P->n, kN = P->k * P->N, l = P->ks_level;
    int64_t d[64];
    for (uint32_t c = 0; c < n; c++) out[c] = 0;
    out[n] = in[kN];
    for (uint32_t u = 0; u < kN; u++) {
        orc_decompose(in[u], l, P->ks_base_log, d);
        for (uint32_t lev = 1; lev <= l; lev++) {
            const uint64_t *row = ksk + ((size_t)u * l + (lev - 1)) * (n + 1);
            for (uint32_t c = 0; c <= n; c++) out[c] -= (uint64_t)d[lev - 1] * row[c];
        }
    }
}

/* modulus switch to 2N: round(x * 2N / 2^64) mod 2N */
void orc_modswitch(const orc_params *P, const uint64_t *in, uint32_t *out)
{
    uint32_t log2N = 0;
    while ((1u << log2N) < 2 * P->N) log2N++;
    for (uint32_t c = 0; c <= P->n; c++)
        out[c] = (uint32_t)(((in[c] + (1ULL << (63 - log2N))) >> (64 - log2N)) & (2ULL * P->N - 1));
}

/* ------------------------------------------------------------------ */
/* Test polynomial of a 16-entry LUT f (values in Z_32):              */
/* v[t] = f[t / box] * Delta, box = N/16, then v <- X^{-box/2} * v     */
/* ------------------------------------------------------------------ */
void orc_lut_poly(const orc_params *P, const uint32_t *f16, uint64_t *v)
{
    uint32_t N = P->N, box = N / 16;
    uint64_t *raw = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (uint32_t t = 0; t < N; t++) raw[t] = (uint64_t)(f16[t / box] & 31u) << 59;
    orc_poly_rotate(raw, 2 * N - box / 2, v, N);
    free(raw);
}

/* ------------------------------------------------------------------ */
/* External product GGSW(s_i) [x] GLWE and the CMux                   */
/* ------------------------------------------------------------------ */
static void external_product(const orc_params *P, const uint64_t *ggsw, const uint64_t *c,
                             uint64_t *out, uint64_t *dig, uint64_t *tmp)
{
    uint32_t k = P->k, N = P->N, l = P->pbs_level, lb = P->pbs_base_log;
    size_t row_words = (size_t)(k + 1) * N;
    int64_t d[16];
    memset(out, 0, sizeof(uint64_t) * row_words);
    for (uint32_t j = 0; j <= k; j++) {
        /* digit polynomials of component j: dig[(lev-1)*N + t] */
        for (uint32_t t = 0; t < N; t++) {
            orc_decompose(c[(size_t)j * N + t], l, lb, d);
            for (uint32_t lev = 1; lev <= l; lev++) dig[(size_t)(lev - 1) * N + t] = (uint64_t)d[lev - 1];
        }
        for (uint32_t lev = 1; lev <= l; lev++) {
            const uint64_t *row = ggsw + (size_t)(j * l + (lev - 1)) * row_words;
            for (uint32_t comp = 0; comp <= k; comp++) {
                orc_negacyclic_mul(dig + (size_t)(lev - 1) * N, row + (size_t)comp * N, tmp, N);
                for (uint32_t t = 0; t < N; t++) out[(size_t)comp * N + t] += tmp[t];
            }
        }
    }
}

/* ACC <- X^{-b} v, then for each i: ACC <- ACC + GGSW_i [x] (X^{a_i} ACC - ACC) */
void orc_blind_rotate(const orc_params *P, const uint64_t *bsk, const uint32_t *ms,
                      const uint64_t *v, uint64_t *acc)
{
    uint32_t n = P->n, k = P->k, N = P->N, l = P->pbs_level;
    size_t row_words = (size_t)(k + 1) * N;
    size_t ggsw_words = (size_t)(k + 1) * l * row_words;
    uint64_t *rot = (uint64_t *)malloc(sizeof(uint64_t) * row_words);
    uint64_t *ep = (uint64_t *)malloc(sizeof(uint64_t) * row_words);
    uint64_t *dig = (uint64_t *)malloc(sizeof(uint64_t) * l * N);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * N);

    memset(acc, 0, sizeof(uint64_t) * row_words);
    orc_poly_rotate(v, (2 * N - ms[n]) % (2 * N), acc + (size_t)k * N, N);
    for (uint32_t i = 0; i < n; i++) {
        for (uint32_t j = 0; j <= k; j++) {
            orc_poly_rotate(acc + (size_t)j * N, ms[i], rot + (size_t)j * N, N);
            for (uint32_t t = 0; t < N; t++) rot[(size_t)j * N + t] -= acc[(size_t)j * N + t];
        }
        external_product(P, bsk + (size_t)i * ggsw_words, rot, ep, dig, tmp);
        for (size_t t = 0; t < row_words; t++) acc[t] += ep[t];
    }
    free(rot); free(ep); free(dig); free(tmp);
}

/* LWE (dim kN) holding coefficient 0 of the GLWE phase */
void orc_sample_extract(const orc_params *P, const uint64_t *acc, uint64_t *out)
{
    uint32_t k = P->k, N = P->N;
    for (uint32_t j = 0; j < k; j++) {
        const uint64_t *A = acc + (size_t)j * N;
        out[(size_t)j * N] = A[0];
        for (uint32_t u = 1; u < N; u++) out[(size_t)j * N + u] = (uint64_t)0 - A[N - u];
    }
    out[(size_t)k * N] = acc[(size_t)k * N];
}

/* PBS = KS -> MS -> BR -> SE with the 16-entry LUT f */
void orc_pbs(const orc_params *P, const uint64_t *ksk, const uint64_t *bsk,
             const uint64_t *in, const uint32_t *f16, uint64_t *out)
{
    uint32_t n = P->n, k = P->k, N = P->N;
    uint64_t *small = (uint64_t *)malloc(sizeof(uint64_t) * (n + 1));
    uint32_t *ms = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
    uint64_t *v = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint64_t *acc = (uint64_t *)malloc(sizeof(uint64_t) * (k + 1) * N);
    orc_keyswitch(P, ksk, in, small);
    orc_modswitch(P, small, ms);
    orc_lut_poly(P, f16, v);
    orc_blind_rotate(P, bsk, ms, v, acc);
    orc_sample_extract(P, acc, out);
    free(small); free(ms); free(v); free(acc);
}

/* ------------------------------------------------------------------ */
/* Independent PBS spread over host threads (used to time the oracle) */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_params *P; const uint64_t *ksk, *bsk, *in; const uint32_t *f16; uint64_t *out;
    size_t count, first, stride;
} pbs_job;

static void *pbs_worker(void *arg)
{
    pbs_job *J = (pbs_job *)arg;
    size_t big = (size_t)J->P->k * J->P->N + 1;
    for (size_t i = J->first; i < J->count; i += J->stride)
        orc_pbs(J->P, J->ksk, J->bsk, J->in + i * big, J->f16 + i * 16, J->out + i * big);
    return NULL;
}

int orc_pbs_many(const orc_params *P, const uint64_t *ksk, const uint64_t *bsk, size_t count,
                 const uint64_t *in, const uint32_t *f16, uint64_t *out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
    int *live = (int *)malloc(sizeof(int) * nthreads);
    pbs_job *jobs = (pbs_job *)malloc(sizeof(pbs_job) * nthreads);
    int started = 0;
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = (pbs_job){P, ksk, bsk, in, f16, out, count, (size_t)t, (size_t)nthreads};
        live[t] = pthread_create(&th[t], NULL, pbs_worker, &jobs[t]) == 0;
        if (live[t]) started++;
        else pbs_worker(&jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) if (live[t]) pthread_join(th[t], NULL);
    free(th); free(live); free(jobs);
    return started;
}
