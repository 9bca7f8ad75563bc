/*
 * lvs.h -- C ABI of the GB300 Leuvenshtein library (encrypted edit distance
 * with one programmable bootstrap per cell).
 *
 * Method: "Leuvenshtein: Efficient FHE-based Edit Distance Computation with
 * Single Bootstrap per Cell" (Legiest, D'Anvers, Spasic, Tran, Verbauwhede,
 * arXiv 2508.14568).  Section references below are to that paper.
 *
 * Problem statement followed by the calls (Section 1, Section 5, Section 6):
 * a client encrypts its strings, a server computes edit distances on the
 * ciphertexts with its server key, and the client decrypts the result.
 *
 * General conventions
 *   - Every call returns lvs_status.  Out-pointers are written only on LVS_OK.
 *     lvs_last_error() returns a thread-local message for the last failure.
 *   - Handles returned through out-pointers are owned by the caller and
 *     released with the matching lvs_*_free (NULL is accepted and ignored).
 *     Input handles are borrowed for the duration of the call.
 *   - Host pointers are plain CPU memory; "device" pointers are CUDA global
 *     memory of the context's device.  All integers are little-endian.
 *   - Ciphertexts: an LWE ciphertext of dimension d is d+1 uint64 words
 *     (mask a[0..d-1], body b), torus Z_{2^64}, plaintext Z_32 encoded as
 *     value * 2^59 (Section 2.2: 4 message bits + 1 padding bit).  "Big"
 *     ciphertexts have d = k*N (the GLWE key seen as an LWE key); all
 *     transmitted and stored ciphertexts are big.
 *   - Batch calls are asynchronous on the context's CUDA stream; calls that
 *     return host data (lvs_decrypt, lvs_result_export) synchronise it.
 *   - String lengths are not hidden (the paper's loops run over m and n).
 *   - There is no CPU fallback: compute calls fail with LVS_ERR_CUDA when no
 *     usable GPU is present.
 */
#ifndef LVS_H
#define LVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LVS_OK = 0,
    LVS_ERR_ARG = 1,          /* invalid argument (NULL, size, alphabet, symbol) */
    LVS_ERR_OOM = 2,          /* host or device allocation failed                */
    LVS_ERR_CUDA = 3,         /* CUDA runtime error (message in lvs_last_error)  */
    LVS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up              */
    LVS_ERR_NOISE_BUDGET = 5, /* predicted key noise exceeds the parameter budget */
    LVS_ERR_STATE = 6         /* not ready / wrong state (e.g. poll before done) */
} lvs_status;

/* Symbol alphabets.  ASCII7: 7-bit characters split into a 4-bit and a 3-bit
 * symbol, 2 ciphertexts per character, 2-PBS equality (Section 4.3, Algorithm
 * alg_ascii).  27: 'A'..'Z' -> 0..25, ' ' -> 26, same 4+1-bit split and 2-PBS
 * equality.  DNA4: A,C,G,T -> 0..3, one ciphertext per character, 1-PBS
 * equality (Section 4.1, used for DNA in Section 6.3). */
typedef enum { LVS_ALPHA_ASCII7 = 0, LVS_ALPHA_27 = 1, LVS_ALPHA_DNA4 = 2 } lvs_alphabet;

/* TFHE parameters (Section 2.2 and Section 6.2 name only the family "4-bit
 * message, 0-bit carry" with a padding bit; numeric values are chosen by this
 * library).  Supported: k = 1, N in {512, 2048}, pbs_level = 2 with
 * pbs_level * pbs_base_log <= 26, ks_level <= 8 with ks_level * ks_base_log
 * <= 30, 1 <= n <= 4096; LVS_ERR_ARG otherwise. */
typedef struct lvs_params {
    uint32_t n;               /* LWE dimension after key switching           */
    uint32_t k;               /* GLWE dimension (1)                          */
    uint32_t N;               /* polynomial size                             */
    uint32_t pbs_level;       /* bootstrapping-key gadget levels             */
    uint32_t pbs_base_log;    /* log2 of the bootstrapping gadget base       */
    uint32_t ks_level;        /* key-switching-key gadget levels             */
    uint32_t ks_base_log;     /* log2 of the key-switching gadget base       */
    uint32_t lwe_noise_log2;  /* TUniform bound (log2) of key-switching noise */
    uint32_t glwe_noise_log2; /* TUniform bound (log2) of GLWE/fresh noise   */
} lvs_params;

/* Default set for the paper's workloads: n=834, k=1, N=2048, pbs 2 x 2^13,
 * ks 5 x 2^3, noise bounds 2^45 / 2^17. */
void lvs_params_default(lvs_params *out);
/* Small INSECURE set (n=64, N=512, same gadgets) for fast parity tests. */
void lvs_params_test(lvs_params *out);

typedef struct lvs_client_key lvs_client_key; /* secret keys, host only          */
typedef struct lvs_server_key lvs_server_key; /* BSK + KSK, host copy            */
typedef struct lvs_ctx lvs_ctx;               /* device, stream, device keys     */
typedef struct lvs_ct_string lvs_ct_string;   /* encrypted string (host memory)  */
typedef struct lvs_result lvs_result;         /* encrypted distances of a batch  */
typedef struct lvs_eq_table lvs_eq_table;     /* preprocessed EQ9 table (device) */
typedef struct lvs_server lvs_server;         /* continuous-batching server      */

const char *lvs_last_error(void);
const char *lvs_version(void);

/* ---------------------------------------------------------------- keys */

/* Key generation from a 64-bit seed (deterministic: the same seed gives the
 * same keys on every machine).  Client key: binary LWE key s (n) and binary
 * GLWE key S (k*N).  Server key: bootstrapping key BSK_i = GGSW_S(s_i) and
 * key-switching key KSK (big key -> s).  Randomness: SplitMix64 streams,
 * TUniform noise.  Runs on host threads. */
lvs_status lvs_keygen(const lvs_params *params, uint64_t seed,
                      lvs_client_key **client, lvs_server_key **server);
void lvs_client_key_free(lvs_client_key *ck);
void lvs_server_key_free(lvs_server_key *sk);

/* Raw key material, for serialisation and tests.  Sizes in uint64 words:
 * lwe_key n, glwe_key k*N, bsk n*(k+1)*pbs_level*(k+1)*N laid out
 * [i][row = j*pbs_level + lev-1][component][coefficient], ksk
 * k*N*ks_level*(n+1) laid out [u][lev-1][n+1].  dst must hold the size;
 * pass dst = NULL to query it in *words. */
lvs_status lvs_client_key_export(const lvs_client_key *ck, uint64_t *lwe_key, size_t *lwe_words,
                                 uint64_t *glwe_key, size_t *glwe_words);
lvs_status lvs_server_key_export(const lvs_server_key *sk, uint64_t *bsk, size_t *bsk_words,
                                 uint64_t *ksk, size_t *ksk_words);
lvs_status lvs_server_key_params(const lvs_server_key *sk, lvs_params *out);
/* Rebuild keys from exported material (the layouts above) for the parameter
 * set params: how a server loads the evaluation keys a client sent it
 * (Section 1's client / server setting), and how a client reloads its secret
 * key.  The words are copied.  LVS_ERR_ARG for a NULL pointer, invalid
 * params, word counts that do not match params, or (client key) a key
 * coefficient other than 0 or 1. */
lvs_status lvs_server_key_import(const lvs_params *params, const uint64_t *bsk, size_t bsk_words,
                                 const uint64_t *ksk, size_t ksk_words, lvs_server_key **out);
lvs_status lvs_client_key_import(const lvs_params *params, const uint64_t *lwe_key, size_t lwe_words,
                                 const uint64_t *glwe_key, size_t glwe_words, lvs_client_key **out);

/* ---------------------------------------------------------------- context */

/* Creates a device context: uploads the server key to GPU `device`, converts
 * the bootstrapping key to the NTT domain (three 30-bit primes, in the
 * register order of the blind-rotation kernel) and sets up tables.  `stream`
 * is a cudaStream_t to run on (NULL = a new non-blocking stream owned by the
 * context).  Device memory: about 1.5x the BSK plus the KSK.
 * Threads: a context may be shared by host threads.  Every call that uses its
 * stream, scratch memory, launch settings, counters or timing state takes the
 * context's lock for the whole call, so such calls (batch calls, the
 * device-pointer calls below, the tuning setters and getters, timing,
 * lvs_ctx_synchronize) run one at a time in the order the lock is taken. */
lvs_status lvs_ctx_create(const lvs_server_key *sk, int device, void *stream, lvs_ctx **out);
void lvs_ctx_free(lvs_ctx *ctx);
/* Waits for the context's stream.  LVS_ERR_TIMEOUT if a bounded device-side
 * wait of a kernel on this device gave up since the last check (the results of
 * that work are void; reported once, the context stays usable); lvs_decrypt,
 * lvs_decrypt_all, lvs_result_export and the server's steps report it too. */
lvs_status lvs_ctx_synchronize(lvs_ctx *ctx);

/* ---------------------------------------------------------------- client */

/* Encrypts s[0..len) (Section 4.3 split for ASCII7 / 27 symbols; one symbol
 * for DNA4).  Each symbol is one fresh big LWE ciphertext whose randomness is
 * the SplitMix64 stream (noise_seed, ENC, string_id, 2*char + symbol).
 * Fails with LVS_ERR_ARG on a character outside the alphabet.  len may be 0. */
lvs_status lvs_encrypt_string(const lvs_client_key *ck, const uint8_t *s, size_t len,
                              lvs_alphabet alphabet, uint64_t noise_seed, uint64_t string_id,
                              lvs_ct_string **out);
void lvs_ct_string_free(lvs_ct_string *s);
/* Number of characters / symbols per character / big dimension k*N. */
lvs_status lvs_ct_string_info(const lvs_ct_string *s, size_t *len, uint32_t *symbols,
                              uint32_t *big_dim, lvs_alphabet *alphabet);
/* Ciphertexts laid out [char][symbol][k*N+1] (host). dst = NULL: size query. */
lvs_status lvs_ct_string_export(const lvs_ct_string *s, uint64_t *dst, size_t *words);
/* Wraps host ciphertexts (copied) as an encrypted string. */
lvs_status lvs_ct_string_import(const uint64_t *src, size_t len, lvs_alphabet alphabet,
                                uint32_t big_dim, lvs_ct_string **out);

/* Copies the ciphertexts of s to device memory of the context's GPU and keeps
 * them with the string (released by lvs_ct_string_free); batch calls then read
 * the device copy instead of uploading.  Synchronous.  Calling it again is a
 * no-op. */
lvs_status lvs_ct_string_upload(lvs_ctx *ctx, lvs_ct_string *s);
/* Keeps a page-locked (pinned) host copy of the ciphertexts, freed with the
 * string; later host-to-device copies of the string (batch calls on host
 * strings, lvs_ct_string_upload) read it, so they run as asynchronous DMA.
 * Calling it again is a no-op. */
lvs_status lvs_ct_string_pin(lvs_ct_string *s);

/* Decrypts one big LWE ciphertext to its Z_32 plaintext (round(phase/2^59)). */
lvs_status lvs_decrypt_lwe(const lvs_client_key *ck, const uint64_t *ct, uint32_t *value);
/* Encrypts one Z_32 value as a big LWE ciphertext with the stream
 * (noise_seed, ENC, i0, i1). */
lvs_status lvs_encrypt_lwe(const lvs_client_key *ck, uint32_t value, uint64_t noise_seed,
                           uint64_t i0, uint64_t i1, uint64_t *ct);

/* ---------------------------------------------------------------- server */

/* Edit-distance options.  band < 0: exact full matrix (the configurations of
 * this library compute every cell). */
typedef struct lvs_opts {
    int32_t band;          /* < 0: full matrix.  >= 0: only the cells with      *
                            * |i - j| <= band for m = n (Algorithm               *
                            * alg_levenshtein; band = floor(m/2) is exact,       *
                            * "Exact Skip", Section 3.2); for m != n the         *
                            * diagonals k = j - i with min(0, n-m) - band <= k   *
                            * <= max(0, n-m) + band, where every edit path of    *
                            * cost <= |n-m| + 2 band lies (exact for band >=     *
                            * ceil(min(m,n)/2)).  Narrower bands give the        *
                            * approximate distance of Section 3.2 (never below   *
                            * the true distance)                                 */
    int32_t use_graph;     /* 1: capture the wavefront launches in a CUDA graph  */
    int32_t refresh_budget;/* noise budget of a key, in units of the variance   *
                            * of a fresh PBS output (Section 3.1.3; the paper's  *
                            * example parameter set allows 25).  0: from the     *
                            * parameter set for a failure probability of 2^-64   *
                            * per PBS (lvs_noise_budget); > 0: this budget;      *
                            * < 0: never refresh.  Anti-diagonals chosen by      *
                            * lvs_noise_plan are refreshed: their cells take two *
                            * PBS (dv and dh as fresh bootstrap outputs) instead *
                            * of one.  LVS_ERR_NOISE_BUDGET if no plan fits.     */
    int32_t reserved[5];
} lvs_opts;
void lvs_opts_default(lvs_opts *o);

/* Noise budget (Section 3.1.3): the largest variance of a key, in units of
 * the variance of a fresh PBS output, for which one bootstrap of it (with
 * the key-switch and modulus-switch noise of the parameter set, binary keys
 * of expected weight) decodes wrongly with probability at most 2^log2_pfail
 * (log2_pfail < 0).  Host only. */
lvs_status lvs_noise_budget(const lvs_params *p, double log2_pfail, double *budget);
/* log2 of the failure probability of one bootstrap whose key carries key_var
 * PBS-output variances (plus the key-switch and modulus-switch noise): the
 * normal tail beyond half a plaintext step.  Host only. */
lvs_status lvs_noise_pfail(const lvs_params *p, double key_var, double *log2_pfail);
/* Refresh plan of one m x n difference matrix (band < 0: full; else the
 * cells of lvs_opts.band).  Each M and EQ9 is a unit noise, dv_out = M - dh_in,
 * dh_out = M - dv_in; a cell costs the larger variance of its key and of its
 * key with dv_in, dh_in exchanged.  An anti-diagonal d = i + j is refreshed
 * when, without it, a cell of d + 1 would cost more than budget (budget <= 0:
 * no refresh).  refresh (may be NULL): m + n + 1 bytes, refresh[d] = 1 for
 * the refreshed anti-diagonals; max_key_var (may be NULL): the largest cost.
 * LVS_ERR_NOISE_BUDGET if a cell exceeds the budget even so.  Host only. */
lvs_status lvs_noise_plan(size_t m, size_t n, int32_t band, double budget, uint8_t *refresh,
                          double *max_key_var);

/* The wavefront plan of one pair, exactly as the distance calls build it,
 * exported for inspection (host only, no GPU).  Rows are indices into the
 * pair's working rows, laid out as
 *   encrypted reference (eq_lookups = 1 or 2): [a: m*C][b: n*C][v: m][h: n]
 *       [band path: m + n][EQ1 ring: 2m, C = 2 only][EQ9 ring: 2m]
 *   plaintext reference (eq_lookups = 0): [table: nsub*m][v: m][h: n]
 *       [band path: m + n]
 * with C = eq_lookups symbols per character (row a + (i-1)*C + symbol), table
 * row T[k][i] at k*m + i - 1 (k the position of the symbol in subset), v[i] at
 * v + i - 1, h[j] at h + j - 1, and ring slot (d & 1) * m + i - 1 for
 * anti-diagonal d = i + j - 2.  Launch step s holds, for C = 2, the EQ1
 * lookups of anti-diagonal s, the EQ9 lookups of s - 1 and the cells of
 * s - 2; for C = 1 the EQ9 lookups of s and the cells of s - 1; for the
 * plaintext reference the cells of s (Section 6.2's parallelism over the
 * cells of an anti-diagonal).
 * Arguments: band as lvs_opts.band; refresh NULL or m + n + 1 bytes as from
 * lvs_noise_plan; plain / subset (nsub symbols, distinct, covering plain) for
 * the plaintext reference, else NULL.  layout (may be NULL) receives the first
 * row of each block (-1 if absent) and the total.  jobs (may be NULL): room
 * for *count entries; on return *count is the number of jobs (LVS_ERR_ARG if
 * the room was too small, nothing written). */
typedef struct lvs_plan_layout {
    int64_t a, b, v, h, path, eq1, eq9, table, rows, steps;
} lvs_plan_layout;
typedef struct lvs_plan_job {
    int64_t step;
    int64_t src[3];      /* input rows, -1 if unused                         */
    int64_t coef[3];     /* input = sum coef * src + cst (times Delta)       */
    int64_t cst;
    int64_t dst[2];      /* rows written: the lookup (store), or v and h (cell) */
    int64_t tap;         /* band path row receiving a copy, -1 if none       */
    int32_t lut;         /* 0 EQ, 1 EQ9, 2 MIN, 3 V                          */
    int32_t kind;        /* 0 store, 1 cell: v = M - h_old, h = M - v_old    */
    int32_t tapsel;      /* store: 1 copies the output; cell: 1 new v, 2 new h */
    int32_t pad;
} lvs_plan_job;
lvs_status lvs_plan_pair(size_t m, size_t n, uint32_t eq_lookups, int32_t band, const uint8_t *refresh,
                         const uint8_t *plain, const uint8_t *subset, size_t nsub, lvs_plan_layout *layout,
                         lvs_plan_job *jobs, size_t *count);
/* The plan of the Section 5 table build of one encrypted string of m
 * characters of `alphabet` against the nsub plaintext symbols of subset, as
 * lvs_preprocess and the server build it (host only, no GPU).  Rows: [a: m*C]
 * [EQ1 scratch: nsub*m, C = 2 only][table: nsub*m], T[k][i] at
 * table + k*m + i - 1; layout.eq1 and layout.table give the blocks (v, h,
 * path, eq9 and b are -1).  Jobs, count and errors as lvs_plan_pair; a subset
 * symbol outside the alphabet or repeated gives LVS_ERR_ARG. */
lvs_status lvs_plan_table(size_t m, lvs_alphabet alphabet, const uint8_t *subset, size_t nsub,
                          lvs_plan_layout *layout, lvs_plan_job *jobs, size_t *count);
/* The launch schedule of a batch (host only, no GPU; the paper runs pairs one
 * per thread, Section 6.2 "Parallelism": here the steps of many pairs share
 * launches).  Pair p has the steps of lvs_plan_pair(m[p], n[p], eq_lookups,
 * band); launch_of receives, pair after pair, the launch of each of its steps
 * (count = total steps; launch_of NULL: size query), nlaunch the number of
 * launches.  wave = 0: all pairs step together, launch s holding step s of
 * every pair.  wave > 0: what batch calls do with wave = the blind-rotation
 * grid (lvs_ctx_set_wave_fill): when a launch's PBS exceed a multiple of wave
 * by r, pairs whose remaining steps are fewer than the longest pair's are
 * held back one launch (smallest step first) until r PBS are held, so the
 * launch ends on a full wave.  Either way a pair's steps are in increasing
 * launches, and nlaunch is the longest pair's step count.  LVS_ERR_ARG for
 * eq_lookups outside 1..2 or too little room. */
lvs_status lvs_plan_batch(const size_t *m, const size_t *n, size_t npairs, uint32_t eq_lookups, int32_t band,
                          size_t wave, int64_t *launch_of, size_t *count, size_t *nlaunch);

/* Encrypted equality of characters a[i] and b[j] (Algorithm alg_ascii: 2 PBS
 * for ASCII7 / 27 symbols; Section 4.1: 1 PBS for DNA4).  times9 != 0 gives
 * enc(9*EQ) (Eq. eq_eqlut9), else enc(EQ).  The result holds one ciphertext. */
lvs_status lvs_eq(lvs_ctx *ctx, const lvs_ct_string *a, size_t i, const lvs_ct_string *b,
                  size_t j, int times9, lvs_result **out);

/* Leuvenshtein edit distances of npairs encrypted pairs (a[p], b[p])
 * (Algorithm algo_complete: per cell 2 equality PBS + 1 cell PBS with the key
 * of Eq. eq_keyeq2; DNA4: 1 + 1).  All pairs advance together: launch s
 * bootstraps the union over pairs of {cell PBS of anti-diagonal s-2, EQ9 of
 * s-1, EQ1 of s} (Section 6.2 "Parallelism": cells of one anti-diagonal are
 * independent).  The result holds, per pair, the encrypted last row
 * h[m][1..n] and the plaintext m; the distance is m + sum_j dec(h[m][j]).
 * With a band (opts->band >= 0) the result holds instead the m + n
 * differences along a monotone path from (0, 0) to (m, n): [v[1][0], h[1][1],
 * ..., v[r][r-1], h[r][r]] (r = min(m, n), the diagonal readout of Section
 * 3.2), then h[m][m+1..n] or v[r+1..m][n]; the distance is their decrypted
 * sum.
 * Both strings of a pair must share the alphabet; lengths may be 0. */
lvs_status lvs_edit_distance_batch(lvs_ctx *ctx, const lvs_ct_string *const *a,
                                   const lvs_ct_string *const *b, size_t npairs,
                                   const lvs_opts *opts, lvs_result **out);

/* Preprocessing of Section 5: for the encrypted string `enc`, the table
 * T[sigma][i] = enc(9 * EQ(a_i, sigma)) for every symbol sigma of `subset`
 * (nsub plaintext characters of the string's alphabet; NULL = whole alphabet:
 * 128 / 27 / 4 symbols).  Cost: nsub * len * (2 or 1) PBS.  Device memory. */
lvs_status lvs_preprocess(lvs_ctx *ctx, const lvs_ct_string *enc, const uint8_t *subset,
                          size_t nsub, lvs_eq_table **out);
/* The tables of count encrypted strings at once (same subset for all): every
 * lookup of every string in the same launches (2 launch steps; 1 for DNA), the
 * offline phase of Section 5 at scale (an encrypted database of strings to be
 * queried with plaintext strings).  outs[k] receives the table of encs[k];
 * on error nothing is returned. */
lvs_status lvs_preprocess_batch(lvs_ctx *ctx, const lvs_ct_string *const *encs, size_t count,
                                const uint8_t *subset, size_t nsub, lvs_eq_table **outs);
void lvs_eq_table_free(lvs_eq_table *t);

/* Online phase of Section 5: distance of each preprocessed encrypted string
 * t[q] to the plaintext string plain[q] (plain_len[q] characters, all in the
 * table's subset).  EQ9[i][j] = T[b_j][i] is a device gather (0 PBS); one
 * cell PBS per cell.  opts as for lvs_edit_distance_batch (band: the result
 * holds the readout path). */
lvs_status lvs_edit_distance_preprocessed_batch(lvs_ctx *ctx, const lvs_eq_table *const *t,
                                                const uint8_t *const *plain,
                                                const size_t *plain_len, size_t n,
                                                const lvs_opts *opts, lvs_result **out);

/* Number of items in a result, and for item `pair`: m and n. */
lvs_status lvs_result_info(const lvs_result *r, size_t *items, size_t pair, size_t *m, size_t *n);
/* Copies the ciphertexts of item `pair` (n big LWE ciphertexts; m + n with a
 * band; 1 for lvs_eq and lvs_result_sum) to host memory dst ([rows][k*N+1]).
 * dst = NULL: size query in *words. */
lvs_status lvs_result_export(const lvs_result *r, size_t pair, uint64_t *dst, size_t *words);
void lvs_result_free(lvs_result *r);

/* Server-side readout (the return of Algorithm algo_complete on ciphertexts):
 * a new result with one big LWE ciphertext per item of r, the sum of the
 * item's rows plus the trivial encryption of its offset (m with the last row
 * h[m][1..n], 0 with a band path), i.e. an encryption of the distance.  No
 * bootstrap: the noise variance is at most that of m + n bootstrap outputs.
 * The sum decodes to the distance with its padding bit clear only below 16, so
 * every item must have max(m, n) <= 15; longer items, an lvs_eq result or a
 * result of another context give LVS_ERR_ARG.  Asynchronous on ctx's stream,
 * ordered after r; r may be freed afterwards.  Decrypt with lvs_decrypt. */
lvs_status lvs_result_sum(lvs_ctx *ctx, const lvs_result *r, lvs_result **out);

/* Client side: decrypts item `pair` to the edit distance m + sum_j h[m][j]
 * (each h decoded to {-1, 0, 1}; with a band, the sum along the readout path;
 * for an lvs_result_sum result, the one decoded sum); for an lvs_eq result,
 * the decoded value. */
lvs_status lvs_decrypt(const lvs_client_key *ck, const lvs_result *r, size_t pair, uint32_t *dist);
/* Decrypts every item of a result; dist has room for `items` values. */
lvs_status lvs_decrypt_all(const lvs_client_key *ck, const lvs_result *r, uint32_t *dist);
/* Client side, for a result received as exported words (lvs_result_export on
 * the server, lvs_result_info for m and n): the distance base + the sum of
 * the `count` rows ([count][k*N+1]) decoded to {-1, 0, 1}, with base = m for
 * the last row h[m][1..n] (count = n) and 0 for a band path (count = m + n);
 * a summed result (lvs_result_sum) is one row with base 0.  Host only. */
lvs_status lvs_decrypt_distance(const lvs_client_key *ck, const uint64_t *rows, size_t count, int64_t base,
                                uint32_t *dist);

/* ---------------------------------------------------------------- serving */

/* One query: an encrypted string against an encrypted reference (ref_enc,
 * same alphabet family) or against a plaintext reference held by the server
 * (ref_enc = NULL, ref_plain[0..ref_plain_len) in the query's alphabet).  The
 * plaintext case first builds the Section 5 table for the symbols occurring in
 * the reference (2 |S| m PBS, 1 for DNA), then runs one cell PBS per cell. */
typedef struct lvs_query {
    const lvs_ct_string *query;
    const lvs_ct_string *ref_enc;
    const uint8_t *ref_plain;
    size_t ref_plain_len;
} lvs_query;

typedef struct lvs_server_stats {
    uint64_t submitted, admitted, completed;
    uint64_t pending, active;   /* queue depth and admitted queries now          */
    uint64_t steps;             /* launch steps run                              */
    uint64_t pbs;               /* PBS run                                       */
    uint64_t max_step_pbs;      /* widest launch step                            */
    uint64_t mem_in_use;        /* device bytes held by admitted queries         */
    double busy_ms;             /* wall time spent inside launch steps           */
    uint64_t requeued;          /* admissions retried after a failed device      *
                                 * allocation while other queries held memory    */
} lvs_server_stats;

/* Continuous batching (Section 6.2 parallelism across cells and across
 * queries): a worker thread owned by the server runs launch steps on the
 * context's stream; each step bootstraps the union of the next anti-diagonal
 * work of every admitted query; queries are admitted in arrival order while
 * a slot is free (at most max_active admitted queries; 0 = no slot limit) and
 * their device footprint (ciphertext state, frontier, tables, result) fits
 * mem_budget_bytes (one query is always admitted when none runs).  A query
 * whose device allocation fails at admission goes back to the head of the
 * queue while other queries run (their memory frees up as they finish);
 * alone, it completes with LVS_ERR_OOM.  The context must not be used by
 * other threads while the server exists. */
lvs_status lvs_server_create(lvs_ctx *ctx, size_t mem_budget_bytes, size_t max_active, lvs_server **out);
/* Copies the query (the caller may free its strings afterwards) and returns a
 * ticket.  LVS_ERR_ARG if a symbol is outside the alphabet or the query alone
 * exceeds the budget. */
lvs_status lvs_server_submit(lvs_server *s, const lvs_query *q, uint64_t *ticket);
/* LVS_OK and the result (one item: m, n, encrypted h[m][1..n]; the caller owns
 * it) once the query is done; LVS_ERR_STATE while it is pending or running;
 * LVS_ERR_ARG for an unknown or already collected ticket. */
lvs_status lvs_server_poll(lvs_server *s, uint64_t ticket, lvs_result **out);
lvs_status lvs_server_stats_get(lvs_server *s, lvs_server_stats *out);
/* Stops the worker after its current step; unfinished queries are dropped. */
void lvs_server_free(lvs_server *s);

/* ---------------------------------------------------------------- low level */

/* PBS on device buffers (Section 2.2; key switch -> modulus switch -> blind
 * rotation -> sample extract).  d_in: count big ciphertexts, row stride
 * in_stride words (>= k*N+1); d_lut: count*16 bytes, LUT values in Z_32 (a
 * 16-entry table, inputs 16..31 give the negation, Table table_lutrelu);
 * d_out: count big ciphertexts with row stride out_stride.  Asynchronous on
 * the context stream; buffers must stay valid until it completes.  Scratch
 * memory is owned by the context. */
lvs_status lvs_pbs_batch_device(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride,
                                const uint8_t *d_lut, uint64_t *d_out, size_t out_stride,
                                size_t count);

/* FP64-FFT variant of the blind rotation (the paper's implementation relies
 * on TFHE-rs, whose bootstrap multiplies polynomials with a double-precision
 * FFT; Section 2.2 defines the PBS itself).  lvs_ctx_prepare_fft64 converts
 * the server key's bootstrapping key into the FFT domain on the context's
 * device (n * 8 * N/2 complex doubles: 109 MB at the default parameters, owned
 * by the context and freed with it); sk must be the key the context was made
 * from (LVS_ERR_ARG if its parameters differ).  A second call does nothing.
 * Synchronous.  lvs_pbs_batch_device_fft64 then takes the arguments of
 * lvs_pbs_batch_device and computes the same function with FFT products: the
 * outputs are not bit-identical to the exact NTT path (the key and the
 * products are rounded to 53-bit mantissas, an error far below the bootstrap
 * noise), but decrypt to the same messages.  LVS_ERR_STATE if the context has
 * no FFT key. */
lvs_status lvs_ctx_prepare_fft64(lvs_ctx *ctx, const lvs_server_key *sk);
lvs_status lvs_pbs_batch_device_fft64(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride,
                                      const uint8_t *d_lut, uint64_t *d_out, size_t out_stride,
                                      size_t count);

/* Allocation-free variant of lvs_pbs_batch_device (the paper has no
 * counterpart; this is a service of the library).  For callers that cannot
 * allocate device memory while they run -- a server that reserves its whole
 * memory budget at start-up and must not fail mid-request, a latency-critical
 * path that cannot take cudaMalloc's implicit synchronisation, or a host
 * program whose device allocator belongs to another framework.  Same
 * arguments, same result bit for bit; it calls no cudaMalloc / cudaFree and no
 * allocating routine on its success path.  Its scratch (job descriptors and
 * the modulus-switched masks passed from the key-switch kernel to the
 * blind-rotation kernel) lives in one static device array of
 * LVS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Limit: count * (64 + 4 (n+1)) bytes plus up to 255 bytes of
 * alignment must fit, i.e. at most 1232 PBS per call for n = 834 (12944 for
 * n = 64); larger counts fail with LVS_ERR_ARG and do nothing.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share the one array and every call rewrites
 * the part it uses before reading it (nothing needs to start at zero): calls
 * that overlap on the GPU -- different streams or contexts of the same device
 * -- race on it; issue them on one stream or serialise them.  The call holds
 * the context's lock like the other calls on a context.  It launches three
 * kernels (job descriptors, key switch, blind rotation; lvs_ctx_launch_count
 * counts them) and, with timing on, records its key-switch and blind-rotation
 * times only with the events lvs_ctx_set_timing created in advance. */
#define LVS_NOALLOC_SCRATCH_BYTES (4u << 20)
lvs_status lvs_pbs_batch_device_noalloc(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride,
                                        const uint8_t *d_lut, uint64_t *d_out, size_t out_stride,
                                        size_t count);

/* Autotuner of the launch shapes (no counterpart in the paper): for each
 * key-switch launch-size bucket (1-4, 5-16, 17-64, 65-256, 257-1024, more
 * PBS per launch) it times every candidate plan -- 4 or 16 PBS per CTA,
 * the 2048 input coefficients split over 1..32 CTAs with a finishing
 * reduction -- on synthetic jobs and keeps the fastest in the context; for
 * the blind rotation it finds the largest launch size for which the
 * three-CTA form (lvs_ctx_set_br_split) is faster, and for the key switch the
 * launch size from which the tensor-core form (lvs_ctx_set_ks_gemm_min) is.
 * Without it a heuristic plan is used (fill about two CTAs per SM).  Every
 * plan gives the same result bit for bit.  Synchronous; takes about a second;
 * allocates and frees its own scratch. */
lvs_status lvs_ctx_autotune(lvs_ctx *ctx);
/* The plan used for a launch of njobs PBS (jobs per CTA, split). */
lvs_status lvs_ctx_ks_plan(lvs_ctx *ctx, size_t njobs, int32_t *jobs_per_cta, int32_t *split);
/* Forces the plan of njobs' bucket (jobs_per_cta 4 or 16, split 1..32;
 * jobs_per_cta 0 restores the heuristic).  For tests and experiments. */
lvs_status lvs_ctx_set_ks_plan(lvs_ctx *ctx, size_t njobs, int32_t jobs_per_cta, int32_t split);
/* Blind-rotation launches of at most max_jobs PBS run as one cluster of three
 * CTAs per ciphertext (one per NTT prime, residues exchanged through
 * distributed shared memory): lower latency when the launch leaves SMs idle.
 * The default is one ciphertext per three SMs; lvs_ctx_autotune measures the
 * crossover.  Same results bit for bit.  lvs_ctx_set_br_split(ctx, 0) turns it
 * off; LVS_ERR_STATE if the device cannot run it. */
lvs_status lvs_ctx_br_split(lvs_ctx *ctx, size_t *max_jobs);
lvs_status lvs_ctx_set_br_split(lvs_ctx *ctx, size_t max_jobs);
/* Batch calls (lvs_edit_distance_batch, lvs_edit_distance_preprocessed_batch)
 * hold short pairs back a launch when that ends the launch on a full wave of
 * the blind-rotation grid (lvs_plan_batch with wave = the grid); on by
 * default, 0 turns it off.  The schedule changes which launch runs a step,
 * never a result: every pair's steps keep their order. */
lvs_status lvs_ctx_set_wave_fill(lvs_ctx *ctx, int32_t enable);
lvs_status lvs_ctx_wave_fill(lvs_ctx *ctx, int32_t *enabled);
/* Blind-rotation key source (no counterpart in the paper; Section 2.2's external
 * product reads one bootstrapping-key row per CMux).  0 (default): every chunk of
 * a row is read from global memory (L2) by the threads that use it.  1: the
 * key-staged form: the first three of the 16 chunks of the next CMux's row (36
 * KB) are copied into shared memory by the TMA engine (`cp.async.bulk`, one 1 KB
 * copy per warp and chunk, completed on an mbarrier) while the current CMux runs;
 * the rest come from global memory.  Same results bit for bit; the staged form
 * measured slower on GB300 and is kept as a measured alternative.  Its waits are
 * bounded (about one second): if one gives up, the launch's results are void and
 * the next lvs_ctx_synchronize (or result read) returns LVS_ERR_TIMEOUT; the
 * context stays usable.  Takes the context lock. */
lvs_status lvs_ctx_set_key_staging(lvs_ctx *ctx, int32_t enable);
lvs_status lvs_ctx_key_staging(lvs_ctx *ctx, int32_t *enabled);
/* Key-switch launches of at least min_jobs PBS run as a dense product on the
 * tensor cores: digits (|d| <= 4) times the key-switching key split into its
 * eight bytes, one bf16 x bf16 -> fp32 product over the whole reduction
 * (every partial sum an integer below 2^24 in magnitude, so exact) in the
 * library's own kernel, which rebuilds the words mod 2^64 and
 * modulus-switches them -- the same result bit for bit.  Default 1024;
 * lvs_ctx_autotune measures the crossover; 0 turns it off.  LVS_ERR_STATE if
 * the context could not set it up (it then uses the kernel for every size). */
lvs_status lvs_ctx_ks_gemm_min(lvs_ctx *ctx, size_t *min_jobs);
lvs_status lvs_ctx_set_ks_gemm_min(lvs_ctx *ctx, size_t min_jobs);
/* Wavefront steps (and PBS batches) wider than max_jobs PBS run as several
 * launches in sequence: bounded launch time and scratch.  The two lookups of
 * a refreshed cell always share a launch (the second reads the v row the
 * first one writes).  Default 65536; max_jobs in [2, 2^20], 0 restores the
 * default (LVS_ERR_ARG otherwise).  Same results bit for bit. */
lvs_status lvs_ctx_max_launch_jobs(lvs_ctx *ctx, size_t *max_jobs);
lvs_status lvs_ctx_set_max_launch_jobs(lvs_ctx *ctx, size_t max_jobs);

/* Test hook (host-side fault injection, no counterpart in the paper): the
 * next `count` allocations of batch / query device memory fail as if the
 * device were out of memory (LVS_ERR_OOM), without allocating.  0 clears it.
 * Lets the error paths (batch calls, server admission) be tested without
 * exhausting or faulting a GPU. */
void lvs_debug_fail_allocations(int32_t count);
/* Test hook (no counterpart in the paper): with `enable`, the key-staged blind
 * rotation (lvs_ctx_set_key_staging) never issues warp 0's copies into its first
 * staging slot, so that slot's first bounded wait runs out (about one second per
 * launch): the launch's results are void and the next lvs_ctx_synchronize
 * returns LVS_ERR_TIMEOUT, with no GPU fault and the context still usable.
 * 0 restores normal copies.  Takes the context lock. */
lvs_status lvs_debug_drop_key_copy(lvs_ctx *ctx, int32_t enable);

/* Measured issue rate of 32-bit integer multiplies on `device`: low-half
 * (mul.lo / IMAD) and high-half (mul.hi) results per SM per clock, from one
 * CTA per SM timed with the SM clock counter.  The roofline of the blind
 * rotation (no counterpart in the paper) uses it: a word-size modular
 * multiplication by a constant (Shoup) costs two low-half and one high-half
 * multiply.  Synchronous; allocates and frees its own buffers. */
lvs_status lvs_probe_int_mul(int device, double *lo_per_sm_clk, double *hi_per_sm_clk);
/* Achievable rates of the blind rotation's arithmetic on `device` (no
 * counterpart in the paper; a measurement aid): modular multiplications by a
 * constant (Shoup, the product of the NTT butterflies, Section 2.2's external
 * product) and complete lazy NTT butterflies, each per SM per clock, from one
 * CTA per SM of independent register-resident streams timed with the SM clock
 * counter.  They bound what a kernel made of these operations can reach, below
 * the multiply issue rates of lvs_probe_int_mul.  Synchronous; allocates and
 * frees its own small buffers.  LVS_ERR_CUDA without a usable device. */
lvs_status lvs_probe_modmul(int device, double *shoup_per_sm_clk, double *butterfly_per_sm_clk);
/* Ceilings of the blind rotation's key product on `device` (no counterpart in
 * the paper; a measurement aid for the pointwise products of Section 2.2's
 * external product in the NTT domain): 32x32 -> 64-bit multiply-accumulates per
 * SM per clock (the Montgomery sums), and L2 -> SM read bytes per SM per clock
 * in the product's access shape (one CTA of 384 threads per SM, each thread 32
 * bytes of each of the 16 chunks of a 192 KB key row, all SMs on the same row,
 * a 96 MB buffer that stays in L2).  Timed with the SM clock counter; each
 * kernel runs twice and the second run counts.  Synchronous; allocates and frees
 * its own buffers (96 MB).  LVS_ERR_CUDA without a usable device, LVS_ERR_OOM if
 * the buffers cannot be allocated. */
lvs_status lvs_probe_key_product(int device, double *wide_per_sm_clk, double *l2_bytes_per_sm_clk);

/* Key switch + modulus switch only: d_out receives count * (n+1) uint32
 * values round(a * 2N / 2^64) of the key-switched ciphertexts. */
lvs_status lvs_keyswitch_batch_device(lvs_ctx *ctx, const uint64_t *d_in, size_t in_stride,
                                      uint32_t *d_out, size_t count);

/* Exact negacyclic products mod 2^64 through the NTT/CRT path of the blind
 * rotation: for each of count items, out = sum_{r<4} dig[r] * poly[r][c] for
 * c in {0,1}, with dig (int32, |d| <= 4096) [count][4][N] and poly (uint64)
 * [count][4][2][N]; out [count][2][N].  Tests the product kernel alone. */
lvs_status lvs_poly_mul_device(lvs_ctx *ctx, const int32_t *d_dig, const uint64_t *d_poly,
                               uint64_t *d_out, size_t count);

/* Kernel timing over a region of calls (CUDA events on the context stream).
 * kind: 0 = blind rotation kernel, 1 = key-switch kernel.  Enabling creates a
 * pool of events up front (calls take events from it and return them once the
 * times are read); a call that finds the pool empty creates more, except the
 * allocation-free entry point, which then leaves its launches untimed.  Batch
 * calls stay on their CUDA graph while timing is on: the events are recorded
 * by event-record nodes of the graph, so the timed launches are the graph's. */
typedef struct lvs_kernel_stats {
    uint64_t launches;        /* kernel launches timed                          */
    uint64_t items;           /* PBS (or key switches) processed by them        */
    double total_ms;          /* sum of event-measured durations                */
} lvs_kernel_stats;
lvs_status lvs_ctx_set_timing(lvs_ctx *ctx, int enable);
lvs_status lvs_ctx_kernel_stats(lvs_ctx *ctx, int kind, lvs_kernel_stats *out);
/* PBS executed by the context since creation (counter, host side). */
lvs_status lvs_ctx_pbs_count(lvs_ctx *ctx, uint64_t *out);
/* CUDA kernels launched by the context since creation (counter, host side;
 * a launch inside a CUDA graph counts when the graph is launched). */
lvs_status lvs_ctx_launch_count(lvs_ctx *ctx, uint64_t *out);

#ifdef __cplusplus
}
#endif
#endif /* LVS_H */
