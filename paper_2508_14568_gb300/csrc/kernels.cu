// CUDA kernels of the Leuvenshtein hot path on GB300 (sm_103a):
//   k_keyswitch     gather of the PBS input (a linear combination of big
//                   ciphertexts), key switch big key -> s and modulus switch
//   k_blind_rotate  persistent blind rotation: test-polynomial (LUT) encoding,
//                   n CMux / external products through the exact NTT path,
//                   sample extract and the Leuvenshtein cell epilogue
//   k_bsk_to_ntt    one-time conversion of the bootstrapping key to the NTT
//                   domain, in the register order of k_blind_rotate
// plus small helpers and a product-only kernel for parity tests.
#include <algorithm>
#include <cstdio>

#include <cooperative_groups.h>

#include "lvs_internal.hpp"
#include "ntt.cuh"

namespace lvs {
namespace dev {

__constant__ PrimeConsts c_pc;

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint32_t residue_of_signed(int64_t x, uint32_t p)
{
    int64_t r = x % (int64_t)p;
    return (uint32_t)(r < 0 ? r + p : r);
}

// NTT-domain key layout: for BSK index i, prime g and register q, the [T][8]
// words of the T threads (slot = row * 2 + column) are stored warp by warp,
// each warp's 32 threads as one contiguous kilobyte [half][lane][4 u32]: the
// word of (tau, slot) is at key_lane_word(tau) + (slot >> 2) * 128 + (slot & 3).
// A warp's piece is one bulk copy, and both halves read conflict-free.
__device__ __forceinline__ uint32_t key_lane_word(uint32_t tau) { return (tau >> 5) * 256u + (tau & 31u) * 4u; }

// Bulk copies global -> shared through the TMA engine, completed on an
// mbarrier (transaction bytes), and bounded waits on the barrier's phase.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *m)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(m)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *m, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(m)), "r"(parity)
                 : "memory");
    return ok != 0;
}
constexpr long long kKeyWaitCycles = 2000000000LL;   // about one second at the GB300's SM clock
// Wait for phase `parity` of m.  Gives up after kKeyWaitCycles, or at once when
// another thread of the CTA has given up (*abort, unless `final`): it then sets
// *abort and the host-visible *fault, and the caller goes on with whatever the
// slot holds, so every barrier of the kernel is still reached and the launch
// ends normally (its results are void; the host reports LVS_ERR_TIMEOUT).
// `final`: the wait for a copy that is known to be in flight before the CTA
// exits, which must not be cut short by another thread's give-up.  Returns
// whether the phase completed.
__device__ __forceinline__ bool key_wait(uint64_t *m, uint32_t parity, volatile uint32_t *abort,
                                         volatile uint32_t *fault, bool final = false)
{
    if (mbar_test(m, parity)) return true;
    const long long t0 = clock64();
    while (final || *abort == 0) {
        if (mbar_test(m, parity)) return true;
        if (clock64() - t0 > kKeyWaitCycles) {
            *abort = 1;
            if (fault) *fault = 1;
            return false;
        }
    }
    return false;
}

// Staging of the head of each BSK row in shared memory (the key-staged form of
// the blind rotation): KR slots, slot q holding chunk q (register q of the row,
// 12 KB for the CTA) of the next CMux's row; each warp's kilobyte is its own
// bulk copy on its own barrier, issued as soon as the warp has used the current
// row's chunk q, so it lands while the rest of the CMux runs.  Every slot is
// used once per CMux: the barrier phase of CMux m is m & 1 (r).  drop: a test
// hook that never issues warp 0's copies into slot 0 (its first wait then runs
// out and the launch reports LVS_ERR_TIMEOUT).  Once any wait of the CTA has
// given up, no warp issues another copy (a slot whose copy may still be in
// flight is never refilled); lane 0 of each warp keeps which of its copies it has
// not yet seen land (pend, with the barrier parity of each in par) and waits for
// those before the CTA exits.
template <int KR>
struct KeyRing {
    uint4 *slots;              // [KR][warps][64] uint4
    uint64_t *mbar;            // [KR][warps]
    volatile uint32_t *abort;  // shared: set once a wait gave up
    volatile uint32_t *fault;  // host-visible (mapped), may be null
    uint32_t r;
    uint32_t drop;
    uint32_t pend, par;        // lane 0 of each warp
};

// Value of the rotated test polynomial v' = X^{-box/2} v, v[t] = f[t / box] * Delta,
// at index idx in [0, 2N) of X^{-b} v' (negacyclic extension).
template <int LOGN>
__device__ __forceinline__ uint64_t test_poly_at(const uint8_t (&f)[16], uint32_t idx)
{
    constexpr uint32_t N = 1u << LOGN, box = N / 16;
    const bool neg = idx >= N;
    const uint32_t t = idx & (N - 1);
    uint64_t v;
    if (t < N - box / 2) v = (uint64_t)(f[(t + box / 2) / box] & 31u) << kDeltaLog;
    else v = 0 - ((uint64_t)(f[0] & 31u) << kDeltaLog);
    return neg ? 0 - v : v;
}

// External product core for prime group g: digit residues d (L0 layout, in
// [0, p)) -> forward NTT -> Montgomery products with the key slice `key`
// ([16][T][8] u32 for this prime, key_lane_word layout) -> inverse NTT ->
// residues of the two output polynomials written to out[j*N + e].
// OUT_IN_BUF: out lies in this group's exchange buffer, so the group first
// waits until every thread has read its last inverse exchange.
// KR > 0: chunks 0 .. KR-1 of `key` come from the staging slots of R (in flight
// or landed on entry); after using chunk q < KR the warp refills slot q with
// chunk q of `key_next` (the next CMux's slice); the other chunks, and the first
// two of them issued before the slots are read, come from global memory.
template <int LOGN, bool OUT_IN_BUF = false, int KR = 0>
__device__ __forceinline__ void ext_product_core(uint32_t (&d)[4][16], const uint32_t *__restrict__ key,
                                                 uint32_t *buf, uint32_t *out, uint32_t tau, int g,
                                                 const uint2 *__restrict__ twf, const uint2 *__restrict__ twi,
                                                 KeyRing<KR> *R = nullptr,
                                                 const uint32_t *__restrict__ key_next = nullptr, int tid = 0)
{
    using Lay = Layout<LOGN>;
    constexpr int N = Lay::N, T = Lay::T;
    const uint32_t p = c_pc.p[g], pinv = c_pc.pinv_neg[g], z = c_pc.zero;
    ntt_forward4<LOGN>(d, reinterpret_cast<uint4 *>(buf), tau, twf, p, 1 + g, z);

    // pointwise: out_c = sum_r D_r * K[r][c] (Montgomery), written over D_0, D_1
    constexpr int NW = 3 * T / 32;   // warps of the CTA (ring)
    const int w = tid >> 5, lane = tid & 31;
    const uint4 *kp = reinterpret_cast<const uint4 *>(key + key_lane_word(tau));
    // chunk q < KR: from slot q, landed during the previous CMux (barrier phase
    // R->r); the others straight from global memory
    auto head_load = [&](int q, uint4 &x, uint4 &y) {
        if (key_wait(R->mbar + q * NW + w, R->r, R->abort, R->fault)) R->pend &= ~(1u << q);
        const uint4 *sp = R->slots + (size_t)(q * NW + w) * 64;
        x = sp[lane];
        y = sp[32 + lane];
    };
    uint4 ka, kb, ea, eb, fa, fb;
    if constexpr (KR > 0) {
        ea = __ldg(kp + (size_t)KR * T * 2);
        eb = __ldg(kp + (size_t)KR * T * 2 + 32);
        fa = __ldg(kp + (size_t)(KR + 1) * T * 2);
        fb = __ldg(kp + (size_t)(KR + 1) * T * 2 + 32);
        head_load(0, ka, kb);
    }
    else {
        ka = __ldg(kp);
        kb = __ldg(kp + 32);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        uint4 na, nb;
        if (q + 1 < 16) {
            if (q + 1 < KR) head_load(q + 1, na, nb);
            else if (KR > 0 && q + 1 == KR) { na = ea; nb = eb; }
            else if (KR > 0 && q + 1 == KR + 1) { na = fa; nb = fb; }
            else {
                const uint4 *np = kp + (size_t)(q + 1) * T * 2;
                na = __ldg(np);
                nb = __ldg(np + 32);
            }
        }
        // transform values in [0, 4p) -> [0, 2p); key residues < p: each sum of
        // four products is below 8 p^2 < 2^63, REDC returns it below 3p, and one
        // more conditional subtraction gives the [0, 2p) the inverse expects
        const uint32_t d0 = csubz(d[0][q], 2 * p, z);
        const uint32_t d1 = csubz(d[1][q], 2 * p, z);
        const uint32_t d2 = csubz(d[2][q], 2 * p, z);
        const uint32_t d3 = csubz(d[3][q], 2 * p, z);
        // slot = row * 2 + column
        const uint64_t t0 = (uint64_t)d0 * ka.x + (uint64_t)d1 * ka.z + (uint64_t)d2 * kb.x + (uint64_t)d3 * kb.z;
        const uint64_t t1 = (uint64_t)d0 * ka.y + (uint64_t)d1 * ka.w + (uint64_t)d2 * kb.y + (uint64_t)d3 * kb.w;
        d[0][q] = csubz(redc(t0, p, pinv), 2 * p, z);
        d[1][q] = csubz(redc(t1, p, pinv), 2 * p, z);
        if (q < KR) {
            // every lane has read chunk q (and used it): its slot takes chunk q of
            // the next CMux
            __syncwarp();
            if (lane == 0 && !(R->drop && w == 0 && q == 0) && *R->abort == 0) {
                fence_proxy_async();
                bulk_g2s(R->slots + (size_t)(q * NW + w) * 64, key_next + (size_t)q * T * 8 + (tau >> 5) * 256u, 1024,
                         R->mbar + q * NW + w);
                R->pend |= 1u << q;   // completes the next CMux's phase
                R->par = (R->par & ~(1u << q)) | ((R->r ^ 1u) << q);
            }
        }
        if (q + 1 < 16) { ka = na; kb = nb; }
    }
    ntt_inverse2<LOGN>(d, reinterpret_cast<uint2 *>(buf), tau, twi, p, 1 + g, z);
    if (OUT_IN_BUF) {
        if (T > 32) group_bar(1 + g, T); else __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint32_t e = tau | ((uint32_t)q << Lay::B0);
        out[0 * N + e] = csubz(d[0][q], p, z);
        out[1 * N + e] = csubz(d[1][q], p, z);
    }
}

// Digit residues (mod this group's prime) of X^a ACC - ACC at the 16 positions
// of the thread in the L0 layout, for the mask (j = 0) and body (j = 1)
// polynomials of the negacyclically extended accumulator acc ([2][2N]).
// Only the rounded top 2*base_log bits of x are used: with
// shift = 64 - 2*base_log >= 32, (x + 2^(shift-1)) >> shift =
// (hi32(x) + 2^(shift-33)) >> (shift-32).  Balanced digits with carry,
// least significant level first; d < 0 is stored as d + p (< 2p is fine).
template <int LOGN>
__device__ __forceinline__ void decompose(uint32_t (&d)[4][16], const uint64_t *acc, uint32_t a, uint32_t tau,
                                          uint32_t base_log, uint32_t pmB)
{
    using Lay = Layout<LOGN>;
    constexpr int N = Lay::N;
    const uint32_t B = 1u << base_log, hB = B >> 1;
    const uint32_t hshift = 64 - 2 * base_log - 32;   // shift - 32
    const uint32_t hround = 1u << (hshift - 1);       // 2^(shift - 33)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint32_t e = tau | ((uint32_t)q << Lay::B0);
        const uint32_t src = (e - a) & (2 * N - 1);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t *A = acc + j * 2 * N;
            const uint64_t x = A[src] - A[e];
            const uint32_t v = ((uint32_t)(x >> 32) + hround) >> hshift;
            const uint32_t u2 = v & (B - 1);
            const uint32_t c2 = u2 >> (base_log - 1);   // u2 >= B/2
            const uint32_t r1 = (v >> base_log) + c2;    // <= B
            const uint32_t c1 = (r1 + hB) >> base_log;   // r1 >= B/2 (r1 = B gives 1)
            d[2 * j + 1][q] = u2 + c2 * pmB;
            d[2 * j + 0][q] = r1 + c1 * pmB;
        }
    }
}

// Digits of X^a ACC - ACC for all 2N coefficients, computed once for the CTA
// instead of once per prime group (threads tid, tid + nthreads, ...), with the
// rounding and balanced-digit rule of decompose(): the digit residues (d < 0
// stored as d + p_g) of every prime g go into prime g's exchange buffer at the
// 16-byte word of position e (pass-0 layout: level-1 and level-2 digits of the
// mask, then of the body), from which each prime group loads its own positions.
template <int LOGN>
__device__ __forceinline__ void decompose_shared(uint32_t *bufs, const uint64_t *acc, uint32_t a, int tid,
                                                 int nthreads, uint32_t base_log)
{
    constexpr int N = 1 << LOGN;
    const uint32_t B = 1u << base_log, hB = B >> 1;
    const uint32_t hshift = 64 - 2 * base_log - 32;
    const uint32_t hround = 1u << (hshift - 1);
    const uint32_t pm0 = c_pc.p[0] - B, pm1 = c_pc.p[1] - B, pm2 = c_pc.p[2] - B;
    for (int c = tid; c < 2 * N; c += nthreads) {
        const int j = c >> LOGN;
        const uint32_t e = c & (N - 1);
        // (X^a ACC)[e] = +-ACC[(e - a) mod N], negative when (e - a) mod 2N >= N
        const uint32_t src = (e - a) & (2 * N - 1);
        const uint64_t *A = acc + j * N;
        const uint64_t rot = A[src & (N - 1)];
        const uint64_t x = (src < (uint32_t)N ? rot : 0 - rot) - A[e];
        const uint32_t v = ((uint32_t)(x >> 32) + hround) >> hshift;
        const uint32_t u2 = v & (B - 1);
        const uint32_t c2 = u2 >> (base_log - 1);
        const uint32_t r1 = (v >> base_log) + c2;
        const uint32_t c1 = (r1 + hB) >> base_log;
        const uint32_t w = w16(e) * 4 + 2 * j;   // u32 index of this component's two digits
        *reinterpret_cast<uint2 *>(bufs + 0 * 4 * ExWords<LOGN>::WORDS + w) = make_uint2(r1 + c1 * pm0, u2 + c2 * pm0);
        *reinterpret_cast<uint2 *>(bufs + 1 * 4 * ExWords<LOGN>::WORDS + w) = make_uint2(r1 + c1 * pm1, u2 + c2 * pm1);
        *reinterpret_cast<uint2 *>(bufs + 2 * 4 * ExWords<LOGN>::WORDS + w) = make_uint2(r1 + c1 * pm2, u2 + c2 * pm2);
    }
}

// Sample extract (coefficient 0) of the extended accumulator and the job's
// epilogue: a_0 = A[0], a_u = -A[N - u] = A[2N - u] (u > 0), b = B[0]; a cell
// job updates v[i] = M - h[i-1][j], h[j] = M - v[i][j-1] in place (and copies
// one of them to its tap row), a store job writes the ciphertext (and its tap).
// EXT: acc negacyclically extended ([2][2N]); otherwise stored once ([2][N]).
template <int LOGN, bool EXT>
__device__ __forceinline__ void sample_extract_epilogue(const Job &J, const uint64_t *acc, int tid, int nthreads)
{
    constexpr int N = 1 << LOGN;
    uint64_t *o0 = J.dst[0];
    uint64_t *o1 = J.dst[1];
    for (int u = tid; u <= N; u += nthreads) {
        const uint64_t val = EXT ? (u == N ? acc[2 * N] : acc[(2 * N - u) & (2 * N - 1)])
                                 : (u == N ? acc[N] : (u == 0 ? acc[0] : 0 - acc[N - u]));
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
}

// ---------------------------------------------------------------- blind rotation
// Shared memory of k_blind_rotate: the accumulator (stored once, [2][N]), one
// exchange buffer per prime group, the three primes' output residues for the
// CRT and, in the key-staged form (KR > 0), the KR staging slots of 12 KB and
// their barriers (one per slot and warp) plus the give-up flag.
constexpr int kKeyStageChunks = 3;   // what fits beside the 182 KB above
template <int LOGN, int KR>
struct BrSmem {
    static constexpr int N = 1 << LOGN;
    static constexpr int NW = 3 * N / 16 / 32;
    static constexpr size_t acc_bytes = 2 * N * sizeof(uint64_t);
    static constexpr size_t buf_bytes = 3 * (size_t)ExWords<LOGN>::WORDS * 16;
    static constexpr size_t crt_bytes = 3 * 2 * N * sizeof(uint32_t);
    static constexpr size_t ring_bytes = (size_t)KR * NW * 1024;
    static constexpr size_t mbar_bytes = KR > 0 ? (size_t)KR * NW * 8 + 16 : 0;
    static constexpr size_t ring_off = acc_bytes + buf_bytes + crt_bytes;
    static constexpr size_t total = ring_off + ring_bytes + mbar_bytes;
};

// KR = 0: every key chunk from global memory (L2); KR = kKeyStageChunks: the
// key-staged form (KeyRing).  drop_copy: KeyRing::drop (tests only).
template <int LOGN, int KR>
__global__ void __launch_bounds__(3 * (1 << LOGN) / 16, 1)
k_blind_rotate(const Job *__restrict__ jobs, uint32_t njobs, const uint32_t *__restrict__ ms, uint32_t n, const uint32_t *__restrict__ bsk,
               const uint2 *__restrict__ tw, const uint8_t *__restrict__ luts, int lut_per_job,
               uint32_t base_log, volatile uint32_t *fault, uint32_t drop_copy)
{
    using Lay = Layout<LOGN>;
    using SM = BrSmem<LOGN, KR>;
    constexpr int N = Lay::N, T = Lay::T, NT = 3 * T, NW = SM::NW;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *acc = reinterpret_cast<uint64_t *>(smem_raw);   // [2][N]: mask, body
    uint32_t *bufs = reinterpret_cast<uint32_t *>(smem_raw + SM::acc_bytes);
    uint32_t *crt = bufs + 3 * 4 * ExWords<LOGN>::WORDS;

    const int tid = threadIdx.x;
    const int g = tid / T;
    const uint32_t tau = tid % T;
    uint32_t *buf = bufs + g * 4 * ExWords<LOGN>::WORDS;
    const uint2 *twf = tw + (size_t)(g * 2 + 0) * N;
    const uint2 *twi = tw + (size_t)(g * 2 + 1) * N;
    const size_t key_row = (size_t)3 * 16 * T * 8;   // u32 per BSK index i
    const uint32_t *bsk_g = bsk + (size_t)g * 16 * T * 8;

    // key staging (KR > 0): the CMux sequence runs through the rows i, i + 1
    // mod n, ... of every job of this CTA; the slots start with the head of row 0
    KeyRing<KR> R;
    const int w = tid >> 5, lane = tid & 31;
    const bool has_work = blockIdx.x < njobs;
    if constexpr (KR > 0) {
        R.slots = reinterpret_cast<uint4 *>(smem_raw + SM::ring_off);
        R.mbar = reinterpret_cast<uint64_t *>(smem_raw + SM::ring_off + SM::ring_bytes);
        R.abort = reinterpret_cast<volatile uint32_t *>(R.mbar + KR * NW);
        R.fault = fault;
        R.r = 0;
        R.drop = drop_copy;
        R.pend = 0;
        R.par = 0;
        if (tid == 0) {
            for (int k = 0; k < KR * NW; ++k) mbar_init(R.mbar + k, 1);
            *R.abort = 0;
            fence_mbar_init();
        }
        __syncthreads();
        if (has_work && lane == 0) {
#pragma unroll
            for (int q = 0; q < KR; ++q)
                if (!(drop_copy && w == 0 && q == 0)) {
                    bulk_g2s(R.slots + (size_t)(q * NW + w) * 64, bsk_g + (size_t)q * T * 8 + (tau >> 5) * 256u, 1024,
                             R.mbar + q * NW + w);
                    R.pend |= 1u << q;   // phase 0
                }
        }
    }

    for (uint32_t job = blockIdx.x; job < njobs; job += gridDim.x) {
        const Job J = jobs[job];
        const uint32_t *msj = ms + (size_t)job * (n + 1);
        uint8_t f[16];
        {
            const uint8_t *lp = luts + (lut_per_job ? (size_t)job * 16 : (size_t)J.lut * 16);
            const uint4 lv = *reinterpret_cast<const uint4 *>(lp);
            memcpy(f, &lv, 16);
        }
        // ACC = (0, X^{-b} v'), each polynomial stored once (acc[j][e], e < N)
        const uint32_t b = __ldg(msj + n);
        for (int t = tid; t < N; t += NT) {
            acc[t] = 0;
            acc[N + t] = test_poly_at<LOGN>(f, (t + b) & (2 * N - 1));
        }
        __syncthreads();

        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t a = __ldg(msj + i);
            // X^0 ACC - ACC = 0: the external product is exactly 0.  The staged
            // form runs it anyway (digits 0, an exactly zero product) so that
            // every CMux takes its row's head from the slots in order.
            if (KR == 0 && a == 0) continue;
            const uint32_t inext = i + 1 == n ? 0 : i + 1;
            // digits once for the CTA into the exchange buffers; each prime group
            // then loads its positions (the same words its first exchange rewrites)
            decompose_shared<LOGN>(bufs, acc, a, tid, NT, base_log);
            __syncthreads();
            uint32_t d[4][16];
            ld4<Lay::B0, 4>(reinterpret_cast<const uint4 *>(buf), d, w16(Lay::base0(tau)));
            ext_product_core<LOGN, false, KR>(d, bsk_g + (size_t)i * key_row, buf, crt + g * 2 * N, tau, g, twf, twi,
                                              &R, bsk_g + (size_t)inext * key_row, tid);
            if constexpr (KR > 0) R.r ^= 1u;
            __syncthreads();
            // four reconstructions in flight per thread (Garner's steps are a
            // dependent chain; 2, 6, 8 and 11 measured slower)
#pragma unroll 4
            for (int c = tid; c < 2 * N; c += NT) {
                const int j = c >> LOGN, e = c & (N - 1);
                const uint64_t x = crt3(crt[(0 * 2 + j) * N + e], crt[(1 * 2 + j) * N + e],
                                        crt[(2 * 2 + j) * N + e], c_pc);
                acc[j * N + e] += x;
            }
            __syncthreads();
        }

        sample_extract_epilogue<LOGN, false>(J, acc, tid, NT);
        __syncthreads();
    }
    // no bulk copy may be in flight when the CTA exits: lane 0 of each warp
    // waits for the copies it has not seen land (normally its last KR, the head
    // of row 0 again, never used)
    if constexpr (KR > 0) {
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < KR; ++k)
                if (R.pend & (1u << k)) key_wait(R.mbar + k * NW + w, (R.par >> k) & 1u, R.abort, R.fault, true);
        }
    }
}

// ---------------------------------------------------------------- key switch
// out = (0, b) - sum_{u, lev} d_{u,lev} KSK[u][lev].  Digits are kept offset to
// d' = d + B/2 in [0, B), so each product is unsigned: the low 32 bits of the
// KSK word go through one 32x32->64 multiply-add into a 64-bit sum and the high
// 32 bits through one 32-bit multiply-add (only needed mod 2^32); the offset
// comes back as (B/2) * colsum[c], colsum[c] = sum_{u,lev} KSK[u][lev][c].
constexpr int KS_THREADS = 128; // output columns per CTA
constexpr int KS_UCH = 64;      // input coefficients per digit chunk
constexpr int KS_MAXL = 8;

// TJ jobs per CTA (a multiple of 4).  blockIdx.z / gridDim.z splits the input
// coefficients into chunk ranges ("split-K"): with one split the epilogue adds
// the body and modulus-switches into ms; with several, each split writes its
// partial sum (mod 2^64, offset not yet removed) to part[z][j][c] and
// k_ks_finish completes them.
template <int TJ>
__global__ void __launch_bounds__(KS_THREADS)
k_keyswitch(const Job *__restrict__ jobs, uint32_t njobs,
            const uint64_t *__restrict__ ksk, const uint64_t *__restrict__ colsum, uint32_t n, uint32_t big,
            uint32_t ks_level, uint32_t ks_base_log, uint32_t log2_2N, uint32_t *__restrict__ ms,
            uint64_t *__restrict__ part)
{
    __shared__ __align__(16) uint32_t dig[KS_UCH][KS_MAXL][TJ];
    __shared__ Job sj[TJ];
    const int t = threadIdx.x;
    const uint32_t j0 = blockIdx.x * TJ;
    const uint32_t c = blockIdx.y * KS_THREADS + t;
    if (t < TJ) {
        if (j0 + t < njobs) sj[t] = jobs[j0 + t];
        else {
            Job z{};
            sj[t] = z;
        }
    }
    __syncthreads();

    const uint32_t beta = ks_level * ks_base_log;
    const uint64_t rnd = 1ull << (63 - beta);
    const uint32_t Bk = 1u << ks_base_log, hBk = Bk >> 1;
    uint64_t lo[TJ];
    uint32_t hi[TJ];
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) { lo[jj] = 0; hi[jj] = 0; }

    // this split's chunk range
    const uint32_t nch = (big + KS_UCH - 1) / KS_UCH, S = gridDim.z, z = blockIdx.z;
    const uint32_t ch0 = (uint32_t)(((uint64_t)nch * z) / S), ch1 = (uint32_t)(((uint64_t)nch * (z + 1)) / S);

    // digit prologue: thread t covers coefficient u0 + (t % KS_UCH) of TJ/2 jobs
    const int tu = t % KS_UCH, tj = (t / KS_UCH) * (TJ / 2);
    for (uint32_t u0 = ch0 * KS_UCH; u0 < ch1 * KS_UCH && u0 < big; u0 += KS_UCH) {
        const uint32_t u = u0 + tu;
#pragma unroll 1
        for (int jj = tj; jj < tj + TJ / 2; ++jj) {
            uint64_t a = 0;
            if (u < big) {
#pragma unroll
                for (int s = 0; s < 3; ++s)
                    if (sj[jj].src[s]) a += (uint64_t)(int64_t)sj[jj].coef[s] * __ldg(sj[jj].src[s] + u);
            }
            const uint64_t v = (a + rnd) >> (64 - beta);
            uint32_t carry = 0;
            for (int lev = (int)ks_level; lev >= 1; --lev) {
                const uint32_t uu = (uint32_t)(v >> ((ks_level - lev) * ks_base_log)) & (Bk - 1);
                const uint32_t r = uu + carry;
                carry = r >= hBk;
                dig[tu][lev - 1][jj] = r - carry * Bk + hBk;   // balanced digit + B/2
            }
        }
        __syncthreads();
        if (c <= n) {
            const uint32_t ucount = min((uint32_t)KS_UCH, big - u0);
            for (uint32_t ul = 0; ul < ucount; ++ul) {
                const uint64_t *krow = ksk + ((size_t)(u0 + ul) * ks_level) * (n + 1) + c;
                for (uint32_t lev = 0; lev < ks_level; ++lev) {
                    const uint64_t kv = __ldg(krow + (size_t)lev * (n + 1));
                    const uint32_t klo = (uint32_t)kv, khi = (uint32_t)(kv >> 32);
                    const uint4 *dp = reinterpret_cast<const uint4 *>(&dig[ul][lev][0]);
#pragma unroll
                    for (int w = 0; w < TJ / 4; ++w) {
                        const uint4 dv = dp[w];
                        lo[4 * w + 0] += (uint64_t)dv.x * klo; hi[4 * w + 0] += dv.x * khi;
                        lo[4 * w + 1] += (uint64_t)dv.y * klo; hi[4 * w + 1] += dv.y * khi;
                        lo[4 * w + 2] += (uint64_t)dv.z * klo; hi[4 * w + 2] += dv.z * khi;
                        lo[4 * w + 3] += (uint64_t)dv.w * klo; hi[4 * w + 3] += dv.w * khi;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (c > n) return;
    if (S > 1) {
#pragma unroll
        for (int jj = 0; jj < TJ; ++jj) {
            const uint32_t j = j0 + jj;
            if (j < njobs) part[((size_t)z * njobs + j) * (n + 1) + c] = lo[jj] + ((uint64_t)hi[jj] << 32);
        }
        return;
    }
    const uint32_t twoN_mask = (1u << log2_2N) - 1;
    const uint64_t offset = (uint64_t)hBk * colsum[c];
#pragma unroll
    for (int jj = 0; jj < TJ; ++jj) {
        const uint32_t j = j0 + jj;
        if (j < njobs) {
            const uint64_t sum = lo[jj] + ((uint64_t)hi[jj] << 32) - offset;   // sum_{u,lev} d * KSK
            uint64_t val = 0 - sum;
            if (c == n) {
                uint64_t bb = (uint64_t)(sj[jj].cst & 31) << kDeltaLog;
                for (int s = 0; s < 3; ++s)
                    if (sj[jj].src[s]) bb += (uint64_t)(int64_t)sj[jj].coef[s] * sj[jj].src[s][big];
                val += bb;
            }
            ms[(size_t)j * (n + 1) + c] = (uint32_t)((val + (1ull << (63 - log2_2N))) >> (64 - log2_2N)) & twoN_mask;
        }
    }
}

// completes a split key switch: sum of the S partial sums, offset removal,
// body, modulus switch (one thread per output value)
__global__ void k_ks_finish(const Job *__restrict__ jobs, uint32_t njobs, const uint64_t *__restrict__ part,
                            uint32_t S, const uint64_t *__restrict__ colsum, uint32_t n, uint32_t big,
                            uint32_t ks_base_log, uint32_t log2_2N, uint32_t *__restrict__ ms)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)njobs * (n + 1)) return;
    const uint32_t j = (uint32_t)(idx / (n + 1)), c = (uint32_t)(idx % (n + 1));
    uint64_t sum = 0;
    for (uint32_t z = 0; z < S; ++z) sum += part[(size_t)z * njobs * (n + 1) + idx];
    sum -= (uint64_t)(1u << (ks_base_log - 1)) * colsum[c];
    uint64_t val = 0 - sum;
    if (c == n) {
        const Job &J = jobs[j];
        uint64_t bb = (uint64_t)(J.cst & 31) << kDeltaLog;
        for (int s = 0; s < 3; ++s)
            if (J.src[s]) bb += (uint64_t)(int64_t)J.coef[s] * J.src[s][big];
        val += bb;
    }
    ms[idx] = (uint32_t)((val + (1ull << (63 - log2_2N))) >> (64 - log2_2N)) & ((1u << log2_2N) - 1);
}

// colsum[c] = sum over all KSK rows of column c (mod 2^64), once per context
__global__ void k_ksk_colsum(const uint64_t *__restrict__ ksk, uint32_t rows, uint32_t n, uint64_t *colsum)
{
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n) return;
    uint64_t s = 0;
    for (uint32_t r = 0; r < rows; ++r) s += ksk[(size_t)r * (n + 1) + c];
    colsum[c] = s;
}

// ---------------------------------------------------------------- key conversion
// BSK (coefficient domain, [i][row][col][N] u64) -> NTT domain
// out[i][g][q][(tau, slot = row*2+col) in key_lane_word order] = NTT_p(row,col)[pos(tau,q)] * R * N^{-1} mod p
template <int LOGN>
__global__ void __launch_bounds__(3 * (1 << LOGN) / 16)
k_bsk_to_ntt(const uint64_t *__restrict__ coef, uint32_t count, uint32_t *__restrict__ out,
             const uint2 *__restrict__ tw, uint32_t m0, uint32_t ms0, uint32_t m1, uint32_t ms1, uint32_t m2,
             uint32_t ms2)
{
    using Lay = Layout<LOGN>;
    constexpr int N = Lay::N, T = Lay::T;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t *bufs = reinterpret_cast<uint32_t *>(smem_raw);
    const int tid = threadIdx.x, g = tid / T;
    const uint32_t tau = tid % T;
    const uint32_t i = blockIdx.x, h = blockIdx.y;   // h: slots 4h..4h+3
    if (i >= count) return;
    const uint32_t p = c_pc.p[g];
    uint32_t v[4][16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t slot = 4 * h + k;   // = row * 2 + col
        const uint64_t *src = coef + ((size_t)i * 8 + slot) * N;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t e = tau | ((uint32_t)q << Lay::B0);
            v[k][q] = residue_of_signed((int64_t)src[e], p);
        }
    }
    ntt_forward4<LOGN>(v, reinterpret_cast<uint4 *>(bufs + g * 4 * ExWords<LOGN>::WORDS), tau, tw + (size_t)(g * 2) * N,
                       p, 1 + g, c_pc.zero);
    const uint32_t m = g == 0 ? m0 : (g == 1 ? m1 : m2), msh = g == 0 ? ms0 : (g == 1 ? ms1 : ms2);
    uint32_t *dst = out + (size_t)i * 3 * 16 * T * 8 + (size_t)g * 16 * T * 8 + key_lane_word(tau) + 128 * h;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t x = csub(csub(v[k][q], 2 * p), p);
            dst[(size_t)q * T * 8 + k] = csub(mul_shoup(m, msh, x, p), p);
        }
    }
}

// ---------------------------------------------------------------- blind rotation, one PBS on three SMs
// For launches too small to fill the GPU (latency): a cluster of three CTAs
// per ciphertext, CTA g running prime g's transforms (the same per-thread work
// as one prime group of k_blind_rotate), so a CMux takes one third of the SM
// work.  Each CTA keeps its own copy of the accumulator; after the inverse
// transforms the residues are exchanged through distributed shared memory:
// CTA g reconstructs every third block of coefficients from the three CTAs'
// residues and writes the new values into all three accumulator copies.  The
// residues are written into the CTA's exchange buffer once its threads have read
// their last inverse exchange (two CTAs per SM fit).  Two
// cluster barriers per CMux (residues ready; accumulators updated).  All CTAs
// of a cluster run the same jobs and the same CMux sequence, so every CTA
// reaches every cluster barrier.
template <int LOGN>
struct BrClSmem {
    static constexpr int N = 1 << LOGN;
    static constexpr size_t acc_bytes = 2 * 2 * N * sizeof(uint64_t);
    static constexpr size_t buf_bytes = (size_t)ExWords<LOGN>::WORDS * 16;   // the residues reuse it
    static constexpr size_t total = acc_bytes + buf_bytes;
};

template <int LOGN>
__global__ void __cluster_dims__(3, 1, 1) __launch_bounds__((1 << LOGN) / 16, 2)
k_blind_rotate_cl(const Job *__restrict__ jobs, uint32_t njobs, const uint32_t *__restrict__ ms, uint32_t n,
                  const uint32_t *__restrict__ bsk, const uint2 *__restrict__ tw, const uint8_t *__restrict__ luts,
                  int lut_per_job, uint32_t base_log)
{
    namespace cg = cooperative_groups;
    using Lay = Layout<LOGN>;
    constexpr int N = Lay::N, T = Lay::T;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint64_t *acc = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *buf = reinterpret_cast<uint32_t *>(smem_raw + BrClSmem<LOGN>::acc_bytes);
    uint32_t *res = buf;   // this prime's residues [2][N], in the exchange buffer after the inverse

    const int g = (int)cl.block_rank();
    const uint32_t tau = threadIdx.x;
    const uint32_t p = c_pc.p[g];
    const uint2 *twf = tw + (size_t)(g * 2 + 0) * N;
    const uint2 *twi = tw + (size_t)(g * 2 + 1) * N;
    const uint32_t pmB = p - (1u << base_log);
    const size_t key_row = (size_t)3 * 16 * T * 8;
    const uint32_t *res_of[3];
    uint64_t *acc_of[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        res_of[r] = cl.map_shared_rank(res, r);
        acc_of[r] = cl.map_shared_rank(acc, r);
    }
    const uint32_t nclusters = gridDim.x / 3, cid = blockIdx.x / 3;

    for (uint32_t job = cid; job < njobs; job += nclusters) {
        const Job J = jobs[job];
        const uint32_t *msj = ms + (size_t)job * (n + 1);
        uint8_t f[16];
        {
            const uint8_t *lp = luts + (lut_per_job ? (size_t)job * 16 : (size_t)J.lut * 16);
            const uint4 lv = *reinterpret_cast<const uint4 *>(lp);
            memcpy(f, &lv, 16);
        }
        const uint32_t b = __ldg(msj + n);
        for (int t = tau; t < 2 * N; t += T) {
            acc[t] = 0;
            acc[2 * N + t] = test_poly_at<LOGN>(f, (t + b) & (2 * N - 1));
        }
        __syncthreads();
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t a = __ldg(msj + i);
            if (a == 0) continue;   // the same for the three CTAs
            uint32_t d[4][16];
            decompose<LOGN>(d, acc, a, tau, base_log, pmB);
            ext_product_core<LOGN, true>(d, bsk + (size_t)i * key_row + (size_t)g * 16 * T * 8, buf, res, tau, g,
                                         twf, twi);
            cl.sync();   // the three primes' residues are in place
            for (int c = g * T + (int)tau; c < 2 * N; c += 3 * T) {
                const int j = c >> LOGN, e = c & (N - 1);
                const uint64_t x = crt3(res_of[0][j * N + e], res_of[1][j * N + e], res_of[2][j * N + e], c_pc);
                const uint64_t y = acc[j * 2 * N + e] + x;
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    acc_of[r][j * 2 * N + e] = y;
                    acc_of[r][j * 2 * N + e + N] = 0 - y;
                }
            }
            cl.sync();   // every copy of the accumulator is updated; residues may be overwritten
        }
        if (g == 0) sample_extract_epilogue<LOGN, true>(J, acc, (int)tau, T);
        __syncthreads();
    }
}

// Product-only kernel (parity of the NTT/CRT path): out[item] = sum_r dig[r] * key[r][col]
template <int LOGN>
__global__ void __launch_bounds__(3 * (1 << LOGN) / 16, 1)
k_poly_mul(const int32_t *__restrict__ dig, const uint32_t *__restrict__ keyntt, uint64_t *__restrict__ out,
           uint32_t count, const uint2 *__restrict__ tw)
{
    using Lay = Layout<LOGN>;
    constexpr int N = Lay::N, T = Lay::T, NT = 3 * T;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint32_t *bufs = reinterpret_cast<uint32_t *>(smem_raw + BrSmem<LOGN, 0>::acc_bytes);
    uint32_t *crt = bufs + 3 * 4 * ExWords<LOGN>::WORDS;
    const int tid = threadIdx.x, g = tid / T;
    const uint32_t tau = tid % T;
    const uint32_t item = blockIdx.x;
    if (item >= count) return;
    const uint32_t p = c_pc.p[g];
    uint32_t d[4][16];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t e = tau | ((uint32_t)q << Lay::B0);
            const int32_t x = dig[((size_t)item * 4 + r) * N + e];
            d[r][q] = x < 0 ? (uint32_t)(x + (int32_t)p) : (uint32_t)x;
        }
    ext_product_core<LOGN>(d, keyntt + (size_t)item * 3 * 16 * T * 8 + (size_t)g * 16 * T * 8,
                           bufs + g * 4 * ExWords<LOGN>::WORDS, crt + g * 2 * N, tau, g, tw + (size_t)(g * 2) * N,
                           tw + (size_t)(g * 2 + 1) * N);
    __syncthreads();
    for (int c = tid; c < 2 * N; c += NT) {
        const int j = c >> LOGN, e = c & (N - 1);
        out[((size_t)item * 2 + j) * N + e] =
            crt3(crt[(0 * 2 + j) * N + e], crt[(1 * 2 + j) * N + e], crt[(2 * 2 + j) * N + e], c_pc);
    }
}

// ---------------------------------------------------------------- small helpers
__global__ void k_fill_trivial(uint64_t *arena, size_t stride, uint32_t big, size_t first, uint32_t count,
                               uint64_t body)
{
    const uint32_t s = blockIdx.x;
    if (s >= count) return;
    uint64_t *row = arena + (first + s) * stride;
    for (uint32_t u = threadIdx.x; u <= big; u += blockDim.x) row[u] = u == big ? body : 0;
}

}  // namespace dev

// ---------------------------------------------------------------- host wrappers
using namespace dev;

int br_threads(uint32_t N) { return 3 * (int)N / 16; }
int br_smem_bytes(uint32_t N) { return N == 2048 ? (int)BrSmem<11, 0>::total : (int)BrSmem<9, 0>::total; }
size_t bsk_ntt_words(uint32_t n, uint32_t N) { return (size_t)n * 3 * 16 * (N / 16) * 8; }

cudaError_t upload_prime_consts(const PrimeConsts &pc) { return cudaMemcpyToSymbol(c_pc, &pc, sizeof(pc)); }

template <int LOGN>
static cudaError_t set_attrs()
{
    cudaError_t e = cudaFuncSetAttribute(k_blind_rotate<LOGN, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BrSmem<LOGN, 0>::total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blind_rotate<LOGN, kKeyStageChunks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BrSmem<LOGN, kKeyStageChunks>::total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_poly_mul<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BrSmem<LOGN, 0>::total);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_blind_rotate_cl<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BrClSmem<LOGN>::total);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_bsk_to_ntt<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(3 * (size_t)ExWords<LOGN>::WORDS * 16));
}

template <int LOGN>
static int max_clusters()
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(3, 1, 1);
    cfg.blockDim = dim3((1 << LOGN) / 16, 1, 1);
    cfg.dynamicSmemBytes = BrClSmem<LOGN>::total;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 3;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_blind_rotate_cl<LOGN>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

int br_cluster_capacity(uint32_t N) { return N == 2048 ? max_clusters<11>() : max_clusters<9>(); }

cudaError_t prepare_kernels(uint32_t N) { return N == 2048 ? set_attrs<11>() : set_attrs<9>(); }

int br_blocks_per_sm(uint32_t N)
{
    int nb = 0;
    cudaError_t e = N == 2048
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blind_rotate<11, 0>, br_threads(N), BrSmem<11, 0>::total)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blind_rotate<9, 0>, br_threads(N), BrSmem<9, 0>::total);
    if (e != cudaSuccess) { cudaGetLastError(); return 1; }
    return nb;
}

cudaError_t launch_bsk_to_ntt_count(uint32_t N, const uint64_t *coef, uint32_t count, uint32_t *out,
                                    const uint32_t *tw, const uint32_t mont[3][2], cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    dim3 grid(count, 2);
    const uint2 *t2 = reinterpret_cast<const uint2 *>(tw);
    const size_t sm = 3 * (size_t)(N + N / 16) * 16;
    if (N == 2048)
        k_bsk_to_ntt<11><<<grid, br_threads(N), sm, s>>>(coef, count, out, t2, mont[0][0], mont[0][1], mont[1][0],
                                                          mont[1][1], mont[2][0], mont[2][1]);
    else
        k_bsk_to_ntt<9><<<grid, br_threads(N), sm, s>>>(coef, count, out, t2, mont[0][0], mont[0][1], mont[1][0],
                                                         mont[1][1], mont[2][0], mont[2][1]);
    return cudaGetLastError();
}

KsPlan ks_plan(const lvs_ctx *ctx, size_t njobs)
{
    const int b = ks_bucket(njobs);
    if (ctx->ks_tuned[b].tj) return ctx->ks_tuned[b];
    // default: 4 jobs per CTA for tiny launches, else 16; split the input
    // coefficients until about two CTAs per SM are busy
    KsPlan pl;
    pl.tj = njobs <= 4 ? 4 : 16;
    const size_t ctas = ((njobs + pl.tj - 1) / pl.tj) * ((ctx->P.p.n + KS_THREADS) / KS_THREADS);
    int split = 1;
    while (split < 32 && ctas * split * 2 <= (size_t)ctx->num_sms * 2) split *= 2;
    pl.split = split;
    return pl;
}

size_t ks_part_words(const lvs_ctx *ctx, size_t njobs)
{
    const KsPlan pl = ks_plan(ctx, njobs);
    return pl.split > 1 ? (size_t)pl.split * njobs * (ctx->P.p.n + 1) : 0;
}

cudaError_t launch_keyswitch_plan(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, uint64_t *part,
                                  KsPlan pl, cudaStream_t s)
{
    if (njobs == 0) return cudaSuccess;
    const auto &p = ctx->P.p;
    if (!part) pl.split = 1;
    const unsigned gy = (p.n + 1 + KS_THREADS - 1) / KS_THREADS;
    const uint32_t log2_2N = ctx->P.log_n() + 1;
    if (pl.tj == 4) {
        dim3 grid((unsigned)((njobs + 3) / 4), gy, (unsigned)pl.split);
        k_keyswitch<4><<<grid, KS_THREADS, 0, s>>>(jobs, (uint32_t)njobs, ctx->ksk, ctx->ksk_colsum, p.n,
                                                   ctx->P.big(), p.ks_level, p.ks_base_log, log2_2N, ms, part);
    } else {
        dim3 grid((unsigned)((njobs + 15) / 16), gy, (unsigned)pl.split);
        k_keyswitch<16><<<grid, KS_THREADS, 0, s>>>(jobs, (uint32_t)njobs, ctx->ksk, ctx->ksk_colsum, p.n,
                                                    ctx->P.big(), p.ks_level, p.ks_base_log, log2_2N, ms, part);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || pl.split == 1) return e;
    const size_t total = njobs * (size_t)(p.n + 1);
    k_ks_finish<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(jobs, (uint32_t)njobs, part, (uint32_t)pl.split,
                                                                 ctx->ksk_colsum, p.n, ctx->P.big(), p.ks_base_log,
                                                                 log2_2N, ms);
    return cudaGetLastError();
}

cudaError_t launch_keyswitch(const lvs_ctx *ctx, const Job *jobs, size_t njobs, uint32_t *ms, cudaStream_t s,
                             int *nlaunch)
{
    // the context's split-K scratch (sized by ensure_scratch), if any
    KsPlan pl = ks_plan(ctx, njobs);
    if (!ctx->ks_part || ctx->ks_part_cap < ks_part_words(ctx, njobs)) pl.split = 1;
    if (nlaunch) *nlaunch = njobs == 0 ? 0 : (pl.split > 1 ? 2 : 1);
    return launch_keyswitch_plan(ctx, jobs, njobs, ms, ctx->ks_part, pl, s);
}

cudaError_t launch_blind_rotate(const lvs_ctx *ctx, const Job *jobs, size_t njobs, const uint32_t *ms,
                                const uint8_t *luts, int lut_per_job, cudaStream_t s)
{
    if (njobs == 0) return cudaSuccess;
    const auto &p = ctx->P.p;
    const uint2 *t2 = reinterpret_cast<const uint2 *>(ctx->tw);
    if (njobs <= ctx->br_split_max && ctx->br_clusters > 0) {
        // small launch: one ciphertext per cluster of three CTAs (one per prime)
        const unsigned grid = 3 * (unsigned)std::min<size_t>(njobs, (size_t)ctx->br_clusters);
        if (p.N == 2048)
            k_blind_rotate_cl<11><<<grid, (1 << 11) / 16, BrClSmem<11>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log);
        else
            k_blind_rotate_cl<9><<<grid, (1 << 9) / 16, BrClSmem<9>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log);
        return cudaGetLastError();
    }
    const unsigned grid = (unsigned)std::min<size_t>(njobs, (size_t)ctx->br_grid);
    const uint32_t drop = ctx->debug_drop_key_copy ? 1u : 0u;
    constexpr int KS = kKeyStageChunks;
    if (p.N == 2048) {
        if (ctx->key_staging)
            k_blind_rotate<11, KS><<<grid, br_threads(p.N), BrSmem<11, KS>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log, ctx->fault_dev, drop);
        else
            k_blind_rotate<11, 0><<<grid, br_threads(p.N), BrSmem<11, 0>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log, ctx->fault_dev, 0u);
    } else {
        if (ctx->key_staging)
            k_blind_rotate<9, KS><<<grid, br_threads(p.N), BrSmem<9, KS>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log, ctx->fault_dev, drop);
        else
            k_blind_rotate<9, 0><<<grid, br_threads(p.N), BrSmem<9, 0>::total, s>>>(
                jobs, (uint32_t)njobs, ms, p.n, ctx->bsk_ntt, t2, luts, lut_per_job, p.pbs_base_log, ctx->fault_dev, 0u);
    }
    return cudaGetLastError();
}

cudaError_t launch_ksk_colsum(const lvs_ctx *ctx, cudaStream_t s)
{
    const auto &p = ctx->P.p;
    const uint32_t rows = ctx->P.big() * p.ks_level;
    k_ksk_colsum<<<(p.n + 1 + 127) / 128, 128, 0, s>>>(ctx->ksk, rows, p.n, ctx->ksk_colsum);
    return cudaGetLastError();
}

cudaError_t launch_poly_mul(const lvs_ctx *ctx, const int32_t *dig, const uint32_t *keyntt, uint64_t *out,
                            size_t count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    const uint32_t N = ctx->P.p.N;
    const uint2 *t2 = reinterpret_cast<const uint2 *>(ctx->tw);
    if (N == 2048)
        k_poly_mul<11><<<(unsigned)count, br_threads(N), BrSmem<11, 0>::total, s>>>(dig, keyntt, out, (uint32_t)count, t2);
    else
        k_poly_mul<9><<<(unsigned)count, br_threads(N), BrSmem<9, 0>::total, s>>>(dig, keyntt, out, (uint32_t)count, t2);
    return cudaGetLastError();
}

cudaError_t launch_fill_trivial(uint64_t *arena, size_t stride, uint32_t big, size_t first, size_t count,
                                uint64_t body, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_fill_trivial<<<(unsigned)count, 256, 0, s>>>(arena, stride, big, first, (uint32_t)count, body);
    return cudaGetLastError();
}

}  // namespace lvs
