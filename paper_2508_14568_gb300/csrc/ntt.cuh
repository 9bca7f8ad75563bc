// Device arithmetic of the exact negacyclic product mod 2^64 used by the
// blind rotation (the external product GGSW [x] GLWE of TFHE, Section 2.2 of
// the paper defers to the standard TFHE construction).
//
// The integer product of a digit polynomial (|d| <= B/2) and a key polynomial
// (signed 64-bit) has coefficients below 2^88 in magnitude, so it is computed
// exactly modulo three 30-bit NTT primes and rebuilt by CRT (Garner), then
// reduced mod 2^64.  Per prime: merged negacyclic number-theoretic transform
// (Cooley-Tukey forward, natural order in / bit-reversed out; Gentleman-Sande
// inverse), with Harvey's lazy butterflies (values kept in [0, 4p)) and
// Shoup's precomputed-quotient modular multiplication by constants;
// Montgomery reduction (R = 2^32) for the key product, whose key operand is
// stored pre-multiplied by R * N^{-1} so the inverse transform needs no scaling.
//
// Register layout: a prime group of T = N/8 threads holds 8 coefficients per
// thread of up to four polynomials.  An N = 2^L point transform runs as
// ceil(L/3) register passes of <= 3 radix-2 stages.  In pass k the register
// index q (3 bits) sits at position bits [R, R + 3), R = max(L - 3 - 3k, 0),
// and the thread index tau fills the other bits in order:
//   e = (tau >> R) << (R + 3) | q << R | (tau & (2^R - 1)).
// Pass 0 (R = L - 3) is e = q << (L - 3) | tau (coefficient order of the
// accumulator); the last pass (R = 0) is e = tau << 3 | q.  The warp index
// (tau >> 5) lands on position bits >= 8 in every pass but the first, so only
// the exchange between pass 0 and pass 1 crosses warps (group barrier); the
// others stay inside a warp.  The four forward polynomials of a position
// travel as one 16-byte shared-memory word at swz16(e) = e ^ ((e >> 3) & 7),
// the two inverse polynomials as one 8-byte word at idx8(e) (same per-warp
// byte region as the 16-byte view); both are bank-conflict free in every
// layout (each quarter-warp, resp. half-warp, of one store instruction lands
// on distinct banks).
#pragma once
#include <cstdint>

namespace lvs {
namespace dev {

struct PrimeConsts {
    uint32_t p[3];
    uint32_t pinv_neg[3];      // -p^{-1} mod 2^32
    uint32_t mont[3];          // R * N^{-1} mod p (for key conversion)
    uint32_t mont_sh[3];       // Shoup companion of mont
    uint32_t r2[3];            // R^2 mod p (unused by the hot path)
    // Garner: x = v0 + p0 v1 + p0 p1 v2
    uint32_t c01, c01_sh;      // p0^{-1} mod p1
    uint32_t p0m2, p0m2_sh;    // p0 mod p2
    uint32_t c012, c012_sh;    // (p0 p1)^{-1} mod p2
    uint64_t p01;              // p0 p1 mod 2^64
    uint64_t m64;              // p0 p1 p2 mod 2^64
    uint32_t half2;            // p2 >> 1
};

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m)
{
    // x in [0, 2m) -> [0, m)
    return min(x, x - m);
}

// w * x mod p in [0, 2p) for any x < 2^32 (Shoup)
__device__ __forceinline__ uint32_t mul_shoup(uint32_t w, uint32_t wsh, uint32_t x, uint32_t p)
{
    const uint32_t q = __umulhi(wsh, x);
    return w * x - q * p;
}

// Montgomery reduction: T * 2^-32 mod p, below p + T / 2^32 (so in [0, 2p) for
// T < p * 2^32); T + m p must not overflow 64 bits
__device__ __forceinline__ uint32_t redc(uint64_t T, uint32_t p, uint32_t pinv_neg)
{
    const uint32_t m = (uint32_t)T * pinv_neg;
    return (uint32_t)((T + (uint64_t)m * p) >> 32);
}

// value barrier: the compiler may not re-associate through it
__device__ __forceinline__ uint32_t opaque(uint32_t x)
{
    asm("" : "+r"(x));
    return x;
}

__device__ __forceinline__ void group_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Geometry of the register passes of an N = 2^L transform.
template <int L>
struct Geo {
    static constexpr int N = 1 << L;
    static constexpr int T = N / 8;                  // threads per prime group
    static constexpr int PASSES = (L + 2) / 3;
    static constexpr int R(int k) { return L - 3 - 3 * k > 0 ? L - 3 - 3 * k : 0; }
    static constexpr int CNT(int k) { return L - 3 * k < 3 ? L - 3 * k : 3; }
};

// thread part of the position in the layout whose register field starts at bit R
template <int L, int R>
__device__ __forceinline__ uint32_t pass_base(uint32_t tau)
{
    if (R == L - 3) return tau;   // pass 0: tau < 2^(L-3)
    return ((tau >> R) << (R + 3)) | (tau & ((1u << R) - 1u));
}

// 16-byte words: e ^ ((e >> 3) & 7).  8-byte words: the same per-warp byte
// region as the 16-byte view (in the warp-local layouts warp w owns positions
// e >> 8 == w, i.e. 16-byte words [256 w, 256 w + 256)), swizzled by
// e ^ ((e >> 3) & 15) inside it.  Both maps are linear over GF(2), and base
// and q << R occupy disjoint bits, so swz(base | q << R) = swz(base) ^
// swz(q << R): the callers pass the thread part once and the register part is
// a compile-time constant.
__host__ __device__ __forceinline__ constexpr uint32_t swz16(uint32_t e) { return e ^ ((e >> 3) & 7u); }
__host__ __device__ __forceinline__ constexpr uint32_t idx8(uint32_t e)
{
    return ((e >> 8) << 9) | ((e ^ ((e >> 3) & 15u)) & 255u);
}

// One register pass of forward (Cooley-Tukey) stages S0 .. S0+CNT-1 on NP
// polynomials that share positions (and hence twiddles).  FRESH: the inputs of
// the first stage are below 2p, so its lazy reduction is skipped (outputs stay
// below 4p).  Stage s pairs positions e and e + 2^(L-1-s), twiddle index
// 2^s + (e >> (L - s)).
template <int L, int R, int S0, int CNT, int NP, int NPA, bool FRESH = false>
__device__ __forceinline__ void fwd_pass(uint32_t (&v)[NPA][8], uint32_t base, const uint2 *__restrict__ tw,
                                         uint32_t p)
{
    const uint32_t p2 = 2 * p;
#pragma unroll
    for (int si = 0; si < CNT; ++si) {
        const int s = S0 + si;
        const int rb = L - 1 - s - R;   // register bit of this stage's span
#pragma unroll
        for (int g = 0; g < (1 << (2 - rb)); ++g) {
            const uint32_t hi = (uint32_t)(g << (rb + 1)) << R;
            const uint32_t pos = (R == L - 3) ? hi : (base | hi);   // pass 0: thread bits are shifted out
            const uint2 w = __ldg(tw + (1u << s) + (pos >> (L - s)));
#pragma unroll
            for (int low = 0; low < (1 << rb); ++low) {
                const int q0 = (g << (rb + 1)) | low, q1 = q0 | (1 << rb);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const uint32_t x = (FRESH && si == 0) ? v[k][q0] : csub(v[k][q0], p2);
                    const uint32_t t = opaque(mul_shoup(w.x, w.y, v[k][q1], p));
                    v[k][q0] = x + t;
                    v[k][q1] = x - t + p2;
                }
            }
        }
    }
}

// One register pass of inverse (Gentleman-Sande) stages S0+CNT-1 .. S0 on the
// first NP polynomials; values stay in [0, 2p).
template <int L, int R, int S0, int CNT, int NP, int NPA>
__device__ __forceinline__ void inv_pass(uint32_t (&v)[NPA][8], uint32_t base, const uint2 *__restrict__ tw,
                                         uint32_t p)
{
    const uint32_t p2 = 2 * p;
#pragma unroll
    for (int si = CNT - 1; si >= 0; --si) {
        const int s = S0 + si;
        const int rb = L - 1 - s - R;
#pragma unroll
        for (int g = 0; g < (1 << (2 - rb)); ++g) {
            const uint32_t hi = (uint32_t)(g << (rb + 1)) << R;
            const uint32_t pos = (R == L - 3) ? hi : (base | hi);
            const uint2 w = __ldg(tw + (1u << s) + (pos >> (L - s)));
#pragma unroll
            for (int low = 0; low < (1 << rb); ++low) {
                const int q0 = (g << (rb + 1)) | low, q1 = q0 | (1 << rb);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const uint32_t x = v[k][q0], y = v[k][q1];
                    v[k][q0] = csub(x + y, p2);
                    v[k][q1] = opaque(mul_shoup(w.x, w.y, x - y + p2, p));
                }
            }
        }
    }
}

// shared-memory exchange of the thread's 8 positions (layout R, thread part sb
// already swizzled): 4 polynomials per 16-byte word, 2 per 8-byte word
template <int R, int NPA>
__device__ __forceinline__ void st16(uint4 *buf, const uint32_t (&v)[NPA][8], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[sb ^ swz16((uint32_t)q << R)] = make_uint4(v[0][q], v[1][q], v[2][q], v[3][q]);
}

template <int R, int NPA>
__device__ __forceinline__ void ld16(const uint4 *buf, uint32_t (&v)[NPA][8], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 w = buf[sb ^ swz16((uint32_t)q << R)];
        v[0][q] = w.x; v[1][q] = w.y; v[2][q] = w.z; v[3][q] = w.w;
    }
}

template <int R, int NPA>
__device__ __forceinline__ void st8(uint2 *buf, const uint32_t (&v)[NPA][8], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) buf[sb ^ idx8((uint32_t)q << R)] = make_uint2(v[0][q], v[1][q]);
}

template <int R, int NPA>
__device__ __forceinline__ void ld8(const uint2 *buf, uint32_t (&v)[NPA][8], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint2 w = buf[sb ^ idx8((uint32_t)q << R)];
        v[0][q] = w.x; v[1][q] = w.y;
    }
}

// Passes 1 .. PASSES-1 of the forward transform (the caller has stored pass
// 0's output and passed the group barrier).
template <int L, int K>
__device__ __forceinline__ void fwd_tail(uint32_t (&v)[4][8], uint4 *buf, uint32_t tau, const uint2 *__restrict__ tw,
                                         uint32_t p)
{
    using G = Geo<L>;
    constexpr int R = G::R(K);
    const uint32_t b = pass_base<L, R>(tau);
    const uint32_t sb = swz16(b);
    ld16<R, 4>(buf, v, sb);
    fwd_pass<L, R, 3 * K, G::CNT(K), 4, 4>(v, b, tw, p);
    if constexpr (K + 1 < G::PASSES) {
        __syncwarp();
        st16<R, 4>(buf, v, sb);
        __syncwarp();
        fwd_tail<L, K + 1>(v, buf, tau, tw, p);
    }
}

// Full forward transform of the 4 polynomials held in the pass-0 layout
// (values in [0, 2p)); returns them in the last layout (bit-reversed
// evaluation order, e = tau << 3 | q), values in [0, 4p).
// buf: N 16-byte words of this group's shared memory.  bar_id / T: group barrier.
template <int L>
__device__ __forceinline__ void ntt_forward4(uint32_t (&v)[4][8], uint4 *buf, uint32_t tau,
                                             const uint2 *__restrict__ tw, uint32_t p, int bar_id)
{
    using G = Geo<L>;
    fwd_pass<L, L - 3, 0, 3, 4, 4, true>(v, tau, tw, p);
    st16<L - 3, 4>(buf, v, swz16(tau));
    if (G::T > 32) group_bar(bar_id, G::T); else __syncwarp();
    fwd_tail<L, 1>(v, buf, tau, tw, p);
}

// Inverse passes K .. 0 of the first 2 polynomials, starting in layout K.
template <int L, int K>
__device__ __forceinline__ void inv_from(uint32_t (&v)[4][8], uint2 *buf, uint32_t tau, const uint2 *__restrict__ tw,
                                         uint32_t p, int bar_id)
{
    using G = Geo<L>;
    constexpr int R = G::R(K);
    const uint32_t b = pass_base<L, R>(tau);
    inv_pass<L, R, 3 * K, G::CNT(K), 2, 4>(v, b, tw, p);
    if constexpr (K > 0) {
        constexpr int R1 = G::R(K - 1);
        const uint32_t b1 = pass_base<L, R1>(tau);
        __syncwarp();
        st8<R, 4>(buf, v, idx8(b));
        if (K == 1) {
            if (G::T > 32) group_bar(bar_id, G::T); else __syncwarp();
        } else {
            __syncwarp();
        }
        ld8<R1, 4>(buf, v, idx8(b1));
        inv_from<L, K - 1>(v, buf, tau, tw, p, bar_id);
    }
}

// Inverse transform of the first 2 polynomials of v, held in the last layout
// (values in [0, 2p)); returns them in the pass-0 layout (natural order),
// values in [0, 2p), NOT scaled by N^{-1}.
template <int L>
__device__ __forceinline__ void ntt_inverse2(uint32_t (&v)[4][8], uint2 *buf, uint32_t tau,
                                             const uint2 *__restrict__ tw, uint32_t p, int bar_id)
{
    inv_from<L, Geo<L>::PASSES - 1>(v, buf, tau, tw, p, bar_id);
}

// Garner reconstruction of the signed integer with residues r0, r1, r2
// (each in [0, p_i)), returned mod 2^64.  Valid for |x| < p0 p1 p2 / 2.
__device__ __forceinline__ uint64_t crt3(uint32_t r0, uint32_t r1, uint32_t r2, const PrimeConsts &C)
{
    const uint32_t p0 = C.p[0], p1 = C.p[1], p2 = C.p[2];
    // v1 = (r1 - r0) * p0^{-1} mod p1
    const uint32_t r0m1 = csub(r0, p1);                    // r0 < p0 < 2 p1
    const uint32_t v1 = csub(mul_shoup(C.c01, C.c01_sh, r1 + p1 - r0m1, p1), p1);
    // v2 = (r2 - (r0 + p0 v1)) * (p0 p1)^{-1} mod p2
    const uint32_t a = csub(mul_shoup(C.p0m2, C.p0m2_sh, v1, p2), p2);
    const uint32_t b = csub(csub(r0, p2) + a, p2);
    const uint32_t v2 = csub(mul_shoup(C.c012, C.c012_sh, r2 + p2 - b, p2), p2);
    uint64_t x = (uint64_t)r0 + (uint64_t)p0 * v1 + C.p01 * (uint64_t)v2;
    if (v2 > C.half2) x -= C.m64;
    return x;
}

}  // namespace dev
}  // namespace lvs
