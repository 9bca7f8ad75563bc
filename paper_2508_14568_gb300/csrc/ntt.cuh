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
// Register layout: a prime group of T = N/16 threads holds 16 coefficients per
// thread of several polynomials.  An N-point transform runs as three register
// passes of <= 4 radix-2 stages:
//   L0: e = tau | q << (logN-4)           stages 0..3
//   L1: e = hi << (logN-4) | q << (logN-8) | lo,   tau = hi << (logN-8) | lo
//                                          stages 4..7
//   L2: e = tau << 4 | q                   stages 8..logN-1
// with shared-memory exchanges between passes.  The four forward polynomials
// of a position travel as one 16-byte word (two inverse polynomials as one
// 8-byte word), stored at the swizzled index e ^ ((e >> 4) & 7) (16 B) or
// e ^ ((e >> 4) & 15) (8 B), which is bank-conflict free for all three
// layouts.  L1 <-> L2 exchanges stay inside a warp; L0 <-> L1 needs the group
// barrier.
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
    uint32_t zero;             // 0, read at run time (see fwd_pass)
};

__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m)
{
    // x in [0, 2m) -> [0, m)
    return min(x, x - m);
}

// csub with a zero the compiler cannot see: x - m + z is a three-input add,
// and the whole reduction becomes one fused add-and-minimum on the integer ALU
// (with x - m alone the compiler may form the difference on the multiply pipe)
__device__ __forceinline__ uint32_t csubz(uint32_t x, uint32_t m, uint32_t z) { return min(x, x - m + z); }

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

// value barrier: the compiler may not see through it
__device__ __forceinline__ uint32_t opaque(uint32_t x)
{
    asm("" : "+r"(x));
    return x;
}

__device__ __forceinline__ void group_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int LOGN>
struct Layout {
    static constexpr int N = 1 << LOGN;
    static constexpr int T = N / 16;
    static constexpr int B0 = LOGN - 4;   // L0 register stride exponent
    static constexpr int B1 = LOGN - 8;   // L1 register stride exponent
    static constexpr int S2 = LOGN - 8;   // stages in the last pass
    __device__ static __forceinline__ uint32_t base0(uint32_t tau) { return tau; }
    __device__ static __forceinline__ uint32_t base1(uint32_t tau)
    {
        return ((tau >> B1) << (B1 + 4)) | (tau & ((1u << B1) - 1u));
    }
    __device__ static __forceinline__ uint32_t base2(uint32_t tau) { return tau << 4; }
};

// Position of register q (= qg << B) of the thread with base `base`, as far as
// the twiddle index of stages s <= 3 needs it: in the L0 layout (B = LOGN - 4)
// the thread bits lie below bit LOGN - 4 and are shifted out by
// e >> (LOGN - s), so the index is the same for every thread (a compile-time
// constant, one broadcast load).
template <int LOGN, int B>
__device__ __forceinline__ uint32_t tw_pos(uint32_t base, int qg)
{
    return (B == LOGN - 4) ? ((uint32_t)qg << B) : (base | ((uint32_t)qg << B));
}

// One register pass of forward (Cooley-Tukey) stages s0 .. s0+cnt-1 on NP
// polynomials that share positions (and hence twiddles).  FRESH: the inputs of
// the first stage are below 2p, so its lazy reduction can be skipped (outputs
// stay below 4p).
// z: a zero the compiler cannot see (from constant memory): adding it makes
// every butterfly addition three-input, which keeps it on the integer ALU pipe
// instead of letting the compiler fold it into the multiply-add pipe that the
// Shoup products already saturate.
template <int LOGN, int B, int S0, int CNT, int NP, int NPA, bool FRESH = false>
__device__ __forceinline__ void fwd_pass(uint32_t (&v)[NPA][16], uint32_t base, const uint2 *__restrict__ tw,
                                         uint32_t p, uint32_t z)
{
    const uint32_t p2 = 2 * p, p2z = p2 + z;
#pragma unroll
    for (int si = 0; si < CNT; ++si) {
        const int s = S0 + si;
        const int rb = LOGN - s - 1 - B;
#pragma unroll
        for (int g = 0; g < (1 << (3 - rb)); ++g) {
            const uint2 w = __ldg(tw + (1u << s) + (tw_pos<LOGN, B>(base, g << (rb + 1)) >> (LOGN - s)));
#pragma unroll
            for (int low = 0; low < (1 << rb); ++low) {
                const int q0 = (g << (rb + 1)) | low, q1 = q0 | (1 << rb);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const uint32_t x = (FRESH && si == 0) ? v[k][q0] : csubz(v[k][q0], p2, z);
                    const uint32_t t = opaque(mul_shoup(w.x, w.y, v[k][q1], p));
                    v[k][q0] = x + t + z;
                    v[k][q1] = x + p2z - t;
                }
            }
        }
    }
}

// One register pass of inverse (Gentleman-Sande) stages s0+cnt-1 .. s0.
template <int LOGN, int B, int S0, int CNT, int NP, int NPA>
__device__ __forceinline__ void inv_pass(uint32_t (&v)[NPA][16], uint32_t base, const uint2 *__restrict__ tw,
                                         uint32_t p, uint32_t z)
{
    const uint32_t p2 = 2 * p, p2z = p2 + z;
#pragma unroll
    for (int si = CNT - 1; si >= 0; --si) {
        const int s = S0 + si;
        const int rb = LOGN - s - 1 - B;
#pragma unroll
        for (int g = 0; g < (1 << (3 - rb)); ++g) {
            const uint2 w = __ldg(tw + (1u << s) + (tw_pos<LOGN, B>(base, g << (rb + 1)) >> (LOGN - s)));
#pragma unroll
            for (int low = 0; low < (1 << rb); ++low) {
                const int q0 = (g << (rb + 1)) | low, q1 = q0 | (1 << rb);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    const uint32_t x = v[k][q0], y = v[k][q1];
                    const uint32_t s2 = x + y + z;
                    v[k][q0] = csubz(s2, p2, z);
                    v[k][q1] = opaque(mul_shoup(w.x, w.y, x + p2z - y, p));
                }
            }
        }
    }
}

// Shared-memory word of position e.  16-byte words (four forward polynomials):
// w16(e) = e + (e >> 4), one padding word after every 16.  8-byte words (two
// inverse polynomials): the same per-warp byte region as the 16-byte view (in
// the L1 / L2 layouts warp w owns positions e >> 9 == w, i.e. 16-byte words
// [544 w, 544 w + 544)): w8(e) = 1088 (e >> 9) + e' + (e' >> 4), e' = e & 511.
// Both are bank-conflict free in the three layouts (the eight lanes of each
// quarter-warp, resp. sixteen of each half-warp, of one access land on
// distinct banks) and additive over disjoint bit fields: w(base | q << B) =
// w(base) + w(q << B), so an access is the thread's base word plus a
// compile-time offset that folds into the instruction's immediate.
template <int LOGN>
struct ExWords {
    static constexpr int N = 1 << LOGN;
    static constexpr int WORDS = N + N / 16;   // 16-byte words per prime group
};
__device__ __forceinline__ constexpr uint32_t w16(uint32_t e) { return e + (e >> 4); }
template <int LOGN>
__device__ __forceinline__ constexpr uint32_t w8(uint32_t e)
{
    return LOGN > 9 ? 1088u * (e >> 9) + (e & 511u) + ((e & 511u) >> 4) : e + (e >> 4);
}

// store / load the polynomials of a thread in layout (B, base): 4 polynomials
// per 16-byte word (forward) or 2 per 8-byte word (inverse); sb = the base's word
template <int B, int NPA>
__device__ __forceinline__ void st4(uint4 *buf, const uint32_t (&v)[NPA][16], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[sb + w16((uint32_t)q << B)] = make_uint4(v[0][q], v[1][q], v[2][q], v[3][q]);
}

template <int B, int NPA>
__device__ __forceinline__ void ld4(const uint4 *buf, uint32_t (&v)[NPA][16], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint4 w = buf[sb + w16((uint32_t)q << B)];
        v[0][q] = w.x; v[1][q] = w.y; v[2][q] = w.z; v[3][q] = w.w;
    }
}

template <int LOGN, int B, int NPA>
__device__ __forceinline__ void st2(uint2 *buf, const uint32_t (&v)[NPA][16], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 16; ++q) buf[sb + w8<LOGN>((uint32_t)q << B)] = make_uint2(v[0][q], v[1][q]);
}

template <int LOGN, int B, int NPA>
__device__ __forceinline__ void ld2(const uint2 *buf, uint32_t (&v)[NPA][16], uint32_t sb)
{
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint2 w = buf[sb + w8<LOGN>((uint32_t)q << B)];
        v[0][q] = w.x; v[1][q] = w.y;
    }
}

// Full forward transform of the 4 polynomials held in L0 layout (values in
// [0, 2p)); returns them in L2 layout (bit-reversed evaluation order), values
// in [0, 4p).
// buf: ExWords<LOGN>::WORDS 16-byte words of this group's shared memory.  bar_id: group barrier.
template <int LOGN>
__device__ __forceinline__ void ntt_forward4(uint32_t (&v)[4][16], uint4 *buf, uint32_t tau,
                                             const uint2 *__restrict__ tw, uint32_t p, int bar_id, uint32_t z)
{
    using Lay = Layout<LOGN>;
    fwd_pass<LOGN, Lay::B0, 0, 4, 4, 4, true>(v, Lay::base0(tau), tw, p, z);
    __syncwarp();
    st4<Lay::B0, 4>(buf, v, w16(Lay::base0(tau)));
    if (Lay::T > 32) group_bar(bar_id, Lay::T); else __syncwarp();
    const uint32_t sb1 = w16(Lay::base1(tau));
    ld4<Lay::B1, 4>(buf, v, sb1);
    fwd_pass<LOGN, Lay::B1, 4, 4, 4, 4>(v, Lay::base1(tau), tw, p, z);
    __syncwarp();
    st4<Lay::B1, 4>(buf, v, sb1);
    __syncwarp();
    ld4<0, 4>(buf, v, w16(Lay::base2(tau)));
    fwd_pass<LOGN, 0, 8, Lay::S2, 4, 4>(v, Lay::base2(tau), tw, p, z);
}

// Inverse transform of the first 2 polynomials of v, held in L2 layout (values
// in [0, 2p)); returns them in L0 layout (natural order), values in [0, 2p),
// NOT scaled by N^{-1}.
template <int LOGN>
__device__ __forceinline__ void ntt_inverse2(uint32_t (&v)[4][16], uint2 *buf, uint32_t tau,
                                             const uint2 *__restrict__ tw, uint32_t p, int bar_id, uint32_t z)
{
    using Lay = Layout<LOGN>;
    inv_pass<LOGN, 0, 8, Lay::S2, 2, 4>(v, Lay::base2(tau), tw, p, z);
    __syncwarp();
    st2<LOGN, 0, 4>(buf, v, w8<LOGN>(Lay::base2(tau)));
    __syncwarp();
    const uint32_t sb1 = w8<LOGN>(Lay::base1(tau));
    ld2<LOGN, Lay::B1, 4>(buf, v, sb1);
    inv_pass<LOGN, Lay::B1, 4, 4, 2, 4>(v, Lay::base1(tau), tw, p, z);
    __syncwarp();
    st2<LOGN, Lay::B1, 4>(buf, v, sb1);
    if (Lay::T > 32) group_bar(bar_id, Lay::T); else __syncwarp();
    ld2<LOGN, Lay::B0, 4>(buf, v, w8<LOGN>(Lay::base0(tau)));
    inv_pass<LOGN, Lay::B0, 0, 4, 2, 4>(v, Lay::base0(tau), tw, p, z);
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
