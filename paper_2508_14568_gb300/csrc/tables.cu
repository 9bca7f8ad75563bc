// Host-side constant tables: NTT twiddles, prime constants for Montgomery /
// Shoup / Garner arithmetic, and the three lookup tables of the method.
#include <algorithm>
#include <vector>

#include "lvs_internal.hpp"
#include "ntt.cuh"

namespace lvs {

static uint32_t mulmod(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }

static uint32_t powmod(uint32_t a, uint64_t e, uint32_t p)
{
    uint32_t r = 1 % p;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod(r, a, p);
        a = mulmod(a, a, p);
        e >>= 1;
    }
    return r;
}

static uint32_t invmod(uint32_t a, uint32_t p) { return powmod(a, p - 2, p); }

static uint32_t shoup_of(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

// smallest generator of Z_p^*
static uint32_t primitive_root(uint32_t p)
{
    std::vector<uint32_t> f;
    uint32_t m = p - 1;
    for (uint32_t q = 2; (uint64_t)q * q <= m; ++q)
        if (m % q == 0) {
            f.push_back(q);
            while (m % q == 0) m /= q;
        }
    if (m > 1) f.push_back(m);
    for (uint32_t g = 2;; ++g) {
        bool ok = true;
        for (uint32_t q : f)
            if (powmod(g, (p - 1) / q, p) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

static uint32_t bit_reverse(uint32_t x, uint32_t bits)
{
    uint32_t r = 0;
    for (uint32_t b = 0; b < bits; ++b) r |= ((x >> b) & 1u) << (bits - 1 - b);
    return r;
}

// uint2 {w, shoup(w)} laid out [prime][0 = forward, 1 = inverse][N]:
// forward w[k] = psi^{bitrev(k)}, psi a primitive 2N-th root of unity;
// inverse w[k] = forward w[k]^{-1}.
void make_twiddles(uint32_t N, std::vector<uint32_t> &out)
{
    uint32_t logn = 0;
    while ((1u << logn) < N) ++logn;
    out.assign((size_t)kPrimes * 2 * N * 2, 0);
    for (int g = 0; g < kPrimes; ++g) {
        const uint32_t p = kPrime[g];
        const uint32_t psi = powmod(primitive_root(p), (p - 1) / (2 * N), p);
        for (uint32_t k = 0; k < N; ++k) {
            const uint32_t w = powmod(psi, bit_reverse(k, logn), p);
            const uint32_t wi = invmod(w, p);
            uint32_t *f = &out[(((size_t)g * 2 + 0) * N + k) * 2];
            uint32_t *i = &out[(((size_t)g * 2 + 1) * N + k) * 2];
            f[0] = w;
            f[1] = shoup_of(w, p);
            i[0] = wi;
            i[1] = shoup_of(wi, p);
        }
    }
}

void make_prime_consts(dev::PrimeConsts &pc)
{
    pc = dev::PrimeConsts{};
    for (int g = 0; g < kPrimes; ++g) {
        const uint32_t p = kPrime[g];
        pc.p[g] = p;
        uint32_t inv = 1;                        // p^{-1} mod 2^32 by Newton iteration
        for (int it = 0; it < 5; ++it) inv *= 2 - p * inv;
        pc.pinv_neg[g] = 0u - inv;
        const uint32_t R = (uint32_t)((1ull << 32) % p);
        pc.r2[g] = mulmod(R, R, p);
    }
    const uint32_t p0 = kPrime[0], p1 = kPrime[1], p2 = kPrime[2];
    pc.c01 = invmod(p0 % p1, p1);
    pc.c01_sh = shoup_of(pc.c01, p1);
    pc.p0m2 = p0 % p2;
    pc.p0m2_sh = shoup_of(pc.p0m2, p2);
    pc.c012 = invmod(mulmod(p0 % p2, p1 % p2, p2), p2);
    pc.c012_sh = shoup_of(pc.c012, p2);
    pc.p01 = (uint64_t)p0 * p1;
    pc.m64 = pc.p01 * p2;
    pc.half2 = p2 >> 1;
    pc.zero = 0;
}

// R * N^{-1} mod p with R = 2^32, and its Shoup companion: the key is stored
// multiplied by this so that Montgomery products need no further scaling and
// the inverse transform needs no 1/N.
void make_mont(uint32_t N, uint32_t mont[3][2])
{
    for (int g = 0; g < kPrimes; ++g) {
        const uint32_t p = kPrime[g];
        const uint32_t R = (uint32_t)((1ull << 32) % p);
        const uint32_t m = mulmod(R, invmod(N % p, p), p);
        mont[g][0] = m;
        mont[g][1] = shoup_of(m, p);
    }
}

// LUT table [256][16] (values in Z_32):
//   LUT_EQ : 1 at 0, else 0                  (Eq. eq_eqlut)
//   LUT_EQ9: 9 at 0, else 0                  (Eq. eq_eqlut9)
//   LUT_MIN: M = 1 + min(-eq, dv, dh) as a function of the key
//            (1 - dv) + 3 (1 + dh) + 9 eq of Eq. eq_keyeq2; keys 16 and 17 fall
//            in the negacyclic half and need M = 0 there and at keys 0, 1.
//   LUT_V  : dv_out = M - dh_in as a function of the same key (refreshed
//            cells, Section 3.1.3); keys 16, 17 give -1 = -(value at 0, 1),
//            so the negacyclic half holds.  With dv_in and dh_in exchanged in
//            the key the same table gives dh_out (M is symmetric).
void make_luts(std::vector<uint8_t> &t)
{
    t.assign(256 * 16, 0);
    t[LUT_EQ * 16 + 0] = 1;
    t[LUT_EQ9 * 16 + 0] = 9;
    for (int eq = 0; eq <= 1; ++eq)
        for (int dh = -1; dh <= 1; ++dh)
            for (int dv = -1; dv <= 1; ++dv) {
                const int key = (1 - dv) + 3 * (1 + dh) + 9 * eq;
                const int M = 1 + std::min(std::min(-eq, dv), dh);
                if (key < 16) {
                    t[LUT_MIN * 16 + key] = (uint8_t)M;
                    t[LUT_V * 16 + key] = (uint8_t)((M - dh + 32) % 32);   // dv_out = M - dh_in
                }
            }
}

}  // namespace lvs
