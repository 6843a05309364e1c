// Device-side primitives shared by the generator kernels: the Philox4x32-10
// counter RNG, 64-bit uniform draws and division by run-time invariant
// divisors. Everything here is integer arithmetic; nothing depends on the
// launch schedule.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pgen {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each
// multiplying words 0 and 2 by the Philox constants (32x32 -> 64), XORing
// the high halves into the other two words together with the round key.
// The round keys (the seed key advanced by the Weyl constants once per
// round) are computed on the host, so inside a kernel they are plain
// constant-bank operands of the XORs.
struct Key {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline Key make_key(uint64_t seed)
{
    Key k;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = a;
        k.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox(uint4 c, const Key& key)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ key.k0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ key.k1[r], (uint32_t)p0);
    }
    return c;
}

// Philox4x32-10 for counters (x0, x1, x2, x3) whose words 1..3 stay fixed
// over many calls (a block's phase-1 entries, the serial method's copy draws).
// In the first round the product of word 2 depends only on the fixed words,
// and so does the second round's product of word 0; PhiloxHead holds what
// those two products contribute, so a call does 18 of the 20 multiplies.
// Same output as philox().
struct PhiloxHead {
    uint32_t f2;   // x3 ^ k1[0]: XORed into word 2 after the first round
    uint32_t f3;   // lo(M1 x2) ^ k0[1]: XORed into word 0 after the second round
    uint32_t f4;   // hi(M0 w0) ^ k1[1], w0 = hi(M1 x2) ^ x1 ^ k0[0]: into word 2, second round
    uint32_t f5;   // lo(M0 w0): word 3 after the second round
};

__host__ __device__ __forceinline__ PhiloxHead philox_head(uint32_t x1, uint32_t x2, uint32_t x3,
                                                           const Key& key)
{
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    const uint32_t w0 = (uint32_t)(p1 >> 32) ^ x1 ^ key.k0[0];
    const uint64_t q0 = (uint64_t)0xD2511F53u * w0;
    PhiloxHead h;
    h.f2 = x3 ^ key.k1[0];
    h.f3 = (uint32_t)p1 ^ key.k0[1];
    h.f4 = (uint32_t)(q0 >> 32) ^ key.k1[1];
    h.f5 = (uint32_t)q0;
    return h;
}

__device__ __forceinline__ uint4 philox_headed(uint32_t x0, const PhiloxHead& h, const Key& key)
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * x0;          // first round, word 0
    const uint32_t y2 = (uint32_t)(p0 >> 32) ^ h.f2, y3 = (uint32_t)p0;
    const uint64_t q1 = (uint64_t)0xCD9E8D57u * y2;          // second round, word 2
    uint4 c = make_uint4((uint32_t)(q1 >> 32) ^ h.f3, (uint32_t)q1, y3 ^ h.f4, h.f5);
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t a0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t a1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(a1 >> 32) ^ c.y ^ key.k0[r], (uint32_t)a1,
                       (uint32_t)(a0 >> 32) ^ c.w ^ key.k1[r], (uint32_t)a0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(uint64_t idx, uint32_t stream, uint32_t tag, const Key& key)
{
    return philox(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), stream, tag), key);
}

// Uniform integer in [0, R): high 64 bits of ((w1 << 32) | w0) * R.
__device__ __forceinline__ uint64_t uniform64(uint32_t w0, uint32_t w1, uint64_t R)
{
    return __umul64hi(((uint64_t)w1 << 32) | w0, R);
}

// floor(n / d) for every 64-bit n with a precomputed multiplier
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Sec. 4: t = mulhi(mul, n),
// q = (t + ((n - t) >> s1)) >> s2 with l = ceil(log2 d),
// mul = floor(2^64 (2^l - d) / d) + 1, s1 = min(l, 1), s2 = max(l - 1, 0)).
struct FastDiv {
    uint64_t mul;
    uint32_t s1, s2;
};

__host__ __device__ __forceinline__ uint64_t fdiv(uint64_t n, const FastDiv& f)
{
#ifdef __CUDA_ARCH__
    const uint64_t t = __umul64hi(f.mul, n);
#else
    const uint64_t t = (uint64_t)(((unsigned __int128)f.mul * n) >> 64);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// floor(n / d) for 32-bit n (same method with 32-bit words).
struct FastDiv32 {
    uint32_t mul, s1, s2;
};

__host__ __device__ __forceinline__ uint32_t fdiv32(uint32_t n, const FastDiv32& f)
{
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.mul, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.mul * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

__host__ inline FastDiv32 make_fastdiv32(uint32_t d)
{
    uint32_t l = 0;
    while (l < 32 && ((uint64_t)1 << l) < d) ++l;
    FastDiv32 f;
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    const uint64_t hi = ((uint64_t)1 << l) - d;   // < d
    f.mul = (uint32_t)((hi << 32) / d + 1);
    return f;
}

// Uniform integer in [0, R) for R < 2^32: the same value as uniform64 (the
// high 64 bits of the 96-bit product), from two 32x32->64 multiplies.
__device__ __forceinline__ uint32_t uniform32(uint32_t w0, uint32_t w1, uint32_t R)
{
    const uint64_t hi = (uint64_t)w1 * R;
    const uint64_t lo = (uint64_t)w0 * R;
    return (uint32_t)((hi + (lo >> 32)) >> 32);
}

// Builds the multiplier for divisor d >= 1 (host or device; the device path
// uses a bitwise long division and is meant for per-launch set-up only).
__host__ __device__ inline FastDiv make_fastdiv(uint64_t d)
{
    uint32_t l = 0;
    while (l < 64 && ((uint64_t)1 << l) < d) ++l;   // l = ceil(log2 d)
    FastDiv f;
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 0 ? l - 1 : 0;
    // numerator 2^64 * (2^l - d), a 128-bit value (hi, lo) with lo = 0
    const uint64_t hi = (l == 64) ? (uint64_t)(0 - d) : (((uint64_t)1 << l) - d);
#ifdef __CUDA_ARCH__
    // restoring long division of (hi:0) by d; hi < d so the quotient fits
    uint64_t rem = hi, quo = 0;
    for (int b = 63; b >= 0; --b) {
        const uint64_t top = rem >> 63;
        rem <<= 1;
        quo <<= 1;
        if (top || rem >= d) {
            rem -= d;
            quo |= 1;
        }
    }
    f.mul = quo + 1;
#else
    const unsigned __int128 num = (unsigned __int128)hi << 64;
    f.mul = (uint64_t)(num / d) + 1;
#endif
    return f;
}

// Endpoint `side` (0 = smaller id) of seed-clique edge e, the edges of
// K_{n0} being listed in lexicographic order (a, b), a < b.
__device__ __forceinline__ uint32_t seed_endpoint(uint64_t e, uint32_t side, uint32_t n0)
{
    uint32_t a = 0;
    uint64_t row = n0 - 1;
    while (e >= row) {
        e -= row;
        ++a;
        --row;
    }
    return side ? a + 1 + (uint32_t)e : a;
}

}  // namespace pgen
