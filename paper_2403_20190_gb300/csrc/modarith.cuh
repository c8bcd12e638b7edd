// modarith.cuh -- 64-bit modular arithmetic for residues modulo NTT-friendly
// primes q < 2^62 (the RNS primes of the ring R_q, Section 2.4).
//
// * Shoup multiplication by a fixed operand w with companion
//   w' = floor(w * 2^64 / q): r = x*w - umulhi(x, w')*q lies in [0, 2q).
// * Montgomery reduction with R = 2^64: for T < q*R,
//   REDC(T) = (T + ((T mod R) * q') mod R * q) / R  in [0, 2q),  q' = -q^-1 mod R.
//   Operands stored "in Montgomery form" are x*R mod q, so REDC(a * bM) = a*b.
#pragma once
#include <cstdint>

typedef uint64_t u64;
typedef uint32_t u32;

struct PrimeConst {
    u64 q;       // the prime
    u64 qneg;    // -q^{-1} mod 2^64
    u64 r2;      // 2^128 mod q
    u64 mu;      // floor((2^64 - 1) / q), Barrett constant for 64-bit inputs
};

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) {
    return a >= b ? a - b : a + q - b;
}

__device__ __forceinline__ u64 neg_mod(u64 a, u64 q) { return a ? q - a : 0; }

// x * w mod q for a fixed w with Shoup companion ws; result in [0, q).
__device__ __forceinline__ u64 shoup_mul(u64 x, u64 w, u64 ws, u64 q) {
    u64 qh = __umul64hi(x, ws);
    u64 r = x * w - qh * q;
    return r >= q ? r - q : r;
}

// Same, result left in [0, 2q) (lazy).
__device__ __forceinline__ u64 shoup_mul_lazy(u64 x, u64 w, u64 ws, u64 q) {
    u64 qh = __umul64hi(x, ws);
    return x * w - qh * q;
}

// Montgomery reduction of hi*2^64 + lo < q*2^64; result in [0, q).
__device__ __forceinline__ u64 redc(u64 hi, u64 lo, const PrimeConst& P) {
    u64 m = lo * P.qneg;
    u64 mqh = __umul64hi(m, P.q);
    u64 t = hi + mqh + (lo != 0 ? 1 : 0);
    return t >= P.q ? t - P.q : t;
}

// a * bM mod q where bM = b * 2^64 mod q (Montgomery form), a, bM < q.
__device__ __forceinline__ u64 mont_mul(u64 a, u64 bM, const PrimeConst& P) {
    return redc(__umul64hi(a, bM), a * bM, P);
}

// x * 2^64 mod q (into Montgomery form), x < q.
__device__ __forceinline__ u64 to_mont(u64 x, const PrimeConst& P) {
    u64 t = mont_mul(x, P.r2, P);  // x * 2^128 * 2^-64
    return t;
}

// xM * 2^-64 mod q (out of Montgomery form).
__device__ __forceinline__ u64 from_mont(u64 xM, const PrimeConst& P) { return redc(0, xM, P); }

// x mod q for any 64-bit x (Barrett with mu = floor((2^64-1)/q); the
// quotient estimate is short by at most 2).
__device__ __forceinline__ u64 reduce64(u64 x, const PrimeConst& P) {
    u64 qh = __umul64hi(x, P.mu);
    u64 r = x - qh * P.q;
    if (r >= P.q) r -= P.q;
    if (r >= P.q) r -= P.q;
    return r;
}

// (hi * 2^64 + lo) mod q for any 128-bit value.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const PrimeConst& P) {
    u64 h = reduce64(hi, P);         // < q, so h*2^64 + lo < q*2^64
    u64 t = redc(h, lo, P);          // (h*2^64 + lo) * 2^-64
    return mont_mul(t, P.r2, P);     // * 2^128 * 2^-64
}

// A signed integer |v| < 2^62 reduced into [0, q).
__device__ __forceinline__ u64 from_signed(int64_t v, u64 q) {
    if (v >= 0) {
        u64 u = (u64)v;
        return u >= q ? u % q : u;
    }
    u64 u = (u64)(-v);
    u = u >= q ? u % q : u;
    return u ? q - u : 0;
}
