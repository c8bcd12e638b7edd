// philox.cuh -- the Philox4x64-10 counter-based generator (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), usable
// on host and device.  Random draws of the scheme (Section 2.1's U and
// G(sigma) sampling) are indexed by counters, so every coefficient of every
// ciphertext has a fixed position in a stream independent of launch shape.
//
// Streams: key = (seed, tag); counter = (c0, c1, c2, 0).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define HW_HD __host__ __device__ __forceinline__
#else
#define HW_HD inline
#endif

enum HwStreamTag : uint64_t {
    HW_TAG_KEY = 1,     // secret key coefficients
    HW_TAG_RGSW_A = 2,  // uniform masks a of RGSW rows
    HW_TAG_RGSW_E = 3,  // Gaussian errors e of RGSW rows
    HW_TAG_PERM = 4,    // the bit permutation pi_r
    HW_TAG_H3 = 5,      // H3 hash matrix rows
    HW_TAG_KSK_A = 7,   // uniform masks of the packing key-switching key
    HW_TAG_KSK_E = 8,   // Gaussian errors of the packing key-switching key
};

struct Philox4 {
    uint64_t v[4];
};

HW_HD void mulhilo64(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo) {
#ifdef __CUDA_ARCH__
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

HW_HD Philox4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                         uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#ifdef __CUDA_ARCH__
#pragma unroll
#endif
    for (int i = 0; i < 10; i++) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, hi0, lo0);
        mulhilo64(M1, c2, hi1, lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    Philox4 r;
    r.v[0] = c0;
    r.v[1] = c1;
    r.v[2] = c2;
    r.v[3] = c3;
    return r;
}

HW_HD Philox4 hw_draw(uint64_t seed, uint64_t tag, uint64_t c0, uint64_t c1, uint64_t c2) {
    return philox4x64(c0, c1, c2, 0, seed, tag);
}
