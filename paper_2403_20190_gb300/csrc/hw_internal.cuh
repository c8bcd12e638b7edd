// hw_internal.cuh -- device-side context and building blocks shared by the
// library's kernels: the block-level negacyclic NTT in shared memory, gadget
// digits, and the fused external product (Section 2.4, "C [x] c").
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "modarith.cuh"
#include "philox.cuh"

#define HW_MAXP 4
#define HW_MAX_DNUM 32
#define HW_MAX_Z 5
#define HW_MAX_GATES 32
#define HW_LIMBS 4

// Everything a kernel needs to know about a context (kept in device memory;
// kernels receive a pointer to it).
struct DevCtx {
    int log_n, n, r, dnum, dpp, log_beta;
    int L, a, k0, k1, z, n_slots, n_data, s, n_classes;
    int therm_bits, tuple_bits, hash_h3, n_values, log_p, act, act_arg;
    int n_gates;
    int ext_loge, ext_np;  // external-product geometry (evaluation layout follows ext_loge)
    PrimeConst P[HW_MAXP];
    u64 n_inv[HW_MAXP], n_inv_s[HW_MAXP];  // N^-1 and its Shoup companion
    u64 mr[HW_MAXP], mr_s[HW_MAXP];        // R = 2^64 mod q_i and its Shoup companion
    u64 mr2_s[HW_MAXP];                    // Shoup companion of R^2 mod q_i (P[i].r2)
    // u^-1 mod 2N for psi_min = psi^u: evaluation position pos holds RGSW
    // mask sampling point brv((a_point_mul (2 brv(pos) + 1) mod 2N) >> 1)
    uint32_t a_point_mul[HW_MAXP];
    u64 delta[HW_MAXP];                    // floor(Q/p) mod q_i
    u64 gconst[HW_MAX_DNUM];               // gadget value of row rho at its prime
    // decryption constants (Q < 2^(64*HW_LIMBS))
    u64 Q[HW_LIMBS], halfQ[HW_LIMBS];
    u64 M[HW_MAXP][HW_LIMBS];              // Q / q_i
    u64 yM[HW_MAXP];                       // (Q/q_i)^-1 mod q_i, Montgomery form
    int8_t gate_lvl[HW_MAX_GATES], gate_j[HW_MAX_GATES];
    int8_t slot_of[1 << HW_MAX_Z];         // tree index v -> stored ciphertext slot, -1 if none
    // device tables
    const ulonglong2* tw_fwd;  // [r][N] (psi^brv(i), Shoup companion)
    const ulonglong2* tw_inv;  // [r][N] (psi^-brv(i), Shoup companion)
    const int32_t* ram_slot;  // [k0][a] encrypted bit slot of RAM j, address bit i (-1: 0)
    const int32_t* perm;      // [s] pi_r
    const u64* h3;            // [tuple_bits] H3 rows
    // Rotation tables in evaluation order: X^e evaluates to Psi^e[pos] =
    // psi^((2 brv(pos) + 1) e); rot_tab[((j*2 + sign)*log_n + t)*N + pos] holds
    // (Psi^(+-2^t) - 1, Shoup) with sign 0 for +2^t and 1 for -2^t, and
    // rot_inv the same for (Psi^(+-2^t) - 1)^-1.
    const ulonglong2* rot_tab;
    const ulonglong2* rot_inv;
    // 32-bit transform tables (w, floor(w 2^32 / q)) when every q_i < 2^30, else null
    const uint2* tw32_fwd;
    const uint2* tw32_inv;
    uint32_t n_inv32[HW_MAXP], n_inv32_s[HW_MAXP];
    int diag;  // one digit per prime: the digit of prime i at prime i is the residue
    int ext32;  // the external product runs in 32-bit words (ext_product32)
    size_t rlwe_words, rgsw_words, lwe_words, sample_words, model_words;
};

// ---------------------------------------------------------------------------
// Gadget digits (inverse of G in EncRGSW, Section 2.4; RNS reading): the
// residue at source prime i is centred into (-q_i/2, q_i/2] and split into
// dpp signed base-2^log_beta digits in [-beta/2, beta/2), least significant
// first, the last one keeping the carry; with log_beta = 0 the only digit is
// the centred residue.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t centre(u64 v, u64 q) {
    return v > (q - 1) / 2 ? (int64_t)v - (int64_t)q : (int64_t)v;
}

__device__ __forceinline__ int64_t gadget_digit(int64_t c, int k, int dpp, int log_beta) {
    if (log_beta == 0) return c;
    const int64_t half = (int64_t)1 << (log_beta - 1);
    const int64_t mask = ((int64_t)1 << log_beta) - 1;
    for (int t = 0; t < k; t++) {
        int64_t m = ((c + half) & mask) - half;
        c = (c - m) >> log_beta;
    }
    if (k == dpp - 1) return c;
    return ((c + half) & mask) - half;
}

// (p * X^e)[x] for e in [0, 2N): coefficient x - e with a sign flip per wrap.
__device__ __forceinline__ u64 rot_read(const u64* p, int x, int e, int n, u64 q) {
    int t = x - e;
    int neg = 0;
    while (t < 0) {
        t += n;
        neg ^= 1;
    }
    u64 v = p[t];
    return neg ? neg_mod(v, q) : v;
}


// RGSW rows are streamed once per (sample, RAM) step: loading them with an
// L2 evict-first policy keeps them from displacing the per-block
// accumulators, which are reread at the next step.  A hint only.
__device__ __forceinline__ u64 rgsw_policy() {
    u64 pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ u64 ld_rgsw(const u64* p, u64 pol) {
    u64 v;
    asm("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
}

// A digit |d| < q_j lifted to [0, q_j).
__device__ __forceinline__ u64 lift_small(int64_t d, u64 q) { return d >= 0 ? (u64)d : (u64)(d + (int64_t)q); }

// Montgomery reduction without the final subtraction: for T < q*2^64 the
// result (T + ((T mod 2^64) q') mod 2^64 * q) / 2^64 lies in [0, 2q).
__device__ __forceinline__ u64 redc_lazy(u64 hi, u64 lo, u64 q, u64 qneg) {
    return hi + __umul64hi(lo * qneg, q) + (lo != 0 ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Block-level negacyclic NTT, specialised on the ring size N = 2^LOGN
// (6 <= LOGN <= 13) and the residues per thread E = 2^LOGE (4, 8 or 16).
// A block of T = N/E threads holds E residues per thread and polynomial in
// registers; a round applies up to LOGE consecutive butterfly stages to
// groups of 2^R residues in registers, and rounds exchange data through one
// of two padded shared-memory buffers (address p + p/E keeps every
// exchange at two wavefronts per warp).
//
// Forward (Cooley-Tukey, psi powers merged, natural order in, bit-reversed
// out): the partial round of LOGN mod LOGE stages comes first, then full
// rounds.  Butterflies are lazy (no reduction): X' = X + t, Y' = X + 2q - t
// with t = Shoup(Y*W) in [0, 2q), so values grow by < 2q per stage and stay
// below (2*LOGN + 1) q < 2^60.
// Inverse (Gentleman-Sande, bit-reversed in, natural out, inputs < 2q):
// full rounds first, the partial round last; the sum is kept below 2q by
// one conditional subtraction, the difference goes through a lazy Shoup
// product.  Scaling by N^-1 is applied by the caller to the inputs.
//
// Register convention: in a round of R stages, v[gg + e*G] (G = E / 2^R) is
// element e of the thread's group gg.  The first forward round reads and the
// last inverse round writes positions tid + k*T (v[k]); the last forward
// round leaves, and the first inverse round takes, positions E*tid + e.
// ---------------------------------------------------------------------------
// Default external-product geometry: 2^3 residues per thread, two
// polynomials per transform below N = 8192 and one at N = 8192 (1024-thread
// blocks).  A context may choose another instantiated geometry
// (hw_create_tuned).
__host__ __device__ constexpr int default_ext_loge(int) { return 3; }
__host__ __device__ constexpr int default_ext_np(int log_n) { return log_n >= 13 ? 1 : 2; }

// Evaluation-form arrays (RGSW rows, the key's evaluation form, rotation
// tables, evaluation-form copies of ciphertexts) are stored thread-major in
// the context's external-product geometry: evaluation position E*t + e
// lives at address e*T + t (E = 2^loge residues per thread, T = N/E
// threads), so every load and store in that geometry is coalesced.
__host__ __device__ inline int eval_addr(int pos, int log_n, int loge) {
    const int T = (1 << log_n) >> loge;
    return (pos & ((1 << loge) - 1)) * T + (pos >> loge);
}

template <int LOGN, int LOGE = 4>
struct Ring {
    static constexpr int N = 1 << LOGN;
    static constexpr int E = 1 << LOGE;         // residues per thread and polynomial
    static constexpr int T = N / E;             // threads per block
    static constexpr int RP = LOGN % LOGE;      // size of the partial round
    static constexpr int PADDED = N + N / E;    // words per exchange buffer
};

// Padded shared-memory address: one spare word every E words keeps the
// stride-E accesses of the last forward / first inverse round conflict-free.
template <int LOGE>
__device__ __forceinline__ int padw(int p) { return p + (p >> LOGE); }

template <int LOGN, int LOGE, int ST0>
struct FwdR {
    static constexpr int R = (ST0 == 0 && Ring<LOGN, LOGE>::RP) ? Ring<LOGN, LOGE>::RP : LOGE;
};
template <int LOGN, int LOGE, int P0>
struct InvR {
    static constexpr int R = (LOGN - P0) < LOGE ? (LOGN - P0) : LOGE;
};

// position of element e of group gg in the forward round (ST0, R)
template <int LOGN, int LOGE, int ST0, int R>
__device__ __forceinline__ int fpos(int gg, int e) {
    constexpr int B_HI = LOGN - 1 - ST0, B_LO = B_HI - R + 1;
    const int g = threadIdx.x + gg * Ring<LOGN, LOGE>::T;
    const int lo = g & ((1 << B_LO) - 1), hi = g >> B_LO;
    return (hi << (B_HI + 1)) | lo | (e << B_LO);
}

// position of element e of group gg in the inverse round (P0, R)
template <int LOGN, int LOGE, int P0, int R>
__device__ __forceinline__ int ipos(int gg, int e) {
    const int g = threadIdx.x + gg * Ring<LOGN, LOGE>::T;
    const int lo = g & ((1 << P0) - 1), hi = g >> P0;
    return (hi << (P0 + R)) | lo | (e << P0);
}

// A round on NP polynomials of the same prime: the twiddles of one group
// for all stages are loaded before any butterfly and serve every polynomial.
template <int LOGN, int LOGE, int NP, int ST0, int R>
__device__ __forceinline__ void fwd_round(u64 (&v)[NP][1 << LOGE], const ulonglong2* __restrict__ tw,
                                          u64 q, u64 q2) {
    constexpr int E = 1 << R, G = (1 << LOGE) / E, B_LO = LOGN - ST0 - R;
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        const int hi = (threadIdx.x + gg * Ring<LOGN, LOGE>::T) >> B_LO;
        ulonglong2 W[E - 1];  // stage s, index j < 2^s at W[2^s - 1 + j]
#pragma unroll
        for (int s = 0; s < R; s++)
#pragma unroll
            for (int jj = 0; jj < (1 << s); jj++)
                W[(1 << s) - 1 + jj] = __ldg(tw + (1 << (ST0 + s)) + ((hi << s) | jj));
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int lb = R - 1 - s;
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << lb)) continue;
                const ulonglong2 w = W[(1 << s) - 1 + (e >> (lb + 1))];
#pragma unroll
                for (int pp = 0; pp < NP; pp++) {
                    u64& X = v[pp][gg + e * G];
                    u64& Y = v[pp][gg + (e | (1 << lb)) * G];
                    const u64 t = shoup_mul_lazy(Y, w.x, w.y, q);
                    Y = X + q2 - t;
                    X = X + t;
                }
            }
        }
    }
}

template <int LOGN, int LOGE, int NP, int P0, int R>
__device__ __forceinline__ void inv_round(u64 (&v)[NP][1 << LOGE], const ulonglong2* __restrict__ tw,
                                          u64 q, u64 q2) {
    constexpr int E = 1 << R, G = (1 << LOGE) / E;
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        const int hi = (threadIdx.x + gg * Ring<LOGN, LOGE>::T) >> P0;
        ulonglong2 W[E - 1];  // stage s, index j < 2^(R-1-s) at W[2^(R-1-s) - 1 + j]
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int h = 1 << (LOGN - 1 - (P0 + s));
#pragma unroll
            for (int jj = 0; jj < (1 << (R - 1 - s)); jj++)
                W[(1 << (R - 1 - s)) - 1 + jj] = __ldg(tw + h + ((hi << (R - 1 - s)) | jj));
        }
#pragma unroll
        for (int s = 0; s < R; s++) {
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << s)) continue;
                const ulonglong2 w = W[(1 << (R - 1 - s)) - 1 + (e >> (s + 1))];
#pragma unroll
                for (int pp = 0; pp < NP; pp++) {
                    u64& U = v[pp][gg + e * G];
                    u64& V = v[pp][gg + (e | (1 << s)) * G];
                    u64 sum = U + V;
                    sum = sum >= q2 ? sum - q2 : sum;
                    V = shoup_mul_lazy(U + q2 - V, w.x, w.y, q);
                    U = sum;
                }
            }
        }
    }
}

// Exchange buffers: two sets, alternated between exchanges (par) so that
// one barrier per exchange suffices -- a set is rewritten only two exchanges
// after it was read, with a barrier in between.  Each set holds NP padded
// polynomials (stride `stride` words).  With b0 == b1 (one set, half the
// shared memory) each exchange takes a second barrier before its writes.
struct Xchg {
    u64* b0;
    u64* b1;
    int stride;
    int par;
    u64* accs = nullptr;  // external-product accumulators in shared memory (mode 2), 2*N words
    __device__ __forceinline__ u64* next() {
        u64* p = par ? b1 : b0;
        par ^= 1;
        return p;
    }
};

template <int LOGN, int LOGE, int NP, int ST0>
__device__ __forceinline__ void fwd_from(u64 (&v)[NP][1 << LOGE], Xchg& xc,
                                         const ulonglong2* __restrict__ tw, u64 q, u64 q2) {
    constexpr int R = FwdR<LOGN, LOGE, ST0>::R, G = (1 << LOGE) >> R;
    fwd_round<LOGN, LOGE, NP, ST0, R>(v, tw, q, q2);
    if constexpr (ST0 + R < LOGN) {
        constexpr int R2 = FwdR<LOGN, LOGE, ST0 + R>::R, G2 = (1 << LOGE) >> R2;
        u64* sm = xc.next();
        if (xc.b0 == xc.b1) __syncthreads();  // one buffer: the last exchange's reads are done
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R); e++)
                    sm[pp * xc.stride + padw<LOGE>(fpos<LOGN, LOGE, ST0, R>(gg, e))] = v[pp][gg + e * G];
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G2; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R2); e++)
                    v[pp][gg + e * G2] = sm[pp * xc.stride + padw<LOGE>(fpos<LOGN, LOGE, ST0 + R, R2>(gg, e))];
        fwd_from<LOGN, LOGE, NP, ST0 + R>(v, xc, tw, q, q2);
    }
}

template <int LOGN, int LOGE, int NP, int P0>
__device__ __forceinline__ void inv_from(u64 (&v)[NP][1 << LOGE], Xchg& xc,
                                         const ulonglong2* __restrict__ tw, u64 q, u64 q2) {
    constexpr int R = InvR<LOGN, LOGE, P0>::R, G = (1 << LOGE) >> R;
    inv_round<LOGN, LOGE, NP, P0, R>(v, tw, q, q2);
    if constexpr (P0 + R < LOGN) {
        constexpr int R2 = InvR<LOGN, LOGE, P0 + R>::R, G2 = (1 << LOGE) >> R2;
        u64* sm = xc.next();
        if (xc.b0 == xc.b1) __syncthreads();  // one buffer: the last exchange's reads are done
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R); e++)
                    sm[pp * xc.stride + padw<LOGE>(ipos<LOGN, LOGE, P0, R>(gg, e))] = v[pp][gg + e * G];
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G2; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R2); e++)
                    v[pp][gg + e * G2] = sm[pp * xc.stride + padw<LOGE>(ipos<LOGN, LOGE, P0 + R, R2>(gg, e))];
        inv_from<LOGN, LOGE, NP, P0 + R>(v, xc, tw, q, q2);
    }
}

// Forward transform at prime j of NP polynomials held as v[p][k] (position
// tid + k*T, values < q); on return v[p][e] is the lazy value
// (< (2 LOGN + 1) q) at evaluation position E*tid + e.
template <int LOGN, int LOGE, int NP>
__device__ __forceinline__ void ntt_fwd(u64 (&v)[NP][1 << LOGE], Xchg& xc, const DevCtx& C, int j) {
    const u64 q = C.P[j].q;
    fwd_from<LOGN, LOGE, NP, 0>(v, xc, C.tw_fwd + (size_t)j * Ring<LOGN>::N, q, 2 * q);
}

// Inverse transform at prime j of v[p][e] (position E*tid + e, values < 2q,
// already multiplied by N^-1); on return v[p][k] (position tid + k*T) < 2q.
template <int LOGN, int LOGE, int NP>
__device__ __forceinline__ void ntt_inv(u64 (&v)[NP][1 << LOGE], Xchg& xc, const DevCtx& C, int j) {
    const u64 q = C.P[j].q;
    inv_from<LOGN, LOGE, NP, 0>(v, xc, C.tw_inv + (size_t)j * Ring<LOGN>::N, q, 2 * q);
}

// ---------------------------------------------------------------------------
// 32-bit transform for primes below 2^30 (Harvey butterflies, values < 4q <
// 2^32): forward X' = X~ + t, Y' = X~ + 2q - t with X~ = X reduced below 2q
// and t = Shoup(Y*W) in [0, 2q); inverse as the 64-bit one.  Same positions,
// rounds and exchanges as the 64-bit transform.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 shoup32_lazy(u32 x, u32 w, u32 ws, u32 q) {
    return x * w - __umulhi(x, ws) * q;
}

template <int LOGN, int LOGE, int NP, int ST0, int R>
__device__ __forceinline__ void fwd_round32(u32 (&v)[NP][1 << LOGE], const uint2* __restrict__ tw,
                                            u32 q, u32 q2) {
    constexpr int E = 1 << R, G = (1 << LOGE) / E, B_LO = LOGN - ST0 - R;
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        const int hi = (threadIdx.x + gg * Ring<LOGN, LOGE>::T) >> B_LO;
        uint2 W[E - 1];
#pragma unroll
        for (int s = 0; s < R; s++)
#pragma unroll
            for (int jj = 0; jj < (1 << s); jj++)
                W[(1 << s) - 1 + jj] = __ldg(tw + (1 << (ST0 + s)) + ((hi << s) | jj));
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int lb = R - 1 - s;
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << lb)) continue;
                const uint2 w = W[(1 << s) - 1 + (e >> (lb + 1))];
#pragma unroll
                for (int pp = 0; pp < NP; pp++) {
                    u32& X = v[pp][gg + e * G];
                    u32& Y = v[pp][gg + (e | (1 << lb)) * G];
                    const u32 x = X >= q2 ? X - q2 : X;
                    const u32 t = shoup32_lazy(Y, w.x, w.y, q);
                    Y = x + q2 - t;
                    X = x + t;
                }
            }
        }
    }
}

template <int LOGN, int LOGE, int NP, int P0, int R>
__device__ __forceinline__ void inv_round32(u32 (&v)[NP][1 << LOGE], const uint2* __restrict__ tw,
                                            u32 q, u32 q2) {
    constexpr int E = 1 << R, G = (1 << LOGE) / E;
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        const int hi = (threadIdx.x + gg * Ring<LOGN, LOGE>::T) >> P0;
        uint2 W[E - 1];
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int h = 1 << (LOGN - 1 - (P0 + s));
#pragma unroll
            for (int jj = 0; jj < (1 << (R - 1 - s)); jj++)
                W[(1 << (R - 1 - s)) - 1 + jj] = __ldg(tw + h + ((hi << (R - 1 - s)) | jj));
        }
#pragma unroll
        for (int s = 0; s < R; s++) {
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << s)) continue;
                const uint2 w = W[(1 << (R - 1 - s)) - 1 + (e >> (s + 1))];
#pragma unroll
                for (int pp = 0; pp < NP; pp++) {
                    u32& U = v[pp][gg + e * G];
                    u32& V = v[pp][gg + (e | (1 << s)) * G];
                    u32 sum = U + V;
                    sum = sum >= q2 ? sum - q2 : sum;
                    V = shoup32_lazy(U + q2 - V, w.x, w.y, q);
                    U = sum;
                }
            }
        }
    }
}

template <int LOGN, int LOGE, int NP, int ST0>
__device__ __forceinline__ void fwd_from32(u32 (&v)[NP][1 << LOGE], Xchg& xc,
                                           const uint2* __restrict__ tw, u32 q, u32 q2) {
    constexpr int R = FwdR<LOGN, LOGE, ST0>::R, G = (1 << LOGE) >> R;
    fwd_round32<LOGN, LOGE, NP, ST0, R>(v, tw, q, q2);
    if constexpr (ST0 + R < LOGN) {
        constexpr int R2 = FwdR<LOGN, LOGE, ST0 + R>::R, G2 = (1 << LOGE) >> R2;
        u32* sm = (u32*)xc.next();
        if (xc.b0 == xc.b1) __syncthreads();  // one buffer: the last exchange's reads are done
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R); e++)
                    sm[pp * xc.stride + padw<LOGE>(fpos<LOGN, LOGE, ST0, R>(gg, e))] = v[pp][gg + e * G];
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G2; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R2); e++)
                    v[pp][gg + e * G2] = sm[pp * xc.stride + padw<LOGE>(fpos<LOGN, LOGE, ST0 + R, R2>(gg, e))];
        fwd_from32<LOGN, LOGE, NP, ST0 + R>(v, xc, tw, q, q2);
    }
}

template <int LOGN, int LOGE, int NP, int P0>
__device__ __forceinline__ void inv_from32(u32 (&v)[NP][1 << LOGE], Xchg& xc,
                                           const uint2* __restrict__ tw, u32 q, u32 q2) {
    constexpr int R = InvR<LOGN, LOGE, P0>::R, G = (1 << LOGE) >> R;
    inv_round32<LOGN, LOGE, NP, P0, R>(v, tw, q, q2);
    if constexpr (P0 + R < LOGN) {
        constexpr int R2 = InvR<LOGN, LOGE, P0 + R>::R, G2 = (1 << LOGE) >> R2;
        u32* sm = (u32*)xc.next();
        if (xc.b0 == xc.b1) __syncthreads();  // one buffer: the last exchange's reads are done
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R); e++)
                    sm[pp * xc.stride + padw<LOGE>(ipos<LOGN, LOGE, P0, R>(gg, e))] = v[pp][gg + e * G];
        __syncthreads();
#pragma unroll
        for (int pp = 0; pp < NP; pp++)
#pragma unroll
            for (int gg = 0; gg < G2; gg++)
#pragma unroll
                for (int e = 0; e < (1 << R2); e++)
                    v[pp][gg + e * G2] = sm[pp * xc.stride + padw<LOGE>(ipos<LOGN, LOGE, P0 + R, R2>(gg, e))];
        inv_from32<LOGN, LOGE, NP, P0 + R>(v, xc, tw, q, q2);
    }
}

// A warp's 32*E consecutive positions E*(32w + lane) + e (thread-held as
// v[e]) moved to/from dst[position] with coalesced global accesses, through
// a warp-private region of 32*(E+1) words of wbuf (padded: conflict-free).
template <int E, typename W>
__device__ __forceinline__ void warp_store_positions(W* dst, const W (&v)[E], W* wbuf) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    W* wb = wbuf + w * 32 * (E + 1);
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; e++) wb[lane * (E + 1) + e] = v[e];
    __syncwarp();
    W* d = dst + (size_t)w * 32 * E;
#pragma unroll
    for (int k = 0; k < E; k++) {
        const int idx = k * 32 + lane;
        d[idx] = wb[idx + idx / E];
    }
    __syncwarp();
}

template <int E, typename W, typename S>
__device__ __forceinline__ void warp_load_positions(const S* src, W (&v)[E], W* wbuf) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    W* wb = wbuf + w * 32 * (E + 1);
    const S* s = src + (size_t)w * 32 * E;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < E; k++) {
        const int idx = k * 32 + lane;
        wb[idx + idx / E] = (W)s[idx];
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; e++) v[e] = wb[lane * (E + 1) + e];
    __syncwarp();
}

// Single-polynomial forms with 16 residues per thread (utility kernels).
template <int LOGN>
__device__ __forceinline__ void ntt_fwd1(u64 (&v)[16], Xchg& xc, const DevCtx& C, int j) {
    ntt_fwd<LOGN, 4, 1>(reinterpret_cast<u64(&)[1][16]>(v), xc, C, j);
}
template <int LOGN>
__device__ __forceinline__ void ntt_inv1(u64 (&v)[16], Xchg& xc, const DevCtx& C, int j) {
    ntt_inv<LOGN, 4, 1>(reinterpret_cast<u64(&)[1][16]>(v), xc, C, j);
}

// x mod q for any 64-bit x (Barrett, quotient short by at most 2).
__device__ __forceinline__ u64 reduce_full(u64 x, const PrimeConst& P) { return reduce64(x, P); }

// Ask L2 to fetch [p, p + words) (one request per 128-byte line, spread over
// the block).  A hint only: it changes no value.
__device__ __forceinline__ void prefetch_l2(const u64* p, size_t words) {
    const char* b = (const char*)p;
    const size_t bytes = words * sizeof(u64);
    for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(b + off));
}

enum ExtOut { EXT_ADD = 0, EXT_PLAIN = 1, EXT_LWE = 2 };

// Evaluation-form companions of an external product.
//   src_ntt  evaluation form of srcA (fully reduced), or null
//   dst_ntt  where to write the evaluation form of the output, or null
//   rot_t    >= 0: the product is a blind-rotation CMUX, srcA == srcB and
//            D = src X^(eB + s 2^rot_t) - src X^eB with s = +1 (rot_sign 0)
//            or -1 (rot_sign 1); -1 otherwise
struct ExtNtt {
    const u64* src_ntt;
    u64* dst_ntt;
    int rot_t;
    int rot_sign;
    const u64* next_rgsw;  // RGSW of the next external product (L2 prefetch), or null
    int prefetch_cur;      // also prefetch this product's RGSW
    // the forward transforms of all 2 dnum digits of D at every prime, as
    // ext_digits writes them ([prime][digit][address]); read by the
    // ext_product<..., DG = true> instances only
    const u64* digits = nullptr;
};

// The external product C [x] D for one RLWE, computed by one thread block.
//
//   D   = srcA * X^eA - srcB * X^eB      (srcB == nullptr: D = srcA * X^eA)
//   out = srcB * X^eB + C [x] D          (EXT_ADD, written as RLWE to dst)
//       = C [x] D                        (EXT_PLAIN)
//       = ExtractLWE(srcB * X^eB + C [x] D, 0)   (EXT_LWE, dst is an LWE)
//
// C [x] D = sum_rho Dec(D.b)_rho * row_rho + Dec(D.a)_rho * row_{dnum+rho}.
// For each target prime j, digit polynomials are built in registers at the
// first-round positions and transformed NP at a time; the last round's
// registers are multiplied into per-thread accumulators (RGSW rows are in
// Montgomery form: one lazy REDC per product).  The accumulators are scaled
// by N^-1, transformed back, and combined with the base at the natural
// positions the last inverse round leaves.  dst must not alias the sources.
//
// With one digit per prime (C.diag), the digit of prime j lifted to q_j is
// the residue D_j itself, so its transform is the evaluation form of the
// source times (Psi^(+-2^t) - 1) for a rotation CMUX, or the evaluation form
// itself for a CDEMUX: those 2 of the 2r digit transforms per target prime
// are skipped when nt.src_ntt is given.  When it is not, a rotation CMUX
// recovers the evaluation form of its base from the diagonal digit's
// transform (times (Psi^(+-2^t) - 1)^-1) so that dst_ntt can still be written.
// The external product's two accumulator polynomials at one prime: E words
// per thread each, in registers (MODE 0), in thread-private shared-memory
// slots (oc*E + e)*T + tid (MODE 1, frees 2E 64-bit registers), or
// component 0 in such slots and component 1 in registers (MODE 2, frees E).
template <int E, int T, int MODE>
struct Acc {
    u64 r[MODE == 1 ? 1 : (MODE == 2 ? 1 : 2)][MODE == 1 ? 1 : E];
    u64* s;
    __device__ __forceinline__ explicit Acc(u64* base) : s(MODE ? base + threadIdx.x : nullptr) {}
    __device__ __forceinline__ u64& at(int oc, int e) {
        if constexpr (MODE == 1) return s[(oc * E + e) * T];
        else if constexpr (MODE == 2) return oc == 0 ? s[e * T] : r[0][e];
        else return r[oc][e];
    }
    __device__ __forceinline__ u64 get(int oc, int e) { return at(oc, e); }
    __device__ __forceinline__ void set(int oc, int e, u64 v) { at(oc, e) = v; }
    __device__ __forceinline__ void add(int oc, int e, u64 v) { at(oc, e) += v; }
};

// The external product in 32-bit words, for contexts whose primes are below
// 2^30 and whose gadget has several digits per prime (no diagonal digit, so
// no evaluation-form companions).  Digits are lifted to q_j and transformed
// as 32-bit words; the MAC adds the exact 64-bit products d * row (d < q_j,
// rows < q_j in Montgomery form x 2^64: a sum of 2 dnum terms stays below
// 2^64, which the host checks before it sets C.ext32); each output residue is
// reduced once and the rows' factor 2^64 taken off with one REDC.  The same
// canonical results as the 64-bit path.
template <int LOGN, int LOGE, int NP, int AS>
__device__ __noinline__ void ext_product32(const DevCtx& C, const u64* __restrict__ rgsw,
                                           const u64* srcA, int eA, const u64* srcB, int eB, int mode,
                                           u64* dst, Xchg& xc, ExtNtt nt) {
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    const int tid = threadIdx.x, r = C.r;
    const int ndig = 2 * C.dnum;
    const u64 rpol = rgsw_policy();
    if (nt.prefetch_cur) prefetch_l2(rgsw, C.rgsw_words);
    if (nt.next_rgsw) prefetch_l2(nt.next_rgsw, C.rgsw_words);
    __syncthreads();  // exchange buffers are free
    for (int j = 0; j < r; j++) {
        const PrimeConst Pj = C.P[j];
        const u64 qj = Pj.q;
        const u32 q32 = (u32)qj, q2 = 2 * q32;
        Acc<E, T, AS> acc(xc.accs);
#pragma unroll
        for (int e = 0; e < E; e++) {
            acc.set(0, e, 0);
            acc.set(1, e, 0);
        }
        for (int u0 = 0; u0 < ndig; u0 += NP) {
            u32 v[NP][E];
            int comps[NP], rhos[NP];
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const int u = u0 + pp;
                const int comp = u / C.dnum, rho = u % C.dnum;
                comps[pp] = comp;
                rhos[pp] = rho;
                const int i = rho / C.dpp, k = rho % C.dpp;
                const u64 qi = C.P[i].q;
                const u64* pa = srcA + ((size_t)comp * r + i) * N;
                const u64* pb = srcB ? srcB + ((size_t)comp * r + i) * N : nullptr;
#pragma unroll
                for (int kk = 0; kk < E; kk++) {
                    const int x = tid + kk * T;
                    u64 val = rot_read(pa, x, eA, N, qi);
                    if (pb) val = sub_mod(val, rot_read(pb, x, eB, N, qi), qi);
                    v[pp][kk] = (u32)lift_small(gadget_digit(centre(val, qi), k, C.dpp, C.log_beta), qj);
                }
            }
            fwd_from32<LOGN, LOGE, NP, 0>(v, xc, C.tw32_fwd + (size_t)j * N, q32, q2);
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const int comp = comps[pp], rho = rhos[pp];
                const int row = comp == 1 ? rho : C.dnum + rho;
                const u64* Ra = rgsw + ((size_t)(row * 2 + 0) * r + j) * N + tid;
                const u64* Rb = rgsw + ((size_t)(row * 2 + 1) * r + j) * N + tid;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    u32 d = v[pp][e];  // < 4q
                    d = d >= q2 ? d - q2 : d;
                    d = d >= q32 ? d - q32 : d;
                    const u32 ra = (u32)ld_rgsw(Ra + e * T, rpol), rb = (u32)ld_rgsw(Rb + e * T, rpol);
                    acc.add(0, e, (u64)d * ra);
                    acc.add(1, e, (u64)d * rb);
                }
            }
        }
        const u32 ninv = C.n_inv32[j], ninv_s = C.n_inv32_s[j];
        constexpr int NPI = NP < 2 ? NP : 2;  // the two output components
        for (int oc0 = 0; oc0 < 2; oc0 += NPI) {
            u32 v[NPI][E];
#pragma unroll
            for (int pp = 0; pp < NPI; pp++)
#pragma unroll
                for (int e = 0; e < E; e++) {
                    // (sum d * row) mod q carries the rows' 2^64: REDC takes it off
                    const u64 sred = redc(0, reduce64(acc.get(oc0 + pp, e), Pj), Pj);
                    v[pp][e] = shoup32_lazy((u32)sred, ninv, ninv_s, q32);
                }
            inv_from32<LOGN, LOGE, NPI, 0>(v, xc, C.tw32_inv + (size_t)j * N, q32, q2);
#pragma unroll
            for (int pp = 0; pp < NPI; pp++) {
                const int oc = oc0 + pp;
                const u64* base = srcB ? srcB + ((size_t)oc * r + j) * N : nullptr;
                if (mode == EXT_LWE) {
                    u64* lw = dst + (size_t)j * (N + 1);
                    if (oc == 0) {
#pragma unroll
                        for (int kk = 0; kk < E; kk++) {
                            const int x = tid + kk * T;
                            u64 val = v[pp][kk] >= q32 ? v[pp][kk] - q32 : v[pp][kk];
                            val = add_mod(val, rot_read(base, x, eB, N, qj), qj);
                            if (x == 0)
                                lw[0] = val;
                            else
                                lw[N - x] = neg_mod(val, qj);
                        }
                    } else if (tid == 0) {
                        u64 val = v[pp][0] >= q32 ? v[pp][0] - q32 : v[pp][0];
                        lw[N] = add_mod(val, rot_read(base, 0, eB, N, qj), qj);
                    }
                } else {
                    u64* dd = dst + ((size_t)oc * r + j) * N;
#pragma unroll
                    for (int kk = 0; kk < E; kk++) {
                        const int x = tid + kk * T;
                        u64 val = v[pp][kk] >= q32 ? v[pp][kk] - q32 : v[pp][kk];
                        if (mode == EXT_ADD) val = add_mod(val, rot_read(base, x, eB, N, qj), qj);
                        dd[x] = val;
                    }
                }
            }
        }
    }
    __syncthreads();  // dst complete for the whole block
}

template <int LOGN, int LOGE, int NP, int AS = 0, bool DG = false, bool B0 = false>
__device__ __noinline__ void ext_product(const DevCtx& C, const u64* __restrict__ rgsw,
                                         const u64* srcA, int eA, const u64* srcB, int eB, int mode,
                                         u64* dst, Xchg& xc, ExtNtt nt) {
    if constexpr (LOGN <= 11) {  // the rings of the 30-bit parameter sets
        if (C.ext32) {
            ext_product32<LOGN, LOGE, NP, AS>(C, rgsw, srcA, eA, srcB, eB, mode, dst, xc, nt);
            return;
        }
    }
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    const int tid = threadIdx.x, r = C.r;
    const bool cmux_rot = nt.rot_t >= 0;
    const bool diag_in = C.diag && nt.src_ntt && !DG &&
                         ((cmux_rot && eB == 0) || (!cmux_rot && srcB == nullptr && eA == 0));
    const bool derive_base = C.diag && !diag_in && cmux_rot && nt.dst_ntt && mode == EXT_ADD;
    // the output's evaluation form is written only when its base's is known:
    // no base (EXT_PLAIN), the source's own (unrotated CMUX base), or derived
    const bool base_given = mode == EXT_ADD && nt.src_ntt != nullptr && srcB == srcA && eB == 0;
    const bool write_ntt =
        C.diag && nt.dst_ntt != nullptr && (mode == EXT_PLAIN || base_given || derive_base);
    // digits that need a forward transform at target prime j
    const int ndig = diag_in ? 2 * (r - 1) : 2 * C.dnum;
    // stream this product's RGSW and the next one's into L2 ahead of the MACs
    const u64 rpol = rgsw_policy();
    if (nt.prefetch_cur) prefetch_l2(rgsw, C.rgsw_words);
    if (nt.next_rgsw) prefetch_l2(nt.next_rgsw, C.rgsw_words);
    __syncthreads();  // exchange buffers are free
    for (int j = 0; j < r; j++) {
        const PrimeConst Pj = C.P[j];
        const u64 qj = Pj.q;
        const ulonglong2* rtab =
            cmux_rot ? C.rot_tab + (((size_t)j * 2 + nt.rot_sign) * C.log_n + nt.rot_t) * N + tid
                     : nullptr;
        Acc<E, T, AS> acc(xc.accs);
#pragma unroll
        for (int e = 0; e < E; e++) {
            acc.set(0, e, 0);
            acc.set(1, e, 0);
        }
        if (diag_in) {
            // the two diagonal digits, straight from the evaluation form
#pragma unroll
            for (int comp = 0; comp < 2; comp++) {
                const int row = comp == 1 ? j : C.dnum + j;
                const u64* sn = nt.src_ntt + ((size_t)comp * r + j) * N + tid;
                const u64* Ra = rgsw + ((size_t)(row * 2 + 0) * r + j) * N + tid;
                const u64* Rb = rgsw + ((size_t)(row * 2 + 1) * r + j) * N + tid;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const u64 ra = ld_rgsw(Ra + e * T, rpol), rb = ld_rgsw(Rb + e * T, rpol);
                    u64 x = sn[e * T];
                    if (cmux_rot) {
                        const ulonglong2 t0 = __ldg(rtab + e * T);
                        x = shoup_mul_lazy(x, t0.x, t0.y, qj);
                    }
                    acc.add(0, e, redc_lazy(__umul64hi(x, ra), x * ra, qj, Pj.qneg));
                    acc.add(1, e, redc_lazy(__umul64hi(x, rb), x * rb, qj, Pj.qneg));
                }
            }
        }
        if constexpr (DG) {
            // the digits' transforms were computed beforehand (the source is
            // shared by other items, DG instances only): only the MACs
            const u64* dg = nt.digits + (size_t)j * ndig * N + tid;
            for (int u = 0; u < ndig; u++) {
                const int comp = u / C.dnum, rho = u % C.dnum;
                const int row = comp == 1 ? rho : C.dnum + rho;
                const u64* Ra = rgsw + ((size_t)(row * 2 + 0) * r + j) * N + tid;
                const u64* Rb = rgsw + ((size_t)(row * 2 + 1) * r + j) * N + tid;
                const u64* du = dg + (size_t)u * N;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const u64 ra = ld_rgsw(Ra + e * T, rpol), rb = ld_rgsw(Rb + e * T, rpol);
                    const u64 x = du[e * T];
                    acc.add(0, e, redc_lazy(__umul64hi(x, ra), x * ra, qj, Pj.qneg));
                    acc.add(1, e, redc_lazy(__umul64hi(x, rb), x * rb, qj, Pj.qneg));
                }
                if (derive_base && rho == j) {
                    const ulonglong2* ri =
                        C.rot_inv + (((size_t)j * 2 + nt.rot_sign) * C.log_n + nt.rot_t) * N + tid;
                    u64* bn = nt.dst_ntt + ((size_t)comp * r + j) * N + tid;
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const ulonglong2 w = __ldg(ri + e * T);
                        bn[e * T] = shoup_mul_lazy(du[e * T], w.x, w.y, qj);
                    }
                }
            }
        }
        for (int u0 = 0; u0 < (DG ? 0 : ndig); u0 += NP) {
            u64 v[NP][E];
            int comps[NP], rhos[NP];
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const int u = u0 + pp;
                int comp, rho;
                if (diag_in) {  // skip source prime j
                    comp = u / (r - 1);
                    const int ii = u % (r - 1);
                    rho = ii < j ? ii : ii + 1;
                } else {
                    comp = u / C.dnum;
                    rho = u % C.dnum;
                }
                comps[pp] = comp;
                rhos[pp] = rho;
                const int i = rho / C.dpp, k = rho % C.dpp;
                const u64 qi = C.P[i].q;
                const u64* pa = srcA + ((size_t)comp * r + i) * N;
                const u64* pb = srcB ? srcB + ((size_t)comp * r + i) * N : nullptr;
#pragma unroll
                for (int kk = 0; kk < E; kk++) {
                    const int x = tid + kk * T;
                    u64 val = rot_read(pa, x, eA, N, qi);
                    if (pb) val = sub_mod(val, rot_read(pb, x, eB, N, qi), qi);
                    v[pp][kk] = lift_small(gadget_digit(centre(val, qi), k, C.dpp, C.log_beta), qj);
                }
            }
            ntt_fwd<LOGN, LOGE, NP>(v, xc, C, j);
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const int comp = comps[pp], rho = rhos[pp];
                const int row = comp == 1 ? rho : C.dnum + rho;
                const u64* Ra = rgsw + ((size_t)(row * 2 + 0) * r + j) * N + tid;
                const u64* Rb = rgsw + ((size_t)(row * 2 + 1) * r + j) * N + tid;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const u64 ra = ld_rgsw(Ra + e * T, rpol), rb = ld_rgsw(Rb + e * T, rpol);
                    const u64 x = v[pp][e];
                    acc.add(0, e, redc_lazy(__umul64hi(x, ra), x * ra, qj, Pj.qneg));
                    acc.add(1, e, redc_lazy(__umul64hi(x, rb), x * rb, qj, Pj.qneg));
                }
                if (derive_base && rho == j) {
                    // the base's evaluation form: D_j / (Psi^(+-2^t) - 1)
                    const ulonglong2* ri =
                        C.rot_inv + (((size_t)j * 2 + nt.rot_sign) * C.log_n + nt.rot_t) * N + tid;
                    u64* bn = nt.dst_ntt + ((size_t)comp * r + j) * N + tid;
#pragma unroll
                    for (int e = 0; e < E; e++) {
                        const ulonglong2 w = __ldg(ri + e * T);
                        bn[e * T] = shoup_mul_lazy(v[pp][e], w.x, w.y, qj);
                    }
                }
            }
        }
        if (write_ntt) {
            // evaluation form of the output: (base +) C [x] D, fully reduced
#pragma unroll
            for (int oc = 0; oc < 2; oc++) {
                u64* dn = nt.dst_ntt + ((size_t)oc * r + j) * N + tid;
                const u64* bn = derive_base ? dn
                                : (base_given ? nt.src_ntt + ((size_t)oc * r + j) * N + tid : nullptr);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    u64 val = acc.get(oc, e) + (bn ? bn[e * T] : 0);
                    dn[e * T] = reduce64(val, Pj);
                }
            }
        }
        const u64 ninv = C.n_inv[j], ninv_s = C.n_inv_s[j];
        constexpr int NPI = NP < 2 ? NP : 2;  // the two output components
        for (int oc0 = 0; oc0 < 2; oc0 += NPI) {
            if (B0 && NPI == 1 && oc0 == 1 && mode == EXT_LWE) {
                // ExtractLWE keeps b_0 only: coefficient 0 of the inverse
                // transform is the sum of the (N^-1-scaled) evaluations, so a
                // block sum replaces the transform (B0 instances only: the
                // others keep their register allocation)
                u64 sum = 0;
#pragma unroll
                for (int e = 0; e < E; e++) {
                    u64 x = shoup_mul_lazy(acc.get(1, e), ninv, ninv_s, qj);
                    sum = add_mod(sum, x >= qj ? x - qj : x, qj);
                }
                u64* red = xc.next();
                if (xc.b0 == xc.b1) __syncthreads();  // one buffer: the last exchange's reads are done
                u64 t = 0;
                if constexpr (T >= 32) {  // whole warps: shuffles, then one warp over the warps' sums
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1)
                        sum = add_mod(sum, __shfl_down_sync(0xffffffffu, sum, off), qj);
                    if ((tid & 31) == 0) red[tid >> 5] = sum;
                    __syncthreads();
                    if (tid < 32) {
                        t = tid < T / 32 ? red[tid] : 0;
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1)
                            t = add_mod(t, __shfl_down_sync(0xffffffffu, t, off), qj);
                    }
                } else {  // fewer threads than a warp (the smallest rings)
                    red[tid] = sum;
                    __syncthreads();
                    if (tid == 0)
                        for (int k = 0; k < T; k++) t = add_mod(t, red[k], qj);
                }
                if (tid == 0)
                    dst[(size_t)j * (N + 1) + N] = add_mod(t, rot_read(srcB + ((size_t)r + j) * N, 0, eB, N, qj), qj);
                continue;
            }
            u64 v[NPI][E];
#pragma unroll
            for (int pp = 0; pp < NPI; pp++)
#pragma unroll
                for (int e = 0; e < E; e++) v[pp][e] = shoup_mul_lazy(acc.get(oc0 + pp, e), ninv, ninv_s, qj);
            ntt_inv<LOGN, LOGE, NPI>(v, xc, C, j);
#pragma unroll
            for (int pp = 0; pp < NPI; pp++) {
                const int oc = oc0 + pp;
                const u64* base = srcB ? srcB + ((size_t)oc * r + j) * N : nullptr;
                if (mode == EXT_LWE) {
                    u64* lw = dst + (size_t)j * (N + 1);
                    if (oc == 0) {
#pragma unroll
                        for (int kk = 0; kk < E; kk++) {
                            const int x = tid + kk * T;
                            u64 val = v[pp][kk] >= qj ? v[pp][kk] - qj : v[pp][kk];
                            val = add_mod(val, rot_read(base, x, eB, N, qj), qj);
                            if (x == 0)
                                lw[0] = val;
                            else
                                lw[N - x] = neg_mod(val, qj);
                        }
                    } else if (tid == 0) {
                        u64 val = v[pp][0] >= qj ? v[pp][0] - qj : v[pp][0];
                        lw[N] = add_mod(val, rot_read(base, 0, eB, N, qj), qj);
                    }
                } else {
                    u64* dd = dst + ((size_t)oc * r + j) * N;
#pragma unroll
                    for (int kk = 0; kk < E; kk++) {
                        const int x = tid + kk * T;
                        u64 val = v[pp][kk] >= qj ? v[pp][kk] - qj : v[pp][kk];
                        if (mode == EXT_ADD) val = add_mod(val, rot_read(base, x, eB, N, qj), qj);
                        dd[x] = val;
                    }
                }
            }
        }
    }
    __syncthreads();  // dst complete for the whole block
}

// The forward transforms ext_product computes for D = srcA X^eA - srcB X^eB
// before its MACs (no evaluation form of the source given): the 2 dnum
// gadget digits lifted to every prime j, written to
// out[(j * 2 dnum + u) * N + address], u = comp * dnum + rho, the lazy values
// of the transform as they are.  ext_product with ExtNtt::digits = out then
// gives the same result as with the source.
template <int LOGN, int LOGE, int NP>
__device__ __noinline__ void ext_digits(const DevCtx& C, const u64* srcA, int eA, const u64* srcB, int eB,
                                        Xchg& xc, u64* out) {
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    const int tid = threadIdx.x, r = C.r;
    const int ndig = 2 * C.dnum;
    __syncthreads();  // exchange buffers are free
    for (int j = 0; j < r; j++) {
        const u64 qj = C.P[j].q;
        for (int u0 = 0; u0 < ndig; u0 += NP) {
            u64 v[NP][E];
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const int u = u0 + pp;
                const int comp = u / C.dnum, rho = u % C.dnum;
                const int i = rho / C.dpp, k = rho % C.dpp;
                const u64 qi = C.P[i].q;
                const u64* pa = srcA + ((size_t)comp * r + i) * N;
                const u64* pb = srcB ? srcB + ((size_t)comp * r + i) * N : nullptr;
#pragma unroll
                for (int kk = 0; kk < E; kk++) {
                    const int x = tid + kk * T;
                    u64 val = rot_read(pa, x, eA, N, qi);
                    if (pb) val = sub_mod(val, rot_read(pb, x, eB, N, qi), qi);
                    v[pp][kk] = lift_small(gadget_digit(centre(val, qi), k, C.dpp, C.log_beta), qj);
                }
            }
            ntt_fwd<LOGN, LOGE, NP>(v, xc, C, j);
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                u64* o = out + ((size_t)j * ndig + u0 + pp) * N + tid;
#pragma unroll
                for (int e = 0; e < E; e++) o[e * T] = v[pp][e];
            }
        }
    }
}

// Launch geometry of the external-product kernels: 2^LOGE residues per
// thread, NP polynomials transformed together, T = N / 2^LOGE threads.
template <int LOGN, int LOGE, int NP_, int SM = 0>
struct ExtCfg {
    static constexpr int LOGE_ = LOGE;
    static constexpr int NP = NP_;
    static constexpr int T = Ring<LOGN, LOGE>::T;
    static constexpr int PADDED = Ring<LOGN, LOGE>::PADDED;
    // shared-memory mode SM: 0 = two exchange sets; 1 = one set, the rest
    // holds the accumulator's evaluation form (2*r*N words, added at launch);
    // 2 = one set plus the two accumulator polynomials of one prime (2*N words)
    // 3 = two exchange sets plus accumulator component 0 (N words; component 1
    // stays in registers)
    static constexpr int ACC = SM == 2 ? 1 : (SM == 3 ? 2 : 0);  // Acc mode of ext_product
    static constexpr size_t XCHG_BYTES = (SM == 1 || SM == 2 ? 1 : 2) * (size_t)NP * PADDED * sizeof(u64);
    static constexpr size_t ACC_BYTES =
        (SM == 2 ? 2 : (SM == 3 ? 1 : 0)) * (size_t)Ring<LOGN>::N * sizeof(u64);
    static constexpr size_t FIXED_BYTES = XCHG_BYTES + ACC_BYTES;
    // blocks that can be resident per SM by shared memory (227 KiB, 1 KiB
    // reserved per block) and by a 512-thread target; the register cap the
    // compiler gets follows from the smaller, so a block that only fits once
    // per SM is not squeezed into registers it cannot use
    static constexpr int SMEM_BLOCKS = SM == 1 ? 1 : (int)((227 * 1024) / (FIXED_BYTES + 1024));
    static constexpr int THR_BLOCKS = (512 / T) < 1 ? 1 : (512 / T);
    static constexpr int MINB0 = SMEM_BLOCKS < THR_BLOCKS ? SMEM_BLOCKS : THR_BLOCKS;
    static constexpr int MINB = MINB0 < 1 ? 1 : (MINB0 > 16 ? 16 : MINB0);
};

// Launch geometry shared by the kernels that run block NTTs.
template <int LOGN>
struct Geo {
    static constexpr int T = Ring<LOGN>::T;
    static constexpr size_t XCHG_BYTES = 2 * (size_t)Ring<LOGN>::PADDED * sizeof(u64);
    static constexpr int MINB = (512 / T) > 16 ? 16 : (512 / T);
};

#define HW_FOR_EACH_LOGN(X) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13)
