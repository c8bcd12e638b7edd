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

// Everything a kernel needs to know about a context, passed by value.
struct DevCtx {
    int log_n, n, r, dnum, dpp, log_beta;
    int L, a, k0, k1, z, n_slots, n_data, s, n_classes;
    int therm_bits, tuple_bits, hash_h3, n_values, log_p, act, act_arg;
    int n_gates;
    PrimeConst P[HW_MAXP];
    u64 n_inv[HW_MAXP], n_inv_s[HW_MAXP];  // N^-1 and its Shoup companion
    u64 delta[HW_MAXP];                    // floor(Q/p) mod q_i
    u64 gconst[HW_MAX_DNUM];               // gadget value of row rho at its prime
    // decryption constants (Q < 2^(64*HW_LIMBS))
    u64 Q[HW_LIMBS], halfQ[HW_LIMBS];
    u64 M[HW_MAXP][HW_LIMBS];              // Q / q_i
    u64 yM[HW_MAXP];                       // (Q/q_i)^-1 mod q_i, Montgomery form
    int8_t gate_lvl[HW_MAX_GATES], gate_j[HW_MAX_GATES];
    int8_t slot_of[1 << HW_MAX_Z];         // tree index v -> stored ciphertext slot, -1 if none
    // device tables
    const u64* tw_fwd;    // [r][N] psi^brv(i)
    const u64* tw_fwd_s;  // Shoup companions
    const u64* tw_inv;    // [r][N] psi^-brv(i)
    const u64* tw_inv_s;
    const int32_t* ram_slot;  // [k0][a] encrypted bit slot of RAM j, address bit i (-1: 0)
    const int32_t* perm;      // [s] pi_r
    const u64* h3;            // [tuple_bits] H3 rows
    size_t rlwe_words, rgsw_words, lwe_words, sample_words, model_words;
};

// ---------------------------------------------------------------------------
// Block-level negacyclic NTT over N = 2^log_n residues in shared memory,
// blockDim.x = N/8 threads, each handling 8 elements per round.
//
// Forward: Cooley-Tukey with the psi powers merged into the butterflies
// (stage with m groups uses psi^brv(m+i)); natural order in, bit-reversed
// order out.  Inverse: Gentleman-Sande with psi^-brv, bit-reversed in,
// natural out, scaled by N^-1.  A round performs R (1..3) consecutive stages
// on register-resident groups of 2^R elements, so shared memory is touched
// once per R stages.  Values stay fully reduced in [0, q).
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void ntt_fwd_round(u64* a, int log_n, int st0, const u64* __restrict__ tw,
                                              const u64* __restrict__ tws, u64 q) {
    constexpr int E = 1 << R;
    constexpr int G = 8 >> R;
    const int T = blockDim.x;
    const int b_hi = log_n - 1 - st0;
    const int b_lo = b_hi - (R - 1);
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        int g = threadIdx.x + gg * T;
        int lo = g & ((1 << b_lo) - 1);
        int hi = g >> b_lo;
        int base = (hi << (b_hi + 1)) | lo;
        u64 x[E];
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = a[base + (e << b_lo)];
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int lb = R - 1 - s;
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << lb)) continue;
                int ti = (1 << (st0 + s)) + ((hi << s) | (e >> (lb + 1)));
                u64 W = tw[ti], Ws = tws[ti];
                u64 U = x[e];
                u64 V = shoup_mul(x[e | (1 << lb)], W, Ws, q);
                x[e] = add_mod(U, V, q);
                x[e | (1 << lb)] = sub_mod(U, V, q);
            }
        }
#pragma unroll
        for (int e = 0; e < E; e++) a[base + (e << b_lo)] = x[e];
    }
}

template <int R>
__device__ __forceinline__ void ntt_inv_round(u64* a, int log_n, int p0, const u64* __restrict__ tw,
                                              const u64* __restrict__ tws, u64 q, bool scale,
                                              u64 ninv, u64 ninv_s) {
    constexpr int E = 1 << R;
    constexpr int G = 8 >> R;
    const int T = blockDim.x;
#pragma unroll
    for (int gg = 0; gg < G; gg++) {
        int g = threadIdx.x + gg * T;
        int lo = g & ((1 << p0) - 1);
        int hi = g >> p0;
        int base = (hi << (p0 + R)) | lo;
        u64 x[E];
#pragma unroll
        for (int e = 0; e < E; e++) x[e] = a[base + (e << p0)];
#pragma unroll
        for (int s = 0; s < R; s++) {
            const int p = p0 + s;
            const int h = 1 << (log_n - 1 - p);
#pragma unroll
            for (int e = 0; e < E; e++) {
                if (e & (1 << s)) continue;
                int ti = h + ((hi << (R - 1 - s)) | (e >> (s + 1)));
                u64 W = tw[ti], Ws = tws[ti];
                u64 U = x[e], V = x[e | (1 << s)];
                x[e] = add_mod(U, V, q);
                x[e | (1 << s)] = shoup_mul(sub_mod(U, V, q), W, Ws, q);
            }
        }
        if (scale) {
#pragma unroll
            for (int e = 0; e < E; e++) x[e] = shoup_mul(x[e], ninv, ninv_s, q);
        }
#pragma unroll
        for (int e = 0; e < E; e++) a[base + (e << p0)] = x[e];
    }
}

// Forward transform of a[0..N) at prime j.  Caller has synchronised the
// block after writing a; the function returns synchronised.
__device__ __forceinline__ void ntt_forward_block(u64* a, const DevCtx& C, int j) {
    const u64* tw = C.tw_fwd + (size_t)j * C.n;
    const u64* tws = C.tw_fwd_s + (size_t)j * C.n;
    const u64 q = C.P[j].q;
    int st = 0;
    while (st < C.log_n) {
        int rem = C.log_n - st;
        if (rem >= 3) {
            ntt_fwd_round<3>(a, C.log_n, st, tw, tws, q);
            st += 3;
        } else if (rem == 2) {
            ntt_fwd_round<2>(a, C.log_n, st, tw, tws, q);
            st += 2;
        } else {
            ntt_fwd_round<1>(a, C.log_n, st, tw, tws, q);
            st += 1;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void ntt_inverse_block(u64* a, const DevCtx& C, int j) {
    const u64* tw = C.tw_inv + (size_t)j * C.n;
    const u64* tws = C.tw_inv_s + (size_t)j * C.n;
    const u64 q = C.P[j].q;
    int p = 0;
    while (p < C.log_n) {
        int rem = C.log_n - p;
        int R = rem >= 3 ? 3 : rem;
        bool last = (p + R == C.log_n);
        if (R == 3)
            ntt_inv_round<3>(a, C.log_n, p, tw, tws, q, last, C.n_inv[j], C.n_inv_s[j]);
        else if (R == 2)
            ntt_inv_round<2>(a, C.log_n, p, tw, tws, q, last, C.n_inv[j], C.n_inv_s[j]);
        else
            ntt_inv_round<1>(a, C.log_n, p, tw, tws, q, last, C.n_inv[j], C.n_inv_s[j]);
        p += R;
        __syncthreads();
    }
}

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

enum ExtOut { EXT_ADD = 0, EXT_PLAIN = 1, EXT_LWE = 2 };

// The external product C [x] D for one RLWE, computed by one thread block.
//
//   D   = srcA * X^eA - srcB * X^eB      (srcB == nullptr: D = srcA * X^eA)
//   out = srcB * X^eB + C [x] D          (EXT_ADD, written as RLWE to dst)
//       = C [x] D                        (EXT_PLAIN)
//       = ExtractLWE(srcB * X^eB + C [x] D, 0)   (EXT_LWE, dst is an LWE)
//
// C [x] D = sum_rho Dec(D.b)_rho * row_rho + Dec(D.a)_rho * row_{dnum+rho}:
// for each target prime j every digit polynomial is lifted to q_j, moved to
// evaluation form in shared memory, multiplied into the two accumulators
// with the RGSW rows (Montgomery form), and the accumulators are brought back
// with the inverse transform.  dst must not alias srcA or srcB (all primes of
// the sources are read while prime j is written).  smem: 3N words.
static __device__ __noinline__ void ext_product_block(const DevCtx& C, const u64* __restrict__ rgsw,
                                               const u64* srcA, int eA, const u64* srcB, int eB,
                                               int mode, u64* dst, u64* smem) {
    const int n = C.n, r = C.r, T = blockDim.x, tid = threadIdx.x;
    u64* buf = smem;
    u64* outA = smem + n;
    u64* outB = smem + 2 * n;
    for (int j = 0; j < r; j++) {
        const PrimeConst Pj = C.P[j];
        const u64 qj = Pj.q;
        for (int x = tid; x < n; x += T) {
            outA[x] = 0;
            outB[x] = 0;
        }
        for (int comp = 0; comp < 2; comp++) {
            for (int rho = 0; rho < C.dnum; rho++) {
                const int i = rho / C.dpp, k = rho % C.dpp;
                const u64 qi = C.P[i].q;
                const u64* pa = srcA + ((size_t)comp * r + i) * n;
                const u64* pb = srcB ? srcB + ((size_t)comp * r + i) * n : nullptr;
                __syncthreads();  // buf is free
                for (int x = tid; x < n; x += T) {
                    u64 v = rot_read(pa, x, eA, n, qi);
                    if (pb) v = sub_mod(v, rot_read(pb, x, eB, n, qi), qi);
                    int64_t d = gadget_digit(centre(v, qi), k, C.dpp, C.log_beta);
                    buf[x] = from_signed(d, qj);
                }
                __syncthreads();
                ntt_forward_block(buf, C, j);
                const int row = comp == 1 ? rho : C.dnum + rho;
                const u64* Ra = rgsw + ((size_t)(row * 2 + 0) * r + j) * n;
                const u64* Rb = rgsw + ((size_t)(row * 2 + 1) * r + j) * n;
                for (int x = tid; x < n; x += T) {
                    u64 d = buf[x];
                    outA[x] = add_mod(outA[x], mont_mul(d, __ldg(Ra + x), Pj), qj);
                    outB[x] = add_mod(outB[x], mont_mul(d, __ldg(Rb + x), Pj), qj);
                }
            }
        }
        __syncthreads();
        ntt_inverse_block(outA, C, j);
        ntt_inverse_block(outB, C, j);
        const u64* ba = srcB ? srcB + ((size_t)0 * r + j) * n : nullptr;
        const u64* bb = srcB ? srcB + ((size_t)1 * r + j) * n : nullptr;
        if (mode == EXT_LWE) {
            u64* lw = dst + (size_t)j * (n + 1);
            for (int y = tid; y < n; y += T) {
                u64 va = add_mod(outA[y], rot_read(ba, y, eB, n, qj), qj);
                // a'_0 = a_0, a'_x = -a_{N-x}
                if (y == 0)
                    lw[0] = va;
                else
                    lw[n - y] = neg_mod(va, qj);
            }
            if (tid == 0) lw[n] = add_mod(outB[0], rot_read(bb, 0, eB, n, qj), qj);
        } else {
            u64* da = dst + ((size_t)0 * r + j) * n;
            u64* db = dst + ((size_t)1 * r + j) * n;
            for (int x = tid; x < n; x += T) {
                u64 va = outA[x], vb = outB[x];
                if (mode == EXT_ADD) {
                    va = add_mod(va, rot_read(ba, x, eB, n, qj), qj);
                    vb = add_mod(vb, rot_read(bb, x, eB, n, qj), qj);
                }
                da[x] = va;
                db[x] = vb;
            }
        }
        __syncthreads();
    }
}
