// k_crypto.cu -- key generation, client encoding, RGSW encryption,
// decryption (phase, CRT, rounding), PD-act and transform utilities.
#include "hw_internal.cuh"
#include "hw_launch.h"

// ---------------------------------------------------------------------------
// SecretKeyGen: ternary S_1; key = [r][N] residues, then [r][N] evaluation
// form in Montgomery representation.
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T) k_keygen(const DevCtx* __restrict__ Cp, u64 seed,
                                                          u64* __restrict__ key) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int j = blockIdx.x, tid = threadIdx.x;
    const PrimeConst P = C.P[j];
    u64 v[16];
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
        const int x = tid + kk * T;
        Philox4 w = hw_draw(seed, HW_TAG_KEY, (u64)x >> 2, 0, 0);
        u64 t = w.v[x & 3] % 3;
        u64 res = t == 0 ? 0 : (t == 1 ? 1 : P.q - 1);
        key[(size_t)j * N + x] = res;
        v[kk] = res;
    }
    ntt_fwd1<LOGN>(v, xc, C, j);
#pragma unroll
    for (int e = 0; e < 16; e++)
        key[(size_t)(C.r + j) * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)] = to_mont(reduce_full(v[e], P), P);
}

// ---------------------------------------------------------------------------
// Client encoding: level = (v*(T+1)) >> 8, thermometer bit i = [i < level];
// hashed contexts permute (t_p = T_{perm[p]}), cut tuples and H3-hash them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int therm_bit(const DevCtx& C, const uint8_t* vals, int p) {
    const int f = p / C.therm_bits, i = p % C.therm_bits;
    const int level = ((int)vals[f] * (C.therm_bits + 1)) >> 8;
    return i < level ? 1 : 0;
}

__global__ void k_encode(const DevCtx* __restrict__ Cp, const uint8_t* __restrict__ values, size_t n,
                         uint8_t* __restrict__ bits) {
    const DevCtx& C = *Cp;
    if (!C.hash_h3) {
        const size_t total = n * (size_t)C.n_data;
        for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
             idx += (size_t)gridDim.x * blockDim.x) {
            const size_t i = idx / C.n_data;
            const int d = (int)(idx % C.n_data);
            bits[idx] = (uint8_t)therm_bit(C, values + i * C.n_values, d);
        }
        return;
    }
    const size_t total = n * (size_t)C.k0;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t i = idx / C.k0;
        const int j = (int)(idx % C.k0);
        u64 h = 0;
        for (int t = 0; t < C.tuple_bits; t++) {
            const int p = j * C.tuple_bits + t;
            if (p < C.s && therm_bit(C, values + i * C.n_values, C.perm[p])) h ^= C.h3[t];
        }
        for (int b = 0; b < C.a; b++)
            bits[i * C.n_data + (size_t)j * C.a + b] = (uint8_t)((h >> b) & 1);
    }
}

// ---------------------------------------------------------------------------
// Decryption: phase per prime, then CRT and rounding with multi-limb integers:
// phi = sum_i [phi_i * (Q/q_i)^-1]_{q_i} * (Q/q_i) mod Q, and
// m = floor((p*phi + floor(Q/2)) / Q) mod p, the quotient found by bisection.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void limbs_add(u64* a, const u64* b) {
    u64 carry = 0;
#pragma unroll
    for (int t = 0; t < HW_LIMBS; t++) {
        u64 s = a[t] + carry;
        u64 c1 = s < carry;
        u64 s2 = s + b[t];
        carry = c1 + (s2 < s);
        a[t] = s2;
    }
}

__device__ __forceinline__ bool limbs_ge(const u64* a, const u64* b) {
#pragma unroll
    for (int t = HW_LIMBS - 1; t >= 0; t--) {
        if (a[t] != b[t]) return a[t] > b[t];
    }
    return true;
}

__device__ __forceinline__ void limbs_sub(u64* a, const u64* b) {
    u64 borrow = 0;
#pragma unroll
    for (int t = 0; t < HW_LIMBS; t++) {
        u64 d = a[t] - b[t];
        u64 b1 = a[t] < b[t];
        u64 d2 = d - borrow;
        u64 b2 = d < borrow;
        a[t] = d2;
        borrow = b1 | b2;
    }
}

// out = a * m for a 64-bit m
__device__ __forceinline__ void limbs_mul64(const u64* a, u64 m, u64* out) {
    u64 carry = 0;
#pragma unroll
    for (int t = 0; t < HW_LIMBS; t++) {
        u64 lo = a[t] * m, hi = __umul64hi(a[t], m);
        lo += carry;
        hi += (lo < carry);
        out[t] = lo;
        carry = hi;
    }
}

__device__ int64_t decode_residues(const DevCtx& C, const u64* phi) {
    u64 acc[HW_LIMBS] = {0, 0, 0, 0};
    for (int i = 0; i < C.r; i++) {
        u64 ci = mont_mul(phi[i], C.yM[i], C.P[i]);
        u64 t[HW_LIMBS];
        limbs_mul64(C.M[i], ci, t);
        limbs_add(acc, t);
    }
    while (limbs_ge(acc, C.Q)) limbs_sub(acc, C.Q);
    // X = p * phi + floor(Q/2)
    u64 X[HW_LIMBS];
    limbs_mul64(acc, (u64)1 << C.log_p, X);
    limbs_add(X, C.halfQ);
    // largest m in [0, p] with m * Q <= X
    u64 lo = 0, hi = (u64)1 << C.log_p;
    while (lo < hi) {
        u64 mid = (lo + hi + 1) >> 1;
        u64 t[HW_LIMBS];
        limbs_mul64(C.Q, mid, t);
        if (limbs_ge(X, t))
            lo = mid;
        else
            hi = mid - 1;
    }
    return (int64_t)(lo & (((u64)1 << C.log_p) - 1));
}

// One block per (RLWE, prime): phase b - a*s at that prime into ph[ct][prime][N].
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_rlwe_phase(const DevCtx* __restrict__ Cp, const u64* __restrict__ key,
                 const u64* __restrict__ ct, u64* __restrict__ ph) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int r = C.r, tid = threadIdx.x;
    const size_t t = blockIdx.x / r;
    const int j = blockIdx.x % r;
    const PrimeConst P = C.P[j];
    const u64* c = ct + t * C.rlwe_words;
    u64 v[16];
#pragma unroll
    for (int kk = 0; kk < 16; kk++) v[kk] = c[(size_t)j * N + tid + kk * T];
    ntt_fwd1<LOGN>(v, xc, C, j);
#pragma unroll
    for (int e = 0; e < 16; e++)
        v[e] = shoup_mul_lazy(mont_mul(v[e], key[(size_t)(r + j) * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)], P), C.n_inv[j],
                              C.n_inv_s[j], P.q);
    ntt_inv1<LOGN>(v, xc, C, j);
    u64* dst = ph + (t * r + j) * N;
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
        const int x = tid + kk * T;
        const u64 as = v[kk] >= P.q ? v[kk] - P.q : v[kk];
        dst[x] = sub_mod(c[(size_t)(r + j) * N + x], as, P.q);
    }
}

// One thread per coefficient: CRT + rounding of the phases.
__global__ void k_decode_phase(const DevCtx* __restrict__ Cp, const u64* __restrict__ ph,
                               size_t count, int64_t* __restrict__ out) {
    const DevCtx& C = *Cp;
    const size_t total = count * C.n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t t = idx / C.n;
        const int x = (int)(idx % C.n);
        u64 phi[HW_MAXP];
        for (int j = 0; j < C.r; j++) phi[j] = ph[(t * C.r + j) * C.n + x];
        out[idx] = decode_residues(C, phi);
    }
}

// The counters W[c][j][addr] of Definition 2's model from the phases of
// RAMs j0 .. j0+nj-1 (ph: [ciphertext (j - j0) * k1 + slot][prime][N]): the
// LUT index m = c + 2^L addr (label bits low, Algorithm 6) sits in stored
// ciphertext slot_of[m mod 2^z] at coefficient m >> z.  One thread per
// counter; out is [class][RAM][address].
__global__ void k_decode_model(const DevCtx* __restrict__ Cp, const u64* __restrict__ ph, int j0, int nj,
                               int64_t* __restrict__ out) {
    const DevCtx& C = *Cp;
    const size_t A = (size_t)1 << C.a;
    const size_t total = (size_t)C.n_classes * nj * A;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t addr = idx % A, rest = idx / A;
        const int jj = (int)(rest % nj), c = (int)(rest / nj);
        const u64 m = (u64)c + ((u64)addr << C.L);
        const int v = (int)(m & (((u64)1 << C.z) - 1));
        const size_t coef = (size_t)(m >> C.z);
        const int slot = C.slot_of[v];
        u64 phi[HW_MAXP];
        const u64* p = ph + ((size_t)jj * C.k1 + slot) * C.r * C.n + coef;
        for (int j = 0; j < C.r; j++) phi[j] = p[(size_t)j * C.n];
        out[((size_t)c * C.k0 + j0 + jj) * A + addr] = decode_residues(C, phi);
    }
}

// One block per LWE: phase b' - <a', s> per prime (s is ternary), decode.
__global__ void k_decrypt_lwe(const DevCtx* __restrict__ Cp, const u64* __restrict__ key,
                              const u64* __restrict__ ct, int64_t* __restrict__ out) {
    __shared__ u64 red_pos[HW_MAXP][32], red_neg[HW_MAXP][32];
    const DevCtx& C = *Cp;
    const int n = C.n, r = C.r, T = blockDim.x, tid = threadIdx.x;
    const u64* c = ct + (size_t)blockIdx.x * C.lwe_words;
    const int lane = tid & 31, warp = tid >> 5, nw = (T + 31) >> 5;
    for (int j = 0; j < r; j++) {
        const u64 q = C.P[j].q;
        const u64* a = c + (size_t)j * (n + 1);
        const u64* s = key + (size_t)j * n;
        u64 pos = 0, neg = 0;
        for (int x = tid; x < n; x += T) {
            u64 sv = s[x];
            if (sv == 1) pos = add_mod(pos, a[x], q);
            else if (sv == q - 1) neg = add_mod(neg, a[x], q);
        }
        for (int off = 16; off > 0; off >>= 1) {
            u64 p2 = __shfl_down_sync(0xffffffffu, pos, off);
            u64 n2 = __shfl_down_sync(0xffffffffu, neg, off);
            pos = add_mod(pos, p2, q);
            neg = add_mod(neg, n2, q);
        }
        if (lane == 0) {
            red_pos[j][warp] = pos;
            red_neg[j][warp] = neg;
        }
    }
    __syncthreads();
    if (tid == 0) {
        u64 phi[HW_MAXP];
        for (int j = 0; j < r; j++) {
            const u64 q = C.P[j].q;
            u64 pos = 0, neg = 0;
            for (int w = 0; w < nw; w++) {
                pos = add_mod(pos, red_pos[j][w], q);
                neg = add_mod(neg, red_neg[j][w], q);
            }
            const u64 b = c[(size_t)j * (n + 1) + n];
            phi[j] = sub_mod(b, sub_mod(pos, neg, q), q);
        }
        out[blockIdx.x] = decode_residues(C, phi);
    }
}

// ---------------------------------------------------------------------------
// PD-act: activate each decrypted response, add per class, arg-max.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t activate(const DevCtx& C, int64_t x) {
    // floor(log2(x + 1)) = bit length of (x + 1) minus one
    int64_t lg = 63 - __clzll((unsigned long long)(x + 1));
    if (C.act == 0) return lg;
    if (C.act == 1) return lg < C.act_arg ? lg : C.act_arg;
    return x > C.act_arg ? 1 : 0;
}

__global__ void k_pdact(const DevCtx* __restrict__ Cp, const int64_t* __restrict__ counts, int n,
                        int64_t* __restrict__ scores, int32_t* __restrict__ labels) {
    const DevCtx& C = *Cp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = C.n_classes;
    int best = 0;
    int64_t best_s = -1;
    for (int c = 0; c < l; c++) {
        const int64_t* u = counts + ((size_t)i * l + c) * C.k0;
        int64_t s = 0;
        for (int j = 0; j < C.k0; j++) s += activate(C, u[j]);
        scores[(size_t)i * l + c] = s;
        if (s > best_s) {
            best_s = s;
            best = c;
        }
    }
    labels[i] = best;
}

// PD-act with the balancing rescale (Section 3.6.1; the rule is a reading):
// every counter of class c is scaled by n_ref / n_c with floor division
// before the activation, n_ref = the largest class count; classes with
// n_c = 0 are left as they are (their counters are 0).
__global__ void k_pdact_balanced(const DevCtx* __restrict__ Cp, const int64_t* __restrict__ counts,
                                 const int64_t* __restrict__ class_counts, int n,
                                 int64_t* __restrict__ scores, int32_t* __restrict__ labels) {
    const DevCtx& C = *Cp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int l = C.n_classes;
    int64_t n_ref = 0;
    for (int c = 0; c < l; c++) n_ref = class_counts[c] > n_ref ? class_counts[c] : n_ref;
    int best = 0;
    int64_t best_s = -1;
    for (int c = 0; c < l; c++) {
        const int64_t* u = counts + ((size_t)i * l + c) * C.k0;
        const int64_t nc = class_counts[c];
        int64_t s = 0;
        for (int j = 0; j < C.k0; j++) s += activate(C, nc > 0 ? (u[j] * n_ref) / nc : u[j]);
        scores[(size_t)i * l + c] = s;
        if (s > best_s) {
            best_s = s;
            best = c;
        }
    }
    labels[i] = best;
}

// ---------------------------------------------------------------------------
// Transform utilities.
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_export_rgsw(const DevCtx* __restrict__ Cp, const u64* __restrict__ in, u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    const size_t poly = blockIdx.x;  // [rgsw][row][comp][prime]
    const int j = (int)(poly % C.r);
    const PrimeConst P = C.P[j];
    u64 v[16];
#pragma unroll
    for (int e = 0; e < 16; e++)
        v[e] = shoup_mul_lazy(from_mont(in[poly * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)], P), C.n_inv[j],
                              C.n_inv_s[j], P.q);
    ntt_inv1<LOGN>(v, xc, C, j);
#pragma unroll
    for (int kk = 0; kk < 16; kk++) out[poly * N + tid + kk * T] = v[kk] >= P.q ? v[kk] - P.q : v[kk];
}

// The inverse of k_export_rgsw: canonical coefficient words (any 64-bit
// values, reduced mod q_i first) -> evaluation form, Montgomery
// representation, the context's thread-major layout.  Every read precedes
// the first barrier and every write follows the last, so it runs in place.
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_import_rgsw(const DevCtx* __restrict__ Cp, const u64* in, u64* out) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    const size_t poly = blockIdx.x;  // [rgsw][row][comp][prime]
    const int j = (int)(poly % C.r);
    const PrimeConst P = C.P[j];
    u64 v[16];
#pragma unroll
    for (int kk = 0; kk < 16; kk++) v[kk] = reduce_full(in[poly * N + tid + kk * T], P);
    ntt_fwd1<LOGN>(v, xc, C, j);
#pragma unroll
    for (int e = 0; e < 16; e++)
        out[poly * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)] = to_mont(reduce_full(v[e], P), P);
}

// Clear counters -> the plaintext tables of unencrypted-model inference.  One
// block per polynomial [RAM j][class c][leaf v][prime]: coefficient k of
// leaf v is counts[c][j][v + 2^zt k] (zt = max(0, z - L); 0 past the RAM's
// 2^a addresses), reduced into the prime, transformed, and stored in the
// external product's evaluation layout in Montgomery form.
template <int LOGN>
__global__ void __launch_bounds__(Ring<LOGN>::T)
    k_plain_load(const DevCtx* __restrict__ Cp, const int64_t* __restrict__ counts, u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    const size_t poly = blockIdx.x;
    const int jp = (int)(poly % C.r);
    const int zt = C.z > C.L ? C.z - C.L : 0;
    const size_t rest = poly / C.r;
    const int v = (int)(rest & ((1u << zt) - 1));
    const size_t jc = rest >> zt;
    const int c = (int)(jc % C.n_classes), j = (int)(jc / C.n_classes);
    const PrimeConst P = C.P[jp];
    const size_t n_addr = (size_t)1 << C.a;
    const int64_t* row = counts + ((size_t)c * C.k0 + j) * n_addr;
    u64 vv[16];
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
        const size_t addr = (size_t)v + ((size_t)(tid + kk * T) << zt);
        vv[kk] = addr < n_addr ? from_signed(row[addr], P.q) : 0;
    }
    ntt_fwd1<LOGN>(vv, xc, C, jp);
#pragma unroll
    for (int e = 0; e < 16; e++)
        out[poly * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)] = to_mont(reduce_full(vv[e], P), P);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define HW_LAUNCHED() ((*li.launches)++, cudaGetLastError())

#define HW_DISPATCH(logn, BODY)      \
    switch (logn) {                  \
        BODY(6) BODY(7) BODY(8) BODY(9) BODY(10) BODY(11) BODY(12) BODY(13) \
        default:                     \
            return cudaErrorInvalidValue; \
    }

cudaError_t launch_keygen(const LaunchInfo& li, uint64_t seed, uint64_t* key, cudaStream_t st) {
#define B(L)                                                                    \
    case L:                                                                     \
        k_keygen<L><<<li.r, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, seed, key); \
        break;
    HW_DISPATCH(li.log_n, B)
#undef B
    return HW_LAUNCHED();
}

cudaError_t launch_encode(const LaunchInfo& li, const uint8_t* values, size_t n, uint8_t* bits,
                          cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    size_t total = n * (size_t)li.n_data;
    size_t blocks = (total + 255) / 256;
    if (blocks > (size_t)li.sm_count * 32) blocks = (size_t)li.sm_count * 32;
    k_encode<<<(unsigned)blocks, 256, 0, st>>>(li.dctx, values, n, bits);
    return HW_LAUNCHED();
}

cudaError_t launch_encrypt(const LaunchInfo& li, const uint64_t* key, const uint8_t* bits,
                           const uint32_t* labels, size_t n, uint64_t seed, uint64_t first,
                           uint64_t* out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int slot0 = labels ? 0 : li.L;
    const int n_enc = li.n_slots - slot0;
    const size_t blocks = n * (size_t)n_enc * 2 * li.dnum;
    if (blocks >= ((size_t)1 << 31)) return cudaErrorInvalidValue;
    cudaError_t e = li.ext->encrypt(li, key, bits, labels, slot0, n_enc, (unsigned)blocks, seed, first,
                                    out, st);
    (*li.launches)++;
    return e;
}

cudaError_t launch_decrypt_rlwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                                size_t count, int64_t* out, uint64_t* phase_scratch,
                                size_t chunk, cudaStream_t st) {
    for (size_t t0 = 0; t0 < count; t0 += chunk) {
        size_t m = count - t0 < chunk ? count - t0 : chunk;
#define B(L)                                                                              \
    case L:                                                                               \
        k_rlwe_phase<L><<<(unsigned)(m * li.r), Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(     \
            li.dctx, key, ct + t0 * li.rlwe_words, phase_scratch);                        \
        break;
        HW_DISPATCH(li.log_n, B)
#undef B
        (*li.launches)++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        size_t total = m * li.n;
        size_t blocks = (total + 255) / 256;
        if (blocks > (size_t)li.sm_count * 32) blocks = (size_t)li.sm_count * 32;
        k_decode_phase<<<(unsigned)blocks, 256, 0, st>>>(li.dctx, phase_scratch, m,
                                                          out + t0 * li.n);
        (*li.launches)++;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The model's counters: the phases of whole RAMs (as many as the phase
// scratch holds), then the counters those RAMs store.
cudaError_t launch_decrypt_model(const LaunchInfo& li, const uint64_t* key, const uint64_t* model, int a,
                                 int64_t* out, uint64_t* phase_scratch, size_t chunk, cudaStream_t st) {
    const int rams = (int)(chunk / (size_t)li.k1) < 1 ? 1 : (int)(chunk / (size_t)li.k1);
    for (int j0 = 0; j0 < li.k0; j0 += rams) {
        const int nj = li.k0 - j0 < rams ? li.k0 - j0 : rams;
        const size_t m = (size_t)nj * li.k1;
#define B(L)                                                                              \
    case L:                                                                               \
        k_rlwe_phase<L><<<(unsigned)(m * li.r), Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(     \
            li.dctx, key, model + (size_t)j0 * li.k1 * li.rlwe_words, phase_scratch);     \
        break;
        HW_DISPATCH(li.log_n, B)
#undef B
        (*li.launches)++;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t total = (size_t)li.n_classes * nj << a;
        size_t blocks = (total + 255) / 256;
        if (blocks > (size_t)li.sm_count * 32) blocks = (size_t)li.sm_count * 32;
        k_decode_model<<<(unsigned)blocks, 256, 0, st>>>(li.dctx, phase_scratch, j0, nj, out);
        (*li.launches)++;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_decrypt_lwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                               size_t count, int64_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_decrypt_lwe<<<(unsigned)count, 256, 0, st>>>(li.dctx, key, ct, out);
    return HW_LAUNCHED();
}

cudaError_t launch_pdact(const LaunchInfo& li, const int64_t* counts, size_t n, int64_t* scores,
                         int32_t* labels, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_pdact<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(li.dctx, counts, (int)n, scores, labels);
    return HW_LAUNCHED();
}

cudaError_t launch_pdact_balanced(const LaunchInfo& li, const int64_t* counts, const int64_t* class_counts,
                                  size_t n, int64_t* scores, int32_t* labels, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_pdact_balanced<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(li.dctx, counts, class_counts, (int)n,
                                                                    scores, labels);
    return HW_LAUNCHED();
}

cudaError_t launch_export_rgsw(const LaunchInfo& li, const uint64_t* rgsw, size_t count,
                               uint64_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    size_t polys = count * 2 * li.dnum * 2 * li.r;
#define B(L)                                                                                      \
    case L:                                                                                       \
        k_export_rgsw<L><<<(unsigned)polys, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, rgsw, out); \
        break;
    HW_DISPATCH(li.log_n, B)
#undef B
    return HW_LAUNCHED();
}

cudaError_t launch_import_rgsw(const LaunchInfo& li, const uint64_t* in, size_t count, uint64_t* rgsw,
                               cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    size_t polys = count * 2 * li.dnum * 2 * li.r;
#define B(L)                                                                                      \
    case L:                                                                                       \
        k_import_rgsw<L><<<(unsigned)polys, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, in, rgsw); \
        break;
    HW_DISPATCH(li.log_n, B)
#undef B
    return HW_LAUNCHED();
}

size_t hw_plain_words_li(const LaunchInfo& li) {
    const int zt = li.z > li.L ? li.z - li.L : 0;
    return (size_t)li.k0 * li.n_classes * ((size_t)1 << zt) * li.r * li.n;
}

cudaError_t launch_plain_load(const LaunchInfo& li, const int64_t* counts, uint64_t* plain, cudaStream_t st) {
    const size_t polys = hw_plain_words_li(li) / li.n;
    if (polys == 0) return cudaSuccess;
    if (polys >= ((size_t)1 << 31)) return cudaErrorInvalidValue;
#define B(L)                                                                                  \
    case L:                                                                                   \
        k_plain_load<L><<<(unsigned)polys, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, counts, plain); \
        break;
    HW_DISPATCH(li.log_n, B)
#undef B
    return HW_LAUNCHED();
}

extern cudaError_t hw_ntt_kernels_init(const LaunchInfo& li);

cudaError_t hw_kernels_init(const LaunchInfo& li) {
    cudaError_t e = cudaSuccess;
#define A(K, L, BYTES) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(BYTES));
#define X(L)                                   \
    case L:                                    \
        A(k_keygen, L, Geo<L>::XCHG_BYTES)     \
        A(k_rlwe_phase, L, Geo<L>::XCHG_BYTES) \
        A(k_export_rgsw, L, Geo<L>::XCHG_BYTES) \
        A(k_import_rgsw, L, Geo<L>::XCHG_BYTES) \
        A(k_plain_load, L, Geo<L>::XCHG_BYTES) \
        break;
    switch (li.log_n) {
        HW_FOR_EACH_LOGN(X)
        default:
            return cudaErrorInvalidValue;
    }
#undef X
#undef A
    if (e == cudaSuccess) e = li.ext->init();
    if (e == cudaSuccess) e = hw_ntt_kernels_init(li);
    if (e == cudaSuccess) e = hw_pack_kernels_init(li);
    return e;
}
