// k_crypto.cu -- key generation, client encoding, RGSW encryption,
// decryption (phase, CRT, rounding), PD-act and transform utilities.
#include "cdt_table.h"
#include "hw_internal.cuh"
#include "hw_launch.h"

__constant__ u64 c_cdt[HW_CDT_LEN];

// Discrete Gaussian G(sigma) by inversion of the cumulative table on the top
// 63 bits of a uniform word: -19 plus the number of thresholds <= u.
__device__ __forceinline__ int gaussian_from_word(u64 w) {
    const u64 u = w >> 1;
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < HW_CDT_LEN; t++) cnt += (u >= c_cdt[t]) ? 1 : 0;
    return cnt - HW_CDT_SUPPORT;
}

// ---------------------------------------------------------------------------
// SecretKeyGen: ternary S_1; key = [r][N] residues, then [r][N] evaluation
// form in Montgomery representation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_keygen(const DevCtx* __restrict__ Cp, u64 seed, u64* __restrict__ key) {
    extern __shared__ u64 smem[];
    const DevCtx& C = *Cp;
    const int j = blockIdx.x, n = C.n, T = blockDim.x;
    const PrimeConst P = C.P[j];
    for (int k = threadIdx.x; k < n; k += T) {
        Philox4 w = hw_draw(seed, HW_TAG_KEY, (u64)k >> 2, 0, 0);
        u64 v = w.v[k & 3] % 3;
        u64 res = v == 0 ? 0 : (v == 1 ? 1 : P.q - 1);
        key[(size_t)j * n + k] = res;
        smem[k] = res;
    }
    __syncthreads();
    ntt_forward_block(smem, C, j);
    for (int k = threadIdx.x; k < n; k += T) key[(size_t)(C.r + j) * n + k] = to_mont(smem[k], P);
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
// EncRGSW.  One block per (sample, bit slot, row).  Row rho < dnum encrypts
// (a, a*s + e + m*g_rho), row dnum+rho encrypts (a + m*g_rho, a*s + e); the
// gadget value g_rho sits at prime rho/dpp only.  a is uniform per prime
// (two 64-bit words -> 128-bit value mod q), e is one integer polynomial for
// all primes.  Rows are stored in evaluation form, Montgomery representation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_encrypt(const DevCtx* __restrict__ Cp, const u64* __restrict__ key,
                          const uint8_t* __restrict__ bits, const uint32_t* __restrict__ labels,
                          int slot0, int n_enc_slots, u64 seed, u64 first, u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    const DevCtx& C = *Cp;
    const int n = C.n, r = C.r, T = blockDim.x, tid = threadIdx.x;
    const int rows = 2 * C.dnum;
    const size_t bid = blockIdx.x;
    const int row = (int)(bid % rows);
    const size_t rest = bid / rows;
    const int slot = slot0 + (int)(rest % n_enc_slots);
    const size_t i = rest / n_enc_slots;
    const int bit = slot < C.L ? (int)((labels[i] >> slot) & 1u)
                               : (int)bits[i * C.n_data + (slot - C.L)];
    const u64 stream = (first + i) * (u64)C.n_slots + (u64)slot;
    u64* A = smem;
    u64* E = smem + n;
    int8_t* ebuf = (int8_t*)(smem + 2 * n);
    for (int c0 = tid; c0 < n / 4; c0 += T) {
        Philox4 w = hw_draw(seed, HW_TAG_RGSW_E, (u64)c0, (u64)row, stream);
#pragma unroll
        for (int t = 0; t < 4; t++) ebuf[4 * c0 + t] = (int8_t)gaussian_from_word(w.v[t]);
    }
    const int rho = row % C.dnum;
    const int gi = rho / C.dpp;
    u64* dst_row = out + i * C.sample_words + (size_t)slot * C.rgsw_words + (size_t)row * C.rlwe_words;
    for (int j = 0; j < r; j++) {
        const PrimeConst P = C.P[j];
        const u64 q = P.q;
        __syncthreads();
        for (int c0 = tid; c0 < n / 2; c0 += T) {
            Philox4 w = hw_draw(seed, HW_TAG_RGSW_A, (u64)c0, (u64)(row * r + j), stream);
            A[2 * c0] = reduce128(w.v[0], w.v[1], P);
            A[2 * c0 + 1] = reduce128(w.v[2], w.v[3], P);
        }
        __syncthreads();
        for (int x = tid; x < n; x += T) E[x] = from_signed((int64_t)ebuf[x], q);
        __syncthreads();
        ntt_forward_block(A, C, j);
        ntt_forward_block(E, C, j);
        const u64 g = (bit && j == gi) ? C.gconst[rho] : 0;
        const u64* sM = key + (size_t)(r + j) * n;
        u64* da = dst_row + (size_t)(0 * r + j) * n;
        u64* db = dst_row + (size_t)(1 * r + j) * n;
        for (int x = tid; x < n; x += T) {
            u64 a = A[x];
            u64 b = add_mod(mont_mul(a, sM[x], P), E[x], q);
            // the evaluation form of the constant polynomial g is g everywhere
            if (row < C.dnum)
                b = add_mod(b, g, q);
            else
                a = add_mod(a, g, q);
            da[x] = to_mont(a, P);
            db[x] = to_mont(b, P);
        }
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
__global__ void __launch_bounds__(1024) k_rlwe_phase(const DevCtx* __restrict__ Cp, const u64* __restrict__ key,
                             const u64* __restrict__ ct, u64* __restrict__ ph) {
    extern __shared__ u64 smem[];
    const DevCtx& C = *Cp;
    const int n = C.n, r = C.r, T = blockDim.x, tid = threadIdx.x;
    const size_t t = blockIdx.x / r;
    const int j = blockIdx.x % r;
    const PrimeConst P = C.P[j];
    const u64* c = ct + t * C.rlwe_words;
    for (int x = tid; x < n; x += T) smem[x] = c[(size_t)j * n + x];
    __syncthreads();
    ntt_forward_block(smem, C, j);
    for (int x = tid; x < n; x += T) smem[x] = mont_mul(smem[x], key[(size_t)(r + j) * n + x], P);
    __syncthreads();
    ntt_inverse_block(smem, C, j);
    u64* dst = ph + (t * r + j) * n;
    for (int x = tid; x < n; x += T) dst[x] = sub_mod(c[(size_t)(r + j) * n + x], smem[x], P.q);
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

// ---------------------------------------------------------------------------
// Transform utilities.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_export_rgsw(const DevCtx* __restrict__ Cp, const u64* __restrict__ in,
                              u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    const DevCtx& C = *Cp;
    const int n = C.n;
    const size_t poly = blockIdx.x;  // [rgsw][row][comp][prime]
    const int j = (int)(poly % C.r);
    const PrimeConst P = C.P[j];
    for (int x = threadIdx.x; x < n; x += blockDim.x) smem[x] = from_mont(in[poly * n + x], P);
    __syncthreads();
    ntt_inverse_block(smem, C, j);
    for (int x = threadIdx.x; x < n; x += blockDim.x) out[poly * n + x] = smem[x];
}

__global__ void __launch_bounds__(1024) k_ntt_batch(const DevCtx* __restrict__ Cp, u64* __restrict__ poly, int inverse) {
    extern __shared__ u64 smem[];
    const DevCtx& C = *Cp;
    const int n = C.n;
    const size_t t = blockIdx.x;
    const int j = (int)(t % C.r);
    u64* p = poly + t * n;
    for (int x = threadIdx.x; x < n; x += blockDim.x) smem[x] = p[x];
    __syncthreads();
    if (inverse)
        ntt_inverse_block(smem, C, j);
    else
        ntt_forward_block(smem, C, j);
    for (int x = threadIdx.x; x < n; x += blockDim.x) p[x] = smem[x];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define HW_LAUNCHED() ((*li.launches)++, cudaGetLastError())

cudaError_t launch_keygen(const LaunchInfo& li, uint64_t seed, uint64_t* key, cudaStream_t st) {
    k_keygen<<<li.r, li.n / 8, (size_t)li.n * 8, st>>>(li.dctx, seed, key);
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
    const size_t smem = (size_t)2 * li.n * 8 + li.n;
    if (blocks >= ((size_t)1 << 31)) return cudaErrorInvalidValue;
    k_encrypt<<<(unsigned)blocks, li.n / 8, smem, st>>>(li.dctx, key, bits, labels, slot0, n_enc,
                                                       seed, first, out);
    return HW_LAUNCHED();
}

cudaError_t launch_decrypt_rlwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                                size_t count, int64_t* out, uint64_t* phase_scratch,
                                size_t chunk, cudaStream_t st) {
    for (size_t t0 = 0; t0 < count; t0 += chunk) {
        size_t m = count - t0 < chunk ? count - t0 : chunk;
        k_rlwe_phase<<<(unsigned)(m * li.r), li.n / 8, (size_t)li.n * 8, st>>>(
            li.dctx, key, ct + t0 * li.rlwe_words, phase_scratch);
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

cudaError_t launch_export_rgsw(const LaunchInfo& li, const uint64_t* rgsw, size_t count,
                               uint64_t* out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    size_t polys = count * 2 * li.dnum * 2 * li.r;
    k_export_rgsw<<<(unsigned)polys, li.n / 8, (size_t)li.n * 8, st>>>(li.dctx, rgsw, out);
    return HW_LAUNCHED();
}

cudaError_t launch_ntt_batch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                             cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    k_ntt_batch<<<(unsigned)count, li.n / 8, (size_t)li.n * 8, st>>>(li.dctx, poly, inverse);
    return HW_LAUNCHED();
}

extern cudaError_t hw_wisard_kernels_init();

cudaError_t hw_kernels_init(int log_n) {
    (void)log_n;
    cudaError_t e = cudaMemcpyToSymbol(c_cdt, hw_cdt_table, sizeof(u64) * HW_CDT_LEN);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_encrypt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * 8192 * 8 + 8192);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rlwe_phase, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_keygen, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_export_rgsw, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_ntt_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 8);
    if (e != cudaSuccess) return e;
    return hw_wisard_kernels_init();
}
