// k_pack.cu -- PackingKeySwitching (Section 2.4): the responses of a test
// sample (k = l * k0 LWE ciphertexts, one per class and RAM) packed into one
// RLWE encrypting sum_i u_i X^i, with a key-switching key of N * dnum RLWE
// rows KS_{x,rho} encrypting s_x * g_rho:
//   C = sum_i X^i (0, b_i) - sum_{x, rho} KS_{x,rho} * D_{x,rho}(X),
//   D_{x,rho}(X) = sum_i Dec_rho(a_{i,x}) X^i.
// Each D_{x,rho} is one transform per prime and a multiply-accumulate with
// the key row in evaluation form; the key and every transform use the
// 16-residues-per-thread geometry (thread-major evaluation layout).
#include "cdt.cuh"
#include "hw_internal.cuh"
#include "hw_launch.h"

#define HW_PACK_CHUNKS 256

// Key row (x, rho) at prime j: a from the KSK_A stream (two words per
// coefficient), e from the KSK_E stream (one integer polynomial per row),
// b = a s + e + s_x g_rho; stored in evaluation form, Montgomery
// representation.  One block per (row, prime).
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_ksk_gen(const DevCtx* __restrict__ Cp, const u64* __restrict__ key, u64 seed, u64* __restrict__ ksk) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const size_t row = blockIdx.x / r;
    const int j = (int)(blockIdx.x % r);
    const int x = (int)(row / C.dnum), rho = (int)(row % C.dnum);
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    u64 va[16], ve[16];
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
        const int k = tid + kk * T;
        const Philox4 wa = hw_draw(seed, HW_TAG_KSK_A, (u64)(k >> 1), (u64)(row * r + j), 0);
        va[kk] = reduce128(wa.v[2 * (k & 1)], wa.v[2 * (k & 1) + 1], P);
        const Philox4 we = hw_draw(seed, HW_TAG_KSK_E, (u64)(k >> 2), (u64)row, 0);
        ve[kk] = from_signed((int64_t)gaussian_from_word(we.v[k & 3]), q);
    }
    ntt_fwd1<LOGN>(va, xc, C, j);
    ntt_fwd1<LOGN>(ve, xc, C, j);
    // the constant s_x g_rho, only at the gadget row's prime
    const u64 m = (j == rho / C.dpp) ? mont_mul(key[(size_t)j * N + x], to_mont(C.gconst[rho], P), P) : 0;
    const size_t rl = C.rlwe_words;
    u64* da = ksk + row * rl + (size_t)(0 * r + j) * N;
    u64* db = ksk + row * rl + (size_t)(1 * r + j) * N;
#pragma unroll
    for (int e = 0; e < 16; e++) {
        const u64 sM = key[(size_t)(r + j) * N + eval_addr(16 * tid + e, LOGN, C.ext_loge)];
        const u64 a = reduce_full(va[e], P);
        const u64 b = add_mod(add_mod(mont_mul(a, sM, P), reduce_full(ve[e], P), q), m, q);
        da[e * T + tid] = to_mont(a, P);
        db[e * T + tid] = to_mont(b, P);
    }
}

// One sample's responses (k LWEs of r*(N+1) words) to A[j][x][i] = a_{i,x}
// at prime j (0 for i >= k), by 32 x 32 tiles through shared memory.
__global__ void k_pack_transpose(const DevCtx* __restrict__ Cp, const u64* __restrict__ resp, int k,
                                 u64* __restrict__ A) {
    __shared__ u64 tile[32][33];
    const DevCtx& C = *Cp;
    const int N = C.n;
    const size_t lw = C.lwe_words;
    const int x0 = blockIdx.x * 32, i0 = blockIdx.y * 32, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int iy = ty; iy < 32; iy += blockDim.y) {
        const int i = i0 + iy;
        tile[iy][tx] = i < k ? resp[(size_t)i * lw + (size_t)j * (N + 1) + x0 + tx] : 0;
    }
    __syncthreads();
    for (int xy = ty; xy < 32; xy += blockDim.y)
        A[((size_t)j * N + x0 + xy) * N + i0 + tx] = tile[tx][xy];
}

// B[j][i] = b_i at prime j (0 for i >= k).
__global__ void k_pack_b(const DevCtx* __restrict__ Cp, const u64* __restrict__ resp, int k,
                         u64* __restrict__ B) {
    const DevCtx& C = *Cp;
    const int N = C.n;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < C.r * N; idx += gridDim.x * blockDim.x) {
        const int j = idx / N, i = idx % N;
        B[idx] = i < k ? resp[(size_t)i * C.lwe_words + (size_t)j * (N + 1) + N] : 0;
    }
}

// Partial sums over a chunk of (x, rho) pairs at prime j:
// sum KS_{x,rho} * D_{x,rho} in evaluation form (both components).
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_pack_mac(const DevCtx* __restrict__ Cp, const u64* __restrict__ ksk, const u64* __restrict__ A,
               u64* __restrict__ partial) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const int ch = blockIdx.x / r, j = (int)(blockIdx.x % r);
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    const size_t rl = C.rlwe_words;
    const int pairs = N * C.dnum;
    const int per = (pairs + HW_PACK_CHUNKS - 1) / HW_PACK_CHUNKS;
    const int p0 = ch * per, p1 = p0 + per < pairs ? p0 + per : pairs;
    u64 acc[2][16];
#pragma unroll
    for (int e = 0; e < 16; e++) acc[0][e] = acc[1][e] = 0;
    for (int pr = p0; pr < p1; pr++) {
        const int x = pr / C.dnum, rho = pr % C.dnum;
        const int gi = rho / C.dpp, gk = rho % C.dpp;
        const u64 qi = C.P[gi].q;
        const u64* Arow = A + ((size_t)gi * N + x) * N;
        u64 v[16];
#pragma unroll
        for (int kk = 0; kk < 16; kk++)
            v[kk] = lift_small(gadget_digit(centre(Arow[tid + kk * T], qi), gk, C.dpp, C.log_beta), q);
        ntt_fwd1<LOGN>(v, xc, C, j);
        const u64* ka = ksk + (size_t)pr * rl + (size_t)(0 * r + j) * N + tid;
        const u64* kb = ksk + (size_t)pr * rl + (size_t)(1 * r + j) * N + tid;
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const u64 d = v[e], wa = __ldg(ka + e * T), wb = __ldg(kb + e * T);
            acc[0][e] = add_mod(acc[0][e], redc(__umul64hi(d, wa), d * wa, P), q);
            acc[1][e] = add_mod(acc[1][e], redc(__umul64hi(d, wb), d * wb, P), q);
        }
    }
#pragma unroll
    for (int comp = 0; comp < 2; comp++)
#pragma unroll
        for (int e = 0; e < 16; e++)
            partial[(((size_t)ch * 2 + comp) * r + j) * N + e * T + tid] = acc[comp][e];
}

// Sum of the partials, inverse transform, and C = (-S_a, B - S_b).
template <int LOGN>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    k_pack_finish(const DevCtx* __restrict__ Cp, const u64* __restrict__ partial, const u64* __restrict__ B,
                  u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = Ring<LOGN>::T;
    Xchg xc{smem, smem + Ring<LOGN>::PADDED, Ring<LOGN>::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const int comp = blockIdx.x / r, j = (int)(blockIdx.x % r);
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    u64 v[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
        u64 s = 0;
        for (int ch = 0; ch < HW_PACK_CHUNKS; ch++)
            s = add_mod(s, partial[(((size_t)ch * 2 + comp) * r + j) * N + e * T + tid], q);
        v[e] = shoup_mul_lazy(s, C.n_inv[j], C.n_inv_s[j], q);
    }
    ntt_inv1<LOGN>(v, xc, C, j);
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
        const int y = tid + kk * T;
        const u64 val = v[kk] >= q ? v[kk] - q : v[kk];
        out[(size_t)(comp * r + j) * N + y] = comp == 0 ? neg_mod(val, q) : sub_mod(B[(size_t)j * N + y], val, q);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define HW_PACK_DISPATCH(logn, BODY) \
    switch (logn) {                  \
        BODY(6) BODY(7) BODY(8) BODY(9) BODY(10) BODY(11) BODY(12) BODY(13) \
        default:                     \
            return cudaErrorInvalidValue; \
    }

size_t hw_pack_scratch_words_li(const LaunchInfo& li) {
    const size_t N = (size_t)li.n, r = (size_t)li.r;
    return r * N * N + r * N + (size_t)HW_PACK_CHUNKS * 2 * r * N;
}

cudaError_t launch_ksk_gen(const LaunchInfo& li, const uint64_t* key, uint64_t seed, uint64_t* ksk,
                           cudaStream_t st) {
    const size_t blocks = (size_t)li.n * li.dnum * li.r;
#define B(L)                                                                                        \
    case L:                                                                                         \
        k_ksk_gen<L><<<(unsigned)blocks, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, key, seed, ksk); \
        break;
    HW_PACK_DISPATCH(li.log_n, B)
#undef B
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t launch_pack(const LaunchInfo& li, const uint64_t* ksk, const uint64_t* resp, size_t n,
                        uint64_t* packed, uint64_t* scratch, cudaStream_t st) {
    const int N = li.n, r = li.r;
    const int k = li.n_classes * li.k0;
    u64* A = scratch;
    u64* Bv = A + (size_t)r * N * N;
    u64* partial = Bv + (size_t)r * N;
    for (size_t s = 0; s < n; s++) {
        const u64* rs = resp + s * (size_t)k * li.lwe_words;
        u64* out = packed + s * li.rlwe_words;
        k_pack_transpose<<<dim3(N / 32, N / 32, r), dim3(32, 8), 0, st>>>(li.dctx, rs, k, A);
        k_pack_b<<<(unsigned)((r * N + 255) / 256), 256, 0, st>>>(li.dctx, rs, k, Bv);
#define B(L)                                                                                          \
    case L:                                                                                           \
        k_pack_mac<L><<<HW_PACK_CHUNKS * r, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, ksk, A, partial); \
        k_pack_finish<L><<<2 * r, Geo<L>::T, Geo<L>::XCHG_BYTES, st>>>(li.dctx, partial, Bv, out);        \
        break;
        HW_PACK_DISPATCH(li.log_n, B)
#undef B
        (*li.launches) += 4;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t hw_pack_kernels_init(const LaunchInfo& li) {
    cudaError_t e = cudaSuccess;
#define A(K, L) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo<L>::XCHG_BYTES);
#define X(L)                  \
    case L:                   \
        A(k_ksk_gen, L)       \
        A(k_pack_mac, L)      \
        A(k_pack_finish, L)   \
        break;
    switch (li.log_n) {
        HW_FOR_EACH_LOGN(X)
        default:
            return cudaErrorInvalidValue;
    }
#undef X
#undef A
    return e;
}
