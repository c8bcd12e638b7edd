// k_pack.cu -- PackingKeySwitching (Section 2.4): the responses of a test
// sample (k = l * k0 LWE ciphertexts, one per class and RAM) packed into one
// RLWE encrypting sum_i u_i X^i, with a key-switching key of N * dnum RLWE
// rows KS_{x,rho} encrypting s_x * g_rho:
//   C = sum_i X^i (0, b_i) - sum_{x, rho} KS_{x,rho} * D_{x,rho}(X),
//   D_{x,rho}(X) = sum_i Dec_rho(a_{i,x}) X^i.
// Each D_{x,rho} is one transform per prime and a multiply-accumulate with
// the key row in evaluation form; the key and every transform use the
// 8-residues-per-thread geometry (PackGeo, thread-major evaluation layout).
#include "cdt.cuh"
#include "hw_internal.cuh"
#include "hw_launch.h"

#define HW_PACK_CHUNKS 256

// The key-switching kernels' transform geometry: 8 residues per thread (N/8
// threads), the widest blocks the transforms take, for latency hiding.
template <int LOGN>
struct PackGeo {
    static constexpr int E = 8;
    static constexpr int T = Ring<LOGN, 3>::T;
    static constexpr int PD = Ring<LOGN, 3>::PADDED;
    static constexpr size_t XCHG_BYTES = 2 * (size_t)PD * sizeof(u64);
};

// Key row (x, rho) at prime j: a from the KSK_A stream (two words per
// coefficient), e from the KSK_E stream (one integer polynomial per row),
// b = a s + e + s_x g_rho; stored in evaluation form, Montgomery
// representation.  One block per (row, prime).
template <int LOGN>
__global__ void __launch_bounds__(PackGeo<LOGN>::T)
    k_ksk_gen(const DevCtx* __restrict__ Cp, const u64* __restrict__ key, u64 seed, u64* __restrict__ ksk) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = PackGeo<LOGN>::T, E = PackGeo<LOGN>::E, PD = PackGeo<LOGN>::PD;
    Xchg xc{smem, smem + PD, PD, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const size_t row = blockIdx.x / r;
    const int j = (int)(blockIdx.x % r);
    const int x = (int)(row / C.dnum), rho = (int)(row % C.dnum);
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    // the constant s_x g_rho, only at the gadget row's prime
    const u64 m = (j == rho / C.dpp) ? mont_mul(key[(size_t)j * N + x], to_mont(C.gconst[rho], P), P) : 0;
    const size_t rl = C.rlwe_words;
    u64* da = ksk + row * rl + (size_t)(0 * r + j) * N;
    u64* db = ksk + row * rl + (size_t)(1 * r + j) * N;
    // a first: its row, and a s + s_x g_rho parked in the b row (each thread
    // rewrites only its own words), then e; one polynomial in registers
    u64 v[1][E];
#pragma unroll
    for (int kk = 0; kk < E; kk++) {
        const int k = tid + kk * T;
        const Philox4 wa = hw_draw(seed, HW_TAG_KSK_A, (u64)(k >> 1), (u64)(row * r + j), 0);
        v[0][kk] = reduce128(wa.v[2 * (k & 1)], wa.v[2 * (k & 1) + 1], P);
    }
    ntt_fwd<LOGN, 3, 1>(v, xc, C, j);
#pragma unroll
    for (int e = 0; e < E; e++) {
        const u64 sM = key[(size_t)(r + j) * N + eval_addr(E * tid + e, LOGN, C.ext_loge)];
        const u64 a = reduce_full(v[0][e], P);
        da[e * T + tid] = to_mont(a, P);
        db[e * T + tid] = add_mod(mont_mul(a, sM, P), m, q);
    }
#pragma unroll
    for (int kk = 0; kk < E; kk++) {
        const int k = tid + kk * T;
        const Philox4 we = hw_draw(seed, HW_TAG_KSK_E, (u64)(k >> 2), (u64)row, 0);
        v[0][kk] = from_signed((int64_t)gaussian_from_word(we.v[k & 3]), q);
    }
    ntt_fwd<LOGN, 3, 1>(v, xc, C, j);
#pragma unroll
    for (int e = 0; e < E; e++) db[e * T + tid] = to_mont(add_mod(db[e * T + tid], reduce_full(v[0][e], P), q), P);
}

// The responses of a group of samples (k LWEs of r*(N+1) words each) to
// A[s][j][x][i] = a_{i,x} of sample s at prime j, i < kp (kp = k rounded up
// to 32; 0 for i >= k), by 32 x 32 tiles through shared memory.  Grid z runs
// over (sample, prime).
__global__ void k_pack_transpose(const DevCtx* __restrict__ Cp, const u64* __restrict__ resp, int k, int kp,
                                 u64* __restrict__ A) {
    __shared__ u64 tile[32][33];
    const DevCtx& C = *Cp;
    const int N = C.n;
    const size_t lw = C.lwe_words;
    const int x0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    const int j = blockIdx.z % C.r;
    const size_t smp = blockIdx.z / C.r;
    const u64* rs = resp + smp * (size_t)k * lw;
    u64* As = A + smp * (size_t)C.r * N * kp;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int iy = ty; iy < 32; iy += blockDim.y) {
        const int i = i0 + iy;
        tile[iy][tx] = i < k ? rs[(size_t)i * lw + (size_t)j * (N + 1) + x0 + tx] : 0;
    }
    __syncthreads();
    for (int xy = ty; xy < 32; xy += blockDim.y)
        As[((size_t)j * N + x0 + xy) * kp + i0 + tx] = tile[tx][xy];
}

// B[s][j][i] = b_i of sample s at prime j (0 for i >= k).
__global__ void k_pack_b(const DevCtx* __restrict__ Cp, const u64* __restrict__ resp, int k, int n_smp,
                         u64* __restrict__ B) {
    const DevCtx& C = *Cp;
    const int N = C.n;
    const size_t total = (size_t)n_smp * C.r * N;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t smp = idx / ((size_t)C.r * N);
        const int j = (int)((idx / N) % C.r), i = (int)(idx % N);
        B[idx] = i < k ? resp[(smp * k + i) * C.lwe_words + (size_t)j * (N + 1) + N] : 0;
    }
}

// ntt_fwd<LOGN, 3, 1> for a polynomial whose upper half is zero (D has k_p
// <= N/2 coefficients) when the first round is the single stage 0
// (LOGN mod 3 = 1): that stage pairs x_p with x_{p+N/2} = 0, so it leaves
// x_p and writes x_p + 2q (the lazy form of x_p - w*0) without a multiply;
// the exchange and the remaining rounds are ntt_fwd's.
template <int LOGN>
__device__ __forceinline__ void fwd_upper_zero(u64 (&v)[1][8], Xchg& xc, const DevCtx& C, int j) {
    if constexpr (LOGN % 3 == 1) {
        constexpr int G = 4, R2 = FwdR<LOGN, 3, 1>::R, G2 = 8 >> R2;
        const u64 q = C.P[j].q, q2 = 2 * q;
#pragma unroll
        for (int gg = 0; gg < G; gg++) v[0][gg + G] = v[0][gg] + q2;
        u64* sm = xc.next();
        if (xc.b0 == xc.b1) __syncthreads();
#pragma unroll
        for (int gg = 0; gg < G; gg++)
#pragma unroll
            for (int e = 0; e < 2; e++) sm[padw<3>(fpos<LOGN, 3, 0, 1>(gg, e))] = v[0][gg + e * G];
        __syncthreads();
#pragma unroll
        for (int gg = 0; gg < G2; gg++)
#pragma unroll
            for (int e = 0; e < (1 << R2); e++) v[0][gg + e * G2] = sm[padw<3>(fpos<LOGN, 3, 1, R2>(gg, e))];
        fwd_from<LOGN, 3, 1, 1>(v, xc, C.tw_fwd + (size_t)j * Ring<LOGN>::N, q, q2);
    } else {
        ntt_fwd<LOGN, 3, 1>(v, xc, C, j);
    }
}

// Partial sums over a chunk of (x, rho) pairs at prime j:
// sum KS_{x,rho} * D_{x,rho} in evaluation form (both components).
template <int LOGN>
__global__ void __launch_bounds__(PackGeo<LOGN>::T)
    k_pack_mac(const DevCtx* __restrict__ Cp, const u64* __restrict__ ksk, const u64* __restrict__ A, int kp,
               int chunks, u64* __restrict__ partial) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = PackGeo<LOGN>::T, E = PackGeo<LOGN>::E, PD = PackGeo<LOGN>::PD;
    Xchg xc{smem, smem + PD, PD, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const int j = (int)(blockIdx.x % r);
    const int ch = (int)((blockIdx.x / r) % chunks);
    const size_t smp = blockIdx.x / ((size_t)r * chunks);
    A += smp * (size_t)r * N * kp;
    partial += smp * (size_t)chunks * 2 * r * N;
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    const size_t rl = C.rlwe_words;
    const int pairs = N * C.dnum;
    const int per = (pairs + chunks - 1) / chunks;
    const int p0 = ch * per, p1 = p0 + per < pairs ? p0 + per : pairs;
    // at N = 8192 the a component's accumulators live in the block's own
    // shared-memory slots (registers would spill); elsewhere in registers
    constexpr bool ACC_SMEM = LOGN >= 13;
    u64 acc[2][E];
    u64* acc0 = smem + 2 * PD + tid;
#pragma unroll
    for (int e = 0; e < E; e++) {
        acc[0][e] = acc[1][e] = 0;
        if (ACC_SMEM) acc0[e * T] = 0;
    }
    for (int pr = p0; pr < p1; pr++) {
        const int x = pr / C.dnum, rho = pr % C.dnum;
        const int gi = rho / C.dpp, gk = rho % C.dpp;
        const u64 qi = C.P[gi].q;
        const u64* Arow = A + ((size_t)gi * N + x) * kp;
        u64 v[1][E];
#pragma unroll
        for (int kk = 0; kk < E; kk++) {
            const int i = tid + kk * T;
            v[0][kk] = i < kp ? lift_small(gadget_digit(centre(Arow[i], qi), gk, C.dpp, C.log_beta), q) : 0;
        }
        if (LOGN % 3 == 1 && 2 * kp <= N)
            fwd_upper_zero<LOGN>(v, xc, C, j);
        else
            ntt_fwd<LOGN, 3, 1>(v, xc, C, j);
        const u64* ka = ksk + (size_t)pr * rl + (size_t)(0 * r + j) * N + tid;
        const u64* kb = ksk + (size_t)pr * rl + (size_t)(1 * r + j) * N + tid;
#pragma unroll
        for (int e = 0; e < E; e++) {
            const u64 d = v[0][e], wa = __ldg(ka + e * T), wb = __ldg(kb + e * T);
            if (ACC_SMEM)
                acc0[e * T] = add_mod(acc0[e * T], redc(__umul64hi(d, wa), d * wa, P), q);
            else
                acc[0][e] = add_mod(acc[0][e], redc(__umul64hi(d, wa), d * wa, P), q);
            acc[1][e] = add_mod(acc[1][e], redc(__umul64hi(d, wb), d * wb, P), q);
        }
    }
#pragma unroll
    for (int comp = 0; comp < 2; comp++)
#pragma unroll
        for (int e = 0; e < E; e++)
            partial[(((size_t)ch * 2 + comp) * r + j) * N + e * T + tid] =
                (ACC_SMEM && comp == 0) ? acc0[e * T] : acc[comp][e];
}

// Sum of the partials, inverse transform, and C = (-S_a, B - S_b).
template <int LOGN>
__global__ void __launch_bounds__(PackGeo<LOGN>::T)
    k_pack_finish(const DevCtx* __restrict__ Cp, const u64* __restrict__ partial, const u64* __restrict__ B,
                  int chunks, u64* __restrict__ out) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN>::N, T = PackGeo<LOGN>::T, E = PackGeo<LOGN>::E, PD = PackGeo<LOGN>::PD;
    Xchg xc{smem, smem + PD, PD, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r;
    const int j = (int)(blockIdx.x % r), comp = (int)((blockIdx.x / r) % 2);
    const size_t smp = blockIdx.x / ((size_t)2 * r);
    partial += smp * (size_t)chunks * 2 * r * N;
    B += smp * (size_t)r * N;
    out += smp * C.rlwe_words;
    const PrimeConst P = C.P[j];
    const u64 q = P.q;
    u64 v[1][E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        u64 s = 0;
        for (int ch = 0; ch < chunks; ch++)
            s = add_mod(s, partial[(((size_t)ch * 2 + comp) * r + j) * N + e * T + tid], q);
        v[0][e] = shoup_mul_lazy(s, C.n_inv[j], C.n_inv_s[j], q);
    }
    ntt_inv<LOGN, 3, 1>(v, xc, C, j);
#pragma unroll
    for (int kk = 0; kk < E; kk++) {
        const int y = tid + kk * T;
        const u64 val = v[0][kk] >= q ? v[0][kk] - q : v[0][kk];
        out[(size_t)(comp * r + j) * N + y] = comp == 0 ? neg_mod(val, q) : sub_mod(B[(size_t)j * N + y], val, q);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// k_pack_mac's shared memory: the exchange buffers, plus one accumulator
// component at N = 8192.
template <int LOGN>
constexpr size_t pack_mac_smem() {
    return PackGeo<LOGN>::XCHG_BYTES + (LOGN >= 13 ? (size_t)Ring<LOGN>::N * sizeof(u64) : 0);
}

#define HW_PACK_DISPATCH(logn, BODY) \
    switch (logn) {                  \
        BODY(6) BODY(7) BODY(8) BODY(9) BODY(10) BODY(11) BODY(12) BODY(13) \
        default:                     \
            return cudaErrorInvalidValue; \
    }

// A pass packs a group of S samples: per sample the transposed masks
// (r * N * kp words, kp = k rounded up to 32) and the b values (r * N), and
// the group's partial sums (chunks(S) * 2 * r * N words per sample), with
// chunks(S) picked so that the group's multiply-accumulate grid runs about
// eight blocks per SM.
static int pack_chunks(const LaunchInfo& li, size_t group) {
    const size_t want = (8 * (size_t)li.sm_count + group * li.r - 1) / (group * li.r);
    return want < 1 ? 1 : (want > HW_PACK_CHUNKS ? HW_PACK_CHUNKS : (int)want);
}

static size_t pack_kp(const LaunchInfo& li) { return ((size_t)li.n_classes * li.k0 + 31) / 32 * 32; }

size_t hw_pack_scratch_words_li(const LaunchInfo& li, size_t group) {
    if (group < 1) group = 1;
    const size_t N = (size_t)li.n, r = (size_t)li.r;
    return group * (r * N * pack_kp(li) + r * N + (size_t)pack_chunks(li, group) * 2 * r * N);
}

cudaError_t launch_ksk_gen(const LaunchInfo& li, const uint64_t* key, uint64_t seed, uint64_t* ksk,
                           cudaStream_t st) {
    const size_t blocks = (size_t)li.n * li.dnum * li.r;
#define B(L)                                                                                        \
    case L:                                                                                         \
        k_ksk_gen<L><<<(unsigned)blocks, PackGeo<L>::T, PackGeo<L>::XCHG_BYTES, st>>>(li.dctx, key, seed, ksk); \
        break;
    HW_PACK_DISPATCH(li.log_n, B)
#undef B
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t launch_pack(const LaunchInfo& li, const uint64_t* ksk, const uint64_t* resp, size_t n,
                        uint64_t* packed, uint64_t* scratch, size_t scratch_words, cudaStream_t st) {
    const int N = li.n, r = li.r;
    const int k = li.n_classes * li.k0;
    const int kp = (int)pack_kp(li);
    // the largest group the scratch holds (the caller checked one sample fits)
    size_t group = n;
    while (group > 1 && hw_pack_scratch_words_li(li, group) > scratch_words) group--;
    for (size_t s0 = 0; s0 < n; s0 += group) {
        const size_t S = n - s0 < group ? n - s0 : group;
        const int chunks = pack_chunks(li, S);
        u64* A = scratch;
        u64* Bv = A + S * (size_t)r * N * kp;
        u64* partial = Bv + S * (size_t)r * N;
        const u64* rs = resp + s0 * (size_t)k * li.lwe_words;
        u64* out = packed + s0 * li.rlwe_words;
        k_pack_transpose<<<dim3(N / 32, kp / 32, (unsigned)(r * S)), dim3(32, 8), 0, st>>>(li.dctx, rs, k, kp, A);
        size_t bb = (S * r * N + 255) / 256;
        if (bb > (size_t)li.sm_count * 32) bb = (size_t)li.sm_count * 32;
        k_pack_b<<<(unsigned)bb, 256, 0, st>>>(li.dctx, rs, k, (int)S, Bv);
#define B(L)                                                                                            \
    case L:                                                                                             \
        k_pack_mac<L><<<(unsigned)(S * chunks * r), PackGeo<L>::T, pack_mac_smem<L>(), st>>>(li.dctx, ksk, A, kp, \
                                                                                       chunks, partial); \
        k_pack_finish<L><<<(unsigned)(S * 2 * r), PackGeo<L>::T, PackGeo<L>::XCHG_BYTES, st>>>(li.dctx, partial, Bv, \
                                                                                     chunks, out);     \
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PackGeo<L>::XCHG_BYTES);
#define X(L)                  \
    case L:                   \
        A(k_ksk_gen, L)       \
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pack_mac<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pack_mac_smem<L>()); \
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
