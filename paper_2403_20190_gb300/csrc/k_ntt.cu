// k_ntt.cu -- the batched negacyclic transform behind hw_ntt_forward /
// hw_ntt_inverse, in the context's variant: 2^LOGE residues per thread
// (radix of the register-level butterflies) and 64-bit or, when every
// q_i < 2^30, 32-bit arithmetic.  Every variant computes the same values.
#include "hw_internal.cuh"
#include "hw_launch.h"

// One block per polynomial (prime t mod r), in place.  Forward takes natural
// order and leaves the evaluation order of the library (position E*t + e
// holds the value at psi^(2 brv(E*t + e) + 1)); inverse undoes it.  Values
// are fully reduced.  Positions E*tid + e go through warp transposes so the
// global accesses are coalesced: the store stages in the exchange buffer the
// last exchange did not use (read two exchanges ago, before a barrier); the
// load stages in b1 and the transform's first exchange then takes b0.  Every
// global read precedes the first barrier and every write follows the last
// one, so the transform runs in place.
template <int LOGN, int LOGE>
__global__ void __launch_bounds__(Ring<LOGN, LOGE>::T)
    k_ntt_batch(const DevCtx* __restrict__ Cp, u64* __restrict__ poly, int inverse) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    constexpr int PD = Ring<LOGN, LOGE>::PADDED;
    Xchg xc{smem, smem + PD, PD, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    const size_t t = blockIdx.x;
    const int j = (int)(t % C.r);
    const PrimeConst P = C.P[j];
    u64* p = poly + t * N;
    u64 v[1][E];
    if (!inverse) {
#pragma unroll
        for (int kk = 0; kk < E; kk++) v[0][kk] = p[tid + kk * T];
        ntt_fwd<LOGN, LOGE, 1>(v, xc, C, j);
#pragma unroll
        for (int e = 0; e < E; e++) v[0][e] = reduce_full(v[0][e], P);
        if constexpr (T >= 32) {
            warp_store_positions<E>(p, v[0], xc.next());
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) p[E * tid + e] = v[0][e];
        }
    } else {
        if constexpr (T >= 32) {
            warp_load_positions<E>(p, v[0], xc.b1);
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) v[0][e] = p[E * tid + e];
        }
#pragma unroll
        for (int e = 0; e < E; e++) v[0][e] = shoup_mul_lazy(v[0][e], C.n_inv[j], C.n_inv_s[j], P.q);
        ntt_inv<LOGN, LOGE, 1>(v, xc, C, j);
#pragma unroll
        for (int kk = 0; kk < E; kk++) p[tid + kk * T] = v[0][kk] >= P.q ? v[0][kk] - P.q : v[0][kk];
    }
}

// The same transform in 32-bit arithmetic (Harvey butterflies, values < 4q
// < 2^32): same evaluation order and results, about a third of the integer
// instructions.  The 32-bit exchanges use the first half of each 64-bit
// buffer; the warp transposes stage 64-bit words in a whole buffer.
template <int LOGN, int LOGE>
__global__ void __launch_bounds__(Ring<LOGN, LOGE>::T)
    k_ntt_batch32(const DevCtx* __restrict__ Cp, u64* __restrict__ poly, int inverse) {
    extern __shared__ u64 smem[];
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    constexpr int PD = Ring<LOGN, LOGE>::PADDED;
    Xchg xc{smem, smem + PD, PD, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    const size_t t = blockIdx.x;
    const int j = (int)(t % C.r);
    const u32 q = (u32)C.P[j].q, q2 = 2 * q;
    u64* p = poly + t * N;
    u32 v[1][E];
    u64 o[E];
    if (!inverse) {
#pragma unroll
        for (int kk = 0; kk < E; kk++) v[0][kk] = (u32)p[tid + kk * T];
        fwd_from32<LOGN, LOGE, 1, 0>(v, xc, C.tw32_fwd + (size_t)j * N, q, q2);
#pragma unroll
        for (int e = 0; e < E; e++) {
            const u32 x = v[0][e] >= q2 ? v[0][e] - q2 : v[0][e];
            o[e] = x >= q ? x - q : x;
        }
        if constexpr (T >= 32) {
            warp_store_positions<E>(p, o, xc.next());
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) p[E * tid + e] = o[e];
        }
    } else {
        if constexpr (T >= 32) {
            warp_load_positions<E>(p, o, xc.b1);
        } else {
#pragma unroll
            for (int e = 0; e < E; e++) o[e] = p[E * tid + e];
        }
#pragma unroll
        for (int e = 0; e < E; e++) v[0][e] = shoup32_lazy((u32)o[e], C.n_inv32[j], C.n_inv32_s[j], q);
        inv_from32<LOGN, LOGE, 1, 0>(v, xc, C.tw32_inv + (size_t)j * N, q, q2);
#pragma unroll
        for (int kk = 0; kk < E; kk++) p[tid + kk * T] = v[0][kk] >= q ? v[0][kk] - q : v[0][kk];
    }
}

template <int LOGN, int LOGE, int W32>
struct NttVariant {
    static constexpr int T = Ring<LOGN, LOGE>::T;
    static constexpr size_t SMEM = 2 * (size_t)Ring<LOGN, LOGE>::PADDED * sizeof(u64);
    static cudaError_t init() {
        if constexpr (W32)
            return cudaFuncSetAttribute(k_ntt_batch32<LOGN, LOGE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        else
            return cudaFuncSetAttribute(k_ntt_batch<LOGN, LOGE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    }
    static cudaError_t launch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                              cudaStream_t st) {
        if constexpr (W32)
            k_ntt_batch32<LOGN, LOGE><<<(unsigned)count, T, SMEM, st>>>(li.dctx, poly, inverse);
        else
            k_ntt_batch<LOGN, LOGE><<<(unsigned)count, T, SMEM, st>>>(li.dctx, poly, inverse);
        return cudaGetLastError();
    }
};

// Calls NttVariant<L, loge, limbs == 1>::F(args...) for the context's variant.
#define HW_NTT_SELECT(li, F, ...)                                                          \
    switch (li.log_n) {                                                                    \
        HW_NTT_CASE(6, F, __VA_ARGS__) HW_NTT_CASE(7, F, __VA_ARGS__)                      \
        HW_NTT_CASE(8, F, __VA_ARGS__) HW_NTT_CASE(9, F, __VA_ARGS__)                      \
        HW_NTT_CASE(10, F, __VA_ARGS__) HW_NTT_CASE(11, F, __VA_ARGS__)                    \
        HW_NTT_CASE(12, F, __VA_ARGS__) HW_NTT_CASE(13, F, __VA_ARGS__)                    \
        default:                                                                           \
            return cudaErrorInvalidValue;                                                  \
    }
#define HW_NTT_CASE(L, F, ...)                                                              \
    case L:                                                                                 \
        if (li.ntt_loge == 3)                                                               \
            return li.ntt_limbs == 1 ? NttVariant<L, 3, 1>::F(__VA_ARGS__)                  \
                                     : NttVariant<L, 3, 0>::F(__VA_ARGS__);                 \
        return li.ntt_limbs == 1 ? NttVariant<L, 4, 1>::F(__VA_ARGS__)                      \
                                 : NttVariant<L, 4, 0>::F(__VA_ARGS__);

cudaError_t hw_ntt_kernels_init(const LaunchInfo& li) { HW_NTT_SELECT(li, init, ) }

cudaError_t launch_ntt_batch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                             cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    (*li.launches)++;
    HW_NTT_SELECT(li, launch, li, poly, count, inverse, st)
}
