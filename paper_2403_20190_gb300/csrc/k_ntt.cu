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

// ---------------------------------------------------------------------------
// Bulk-asynchronous form of the same transforms (the default for the 32-bit
// arithmetic when the buffer is 16-byte aligned): a persistent grid, each
// block streaming its
// polynomials through two shared-memory stages.  One thread issues the
// bulk copy (cp.async.bulk) of polynomial k+1 into one stage, completing on
// that stage's mbarrier, while the block transforms polynomial k in the
// other; the result goes back in place with a bulk store from the stage it
// was read from.  Stage reuse: the load into a stage is issued only after
// the store that last read it has finished reading (wait_group.read), and
// after a proxy fence.  Every wait on an mbarrier is bounded: if one runs
// out the whole block stops, counts the event in g_ntt_wait_timeouts, waits
// (bounded again) for its copies in flight and returns.  Same values as
// k_ntt_batch / k_ntt_batch32.
// ---------------------------------------------------------------------------
__device__ unsigned int g_ntt_wait_timeouts;

namespace {

__device__ __forceinline__ unsigned s_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(u64* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(u64* bar, unsigned parity) {
    for (int i = 0; i < (1 << 22); i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared, completing `bytes` on the mbarrier (16-byte aligned
// addresses, bytes a multiple of 16)
__device__ __forceinline__ void bulk_load(u64* dst, const u64* src, unsigned bytes, u64* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s_addr(dst)),
        "l"(src), "r"(bytes), "r"(s_addr(bar))
        : "memory");
}
// shared -> global as one bulk group
__device__ __forceinline__ void bulk_store(u64* dst, const u64* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(s_addr(src)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

}  // namespace

template <int LOGN, int LOGE>
struct NttBulkCfg {
    static constexpr int N = Ring<LOGN, LOGE>::N;
    static constexpr int PD = Ring<LOGN, LOGE>::PADDED;
    // two exchange buffers when they fit beside the two stages, else one
    static constexpr bool ONE_XCHG = (size_t)(2 * N + 2 * PD) * 8 + 16 > 227 * 1024;
    static constexpr size_t SMEM = (size_t)(2 * N + (ONE_XCHG ? 1 : 2) * PD) * 8 + 16;
};

template <int LOGN, int LOGE, int W32>
__global__ void __launch_bounds__(Ring<LOGN, LOGE>::T)
    k_ntt_bulk(const DevCtx* __restrict__ Cp, u64* __restrict__ poly, size_t count, int inverse) {
    extern __shared__ __align__(128) u64 smem_bulk[];
    u64* smem = smem_bulk;
    using B = NttBulkCfg<LOGN, LOGE>;
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE, PD = B::PD;
    constexpr unsigned BYTES = (unsigned)N * 8;
    u64* xb = smem + 2 * N;
    u64* bars = xb + (B::ONE_XCHG ? 1 : 2) * PD;
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    size_t item = blockIdx.x;
    if (tid == 0 && item < count) {
        mbar_expect_tx(&bars[0], BYTES);
        bulk_load(smem, poly + item * N, BYTES, &bars[0]);
    }
    int k = 0;
    bool failed = false, pending_next = false;
    for (; item < count; item += gridDim.x, k++) {
        const int s = k & 1;
        u64* st = smem + s * N;
        const size_t next = item + gridDim.x;
        pending_next = next < count;
        if (tid == 0 && pending_next) {
            u64* sn = smem + (s ^ 1) * N;
            bulk_wait_read();  // the store that last read this stage has read it
            proxy_fence();
            mbar_expect_tx(&bars[s ^ 1], BYTES);
            bulk_load(sn, poly + next * N, BYTES, &bars[s ^ 1]);
        }
        const bool ok = mbar_wait(&bars[s], (unsigned)(k >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        Xchg xc{xb, B::ONE_XCHG ? xb : xb + PD, PD, 0};
        const int j = (int)(item % C.r);
        const u64 q = C.P[j].q;
        if (!inverse) {
            u64 o[E];
            if constexpr (W32) {
                u32 v[1][E];
#pragma unroll
                for (int kk = 0; kk < E; kk++) v[0][kk] = (u32)st[tid + kk * T];
                fwd_from32<LOGN, LOGE, 1, 0>(v, xc, C.tw32_fwd + (size_t)j * N, (u32)q, 2 * (u32)q);
#pragma unroll
                for (int e = 0; e < E; e++) {
                    const u32 x = v[0][e] >= 2 * (u32)q ? v[0][e] - 2 * (u32)q : v[0][e];
                    o[e] = x >= (u32)q ? x - (u32)q : x;
                }
            } else {
                u64 v[1][E];
#pragma unroll
                for (int kk = 0; kk < E; kk++) v[0][kk] = st[tid + kk * T];
                ntt_fwd<LOGN, LOGE, 1>(v, xc, C, j);
#pragma unroll
                for (int e = 0; e < E; e++) o[e] = reduce_full(v[0][e], C.P[j]);
            }
            // every thread has read its input (the transform's barriers):
            // the results go to the same stage in evaluation order
            if constexpr (T >= 32) {
                if (B::ONE_XCHG) __syncthreads();  // one buffer: the last exchange's reads are done
                warp_store_positions<E>(st, o, xc.next());
            } else {
#pragma unroll
                for (int e = 0; e < E; e++) st[E * tid + e] = o[e];
            }
        } else {
            u64 o[E];
            if constexpr (T >= 32) {
                warp_load_positions<E>(st, o, xc.b1);
            } else {
#pragma unroll
                for (int e = 0; e < E; e++) o[e] = st[E * tid + e];
            }
            if constexpr (W32) {
                u32 v[1][E];
#pragma unroll
                for (int e = 0; e < E; e++) v[0][e] = shoup32_lazy((u32)o[e], C.n_inv32[j], C.n_inv32_s[j], (u32)q);
                inv_from32<LOGN, LOGE, 1, 0>(v, xc, C.tw32_inv + (size_t)j * N, (u32)q, 2 * (u32)q);
#pragma unroll
                for (int kk = 0; kk < E; kk++) st[tid + kk * T] = v[0][kk] >= (u32)q ? v[0][kk] - (u32)q : v[0][kk];
            } else {
                u64 v[1][E];
#pragma unroll
                for (int e = 0; e < E; e++) v[0][e] = shoup_mul_lazy(o[e], C.n_inv[j], C.n_inv_s[j], q);
                ntt_inv<LOGN, LOGE, 1>(v, xc, C, j);
#pragma unroll
                for (int kk = 0; kk < E; kk++) st[tid + kk * T] = v[0][kk] >= q ? v[0][kk] - q : v[0][kk];
            }
        }
        proxy_fence();  // this thread's writes, before the bulk store reads them
        __syncthreads();
        if (tid == 0) bulk_store(poly + item * N, st, BYTES);
    }
    if (tid == 0) {
        bulk_wait_all();
        if (failed) {
            atomicAdd(&g_ntt_wait_timeouts, 1u);
            // the loads still in flight land in this block's stages: wait
            // for them (bounded) before the block's shared memory is released
            mbar_wait(&bars[k & 1], (unsigned)(k >> 1) & 1u);
            if (pending_next) mbar_wait(&bars[(k + 1) & 1], (unsigned)((k + 1) >> 1) & 1u);
        }
    }
}

template <int LOGN, int LOGE, int W32>
struct NttVariant {
    static constexpr int T = Ring<LOGN, LOGE>::T;
    static constexpr size_t SMEM = 2 * (size_t)Ring<LOGN, LOGE>::PADDED * sizeof(u64);
    static cudaError_t init() {
        cudaError_t e = cudaFuncSetAttribute(k_ntt_bulk<LOGN, LOGE, W32>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)NttBulkCfg<LOGN, LOGE>::SMEM);
        if (e != cudaSuccess) return e;
        if constexpr (W32)
            return cudaFuncSetAttribute(k_ntt_batch32<LOGN, LOGE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        else
            return cudaFuncSetAttribute(k_ntt_batch<LOGN, LOGE>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    }
    static cudaError_t launch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                              cudaStream_t st) {
        // the bulk pipeline for the 32-bit arithmetic, whose transform is
        // bound by HBM; the 64-bit one is bound by integer issue and keeps
        // more resident warps per SM with one block per polynomial (its two
        // stages would cost it blocks); bulk copies need 16-byte aligned
        // addresses
        if (W32 && ((uintptr_t)poly & 15) == 0) {
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ntt_bulk<LOGN, LOGE, W32>, T,
                                                          NttBulkCfg<LOGN, LOGE>::SMEM);
            if (occ < 1) occ = 1;
            size_t grid = (size_t)li.sm_count * occ;
            if (grid > count) grid = count;
            k_ntt_bulk<LOGN, LOGE, W32><<<(unsigned)grid, T, NttBulkCfg<LOGN, LOGE>::SMEM, st>>>(li.dctx, poly,
                                                                                                count, inverse);
            return cudaGetLastError();
        }
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

// Bulk-copy waits that ran out since the library was loaded on the current
// device (0 in normal operation); UINT_MAX if the counter cannot be read.
unsigned ntt_wait_timeouts() {
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_ntt_wait_timeouts, sizeof(v)) != cudaSuccess) return ~0u;
    return v;
}

cudaError_t launch_ntt_batch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                             cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    (*li.launches)++;
    HW_NTT_SELECT(li, launch, li, poly, count, inverse, st)
}
