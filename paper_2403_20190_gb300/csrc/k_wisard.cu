// k_wisard.cu -- encrypted training (Algorithm 6 via the Inverse Vertical
// Packing of Algorithm 5) and encrypted inference (Algorithm 7 via the
// Vertical Packing of Algorithm 3), plus the accumulation into the model and
// the per-class response sums.
#include "hw_internal.cuh"
#include "hw_launch.h"

// Encrypted bit slot that drives LUT-index bit t of RAM j: label bits first
// (slots 0..L-1), then the RAM's tuple bits; -1 for a constant-0 bit.
__device__ __forceinline__ int bit_slot(const DevCtx& C, int j, int t) {
    return t < C.L ? t : C.ram_slot[(size_t)j * C.a + (t - C.L)];
}

// ---------------------------------------------------------------------------
// IVP training.  One thread block per work item (sample i, RAM j), persistent
// over items.  For each item: acc = (0, Delta); for each rotation bit t in
// z..L+a-1 with an encrypted control C_t: acc <- acc + C_t [x] (acc X^{2^(t-z)}
// - acc) (BlindRotate with weights -2^k); then the CDEMUX tree over bits
// 0..z-1, level i splitting L_j into (L_j - C_i [x] L_j, C_i [x] L_j).
// Outputs: out[item][slot] for every stored ciphertext index.
// Per-block scratch: two accumulators, their evaluation forms, and the
// evaluation forms of the k1 tree slots.
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(ExtCfg<LOGN>::T, ExtCfg<LOGN>::MINB)
    k_ivp_train(const DevCtx* __restrict__ Cp, const u64* __restrict__ rgsw, int n_items,
                u64* __restrict__ out, u64* __restrict__ scratch) {
    using X = ExtCfg<LOGN>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, smem + X::NP * X::PADDED, X::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, T = blockDim.x;
    const size_t rl = C.rlwe_words;
    u64* blk = scratch + (size_t)blockIdx.x * (4 + C.k1) * rl;
    u64* acc[2] = {blk, blk + rl};
    u64* accn[2] = {blk + 2 * rl, blk + 3 * rl};
    u64* tn = blk + 4 * rl;  // evaluation forms of the tree slots
    const int kbits = C.L + C.a;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int i = item / C.k0, j = item % C.k0;
        const u64* sample = rgsw + (size_t)i * C.sample_words;
        u64* Lout = out + (size_t)item * C.k1 * rl;
        // last encrypted rotation bit: its CMUX writes straight into slot 0
        int last = -1;
        for (int t = C.z; t < kbits; t++)
            if (bit_slot(C, j, t) >= 0) last = t;
        // acc = trivial RLWE (0, Delta * 1); its evaluation form is Delta everywhere in b
        u64* first_dst = last >= 0 ? acc[0] : Lout;
        u64* first_ntt = last >= 0 ? accn[0] : tn;
        for (size_t w = tid; w < rl; w += T) {
            size_t comp = w / ((size_t)C.r * C.n), rem = w % ((size_t)C.r * C.n);
            int p = (int)(rem / C.n), x = (int)(rem % C.n);
            first_dst[w] = (comp == 1 && x == 0) ? C.delta[p] : 0;
            first_ntt[w] = comp == 1 ? C.delta[p] : 0;
        }
        __syncthreads();
        int cur = 0;
        for (int t = C.z; t < kbits; t++) {
            int slot = bit_slot(C, j, t);
            if (slot < 0) continue;  // constant-0 control: the CMUX keeps acc
            const int w = 1 << (t - C.z);
            u64* dst = (t == last) ? Lout : acc[cur ^ 1];
            u64* dstn = (t == last) ? tn : accn[cur ^ 1];
            int nslot = -1;  // the next encrypted control (rotation bit or first tree gate)
            for (int t2 = t + 1; t2 < kbits && nslot < 0; t2++) nslot = bit_slot(C, j, t2);
            if (nslot < 0 && C.n_gates > 0) nslot = bit_slot(C, j, C.gate_lvl[0]);
            ext_product<LOGN, X::LOGE, X::NP>(
                C, sample + (size_t)slot * C.rgsw_words, acc[cur], w, acc[cur], 0, EXT_ADD, dst, xc,
                ExtNtt{accn[cur], dstn, t - C.z, 0,
                       nslot >= 0 ? sample + (size_t)nslot * C.rgsw_words : nullptr, 1});
            cur ^= 1;
        }
        // CDEMUX tree (pruned gate list, level by level)
        for (int g = 0; g < C.n_gates; g++) {
            const int lvl = C.gate_lvl[g], jj = C.gate_j[g];
            const int nn = 1 << lvl;
            const size_t slo = C.slot_of[jj], shi = C.slot_of[jj + nn];
            u64* lo = Lout + slo * rl;
            u64* hi = Lout + shi * rl;
            u64* lon = tn + slo * rl;
            u64* hin = tn + shi * rl;
            int slot = bit_slot(C, j, lvl);
            if (slot < 0) {  // constant-0 control: everything stays in L_j
                for (size_t w = tid; w < rl; w += T) hi[w] = hin[w] = 0;
                __syncthreads();
                continue;
            }
            const int nslot = g + 1 < C.n_gates ? bit_slot(C, j, C.gate_lvl[g + 1]) : -1;
            ext_product<LOGN, X::LOGE, X::NP>(
                C, sample + (size_t)slot * C.rgsw_words, lo, 0, nullptr, 0, EXT_PLAIN, hi, xc,
                ExtNtt{lon, hin, -1, 0, nslot >= 0 ? sample + (size_t)nslot * C.rgsw_words : nullptr,
                       1});
            for (size_t w = tid; w < rl; w += T) {
                const u64 q = C.P[(w / C.n) % C.r].q;
                lo[w] = sub_mod(lo[w], hi[w], q);
                lon[w] = sub_mod(lon[w], hin[w], q);
            }
            __syncthreads();
        }
    }
}

// H[j][t] += sum over the batch of out[i][j][t] (mod q), one word per thread.
__global__ void k_accumulate(const DevCtx* __restrict__ Cp, u64* __restrict__ model,
                             const u64* __restrict__ out, int n) {
    const DevCtx& C = *Cp;
    const size_t total = C.model_words;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(((idx % C.rlwe_words) / C.n) % C.r);
        const u64 q = C.P[p].q;
        u64 s = model[idx];
        for (int i = 0; i < n; i++) s = add_mod(s, out[(size_t)i * total + idx], q);
        model[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// VP inference.  One thread block per item (sample i, RAM j, class c).
// Label bits are in clear: tree levels driven by label bits select a stored
// ciphertext directly; a tree level driven by an encrypted address bit (z > L)
// is a CMUX(C, L_{v+n}, L_v); label bits among the rotation bits are a plain
// rotation X^-(c >> z).  The encrypted address bits then blind-rotate with
// weights +2^k (X^-2^k) and the last CMUX writes ExtractLWE(., 0) directly.
// Per-block scratch: two accumulators and their evaluation forms.
// ---------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(ExtCfg<LOGN>::T, ExtCfg<LOGN>::MINB)
    k_vp_infer(const DevCtx* __restrict__ Cp, const u64* __restrict__ model,
               const u64* __restrict__ rgsw, int n_items, u64* __restrict__ resp,
               u64* __restrict__ scratch) {
    using X = ExtCfg<LOGN>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, smem + X::NP * X::PADDED, X::PADDED, 0};
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, T = blockDim.x;
    const size_t rl = C.rlwe_words;
    const int two_n = 2 * C.n;
    u64* blk = scratch + (size_t)blockIdx.x * 4 * rl;
    u64* acc[2] = {blk, blk + rl};
    u64* accn[2] = {blk + 2 * rl, blk + 3 * rl};
    const int kbits = C.L + C.a;
    const int l = C.n_classes;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int c = item % l;
        const int ij = item / l;
        const int i = ij / C.k0, j = ij % C.k0;
        const u64* sample = rgsw + (size_t)i * C.sample_words;
        const u64* Hj = model + (size_t)j * C.k1 * rl;
        // items run class-fastest (the l classes of a (sample, RAM) share its
        // RGSW bits); responses are stored [sample][class][RAM]
        u64* lwe = resp + (((size_t)i * l + c) * C.k0 + j) * C.lwe_words;
        const u64* src;
        const u64* srcn = nullptr;  // evaluation form of src, once known
        int e0;
        if (C.z <= C.L) {
            src = Hj + (size_t)C.slot_of[c & ((1 << C.z) - 1)] * rl;
            const int R = c >> C.z;  // clear label bits among the rotation bits
            e0 = (two_n - R) % two_n;
        } else {
            // one encrypted tree level (bit z-1, an address bit): CMUX(C, L_{v+n}, L_v)
            const int nn = 1 << (C.z - 1);
            const u64* lo = Hj + (size_t)C.slot_of[c] * rl;
            const u64* hi = Hj + (size_t)C.slot_of[c + nn] * rl;
            const int slot = bit_slot(C, j, C.z - 1);
            if (slot < 0) {
                src = lo;
            } else {
                ext_product<LOGN, X::LOGE, X::NP>(C, sample + (size_t)slot * C.rgsw_words, hi, 0, lo,
                                                  0, EXT_ADD, acc[0], xc,
                                                  ExtNtt{nullptr, nullptr, -1, 0, nullptr, 0});
                src = acc[0];
            }
            e0 = 0;
        }
        int last = -1;
        for (int t = (C.z > C.L ? C.z : C.L); t < kbits; t++)
            if (bit_slot(C, j, t) >= 0) last = t;
        if (last < 0) {  // nothing encrypted left: extract src * X^e0
            for (int jp = 0; jp < C.r; jp++) {
                const u64 q = C.P[jp].q;
                const u64* pa = src + (size_t)jp * C.n;
                const u64* pb = src + (size_t)(C.r + jp) * C.n;
                u64* lw = lwe + (size_t)jp * (C.n + 1);
                for (int y = tid; y < C.n; y += T) {
                    u64 va = rot_read(pa, y, e0, C.n, q);
                    if (y == 0)
                        lw[0] = va;
                    else
                        lw[C.n - y] = neg_mod(va, q);
                }
                if (tid == 0) lw[C.n] = rot_read(pb, 0, e0, C.n, q);
            }
            __syncthreads();
            continue;
        }
        int cur = (src == acc[0]) ? 0 : 1;  // acc[cur ^ 1] is free
        for (int t = (C.z > C.L ? C.z : C.L); t < kbits; t++) {
            int slot = bit_slot(C, j, t);
            if (slot < 0) continue;
            const int w = 1 << (t - C.z);
            const int eA = (e0 + two_n - w) % two_n;
            // the l classes of a (sample, RAM) share its RGSW bits: only the
            // class-0 block asks L2 for the next one
            int nslot = -1;
            if (c == 0)
                for (int t2 = t + 1; t2 < kbits && nslot < 0; t2++) nslot = bit_slot(C, j, t2);
            const ExtNtt nt{srcn, t == last ? nullptr : accn[cur ^ 1], t - C.z, 1,
                            nslot >= 0 ? sample + (size_t)nslot * C.rgsw_words : nullptr, 0};
            if (t == last) {
                ext_product<LOGN, X::LOGE, X::NP>(C, sample + (size_t)slot * C.rgsw_words, src, eA, src,
                                                  e0, EXT_LWE, lwe, xc, nt);
            } else {
                ext_product<LOGN, X::LOGE, X::NP>(C, sample + (size_t)slot * C.rgsw_words, src, eA, src,
                                                  e0, EXT_ADD, acc[cur ^ 1], xc, nt);
                src = acc[cur ^ 1];
                srcn = accn[cur ^ 1];
                cur ^= 1;
            }
            e0 = 0;
        }
    }
}

// sums[i][c] = sum_j resp[i][c][j] (mod q), one word per thread.
__global__ void k_class_sums(const DevCtx* __restrict__ Cp, const u64* __restrict__ resp,
                             int n_pairs, u64* __restrict__ sums) {
    const DevCtx& C = *Cp;
    const size_t lw = C.lwe_words;
    const size_t total = (size_t)n_pairs * lw;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const size_t pair = idx / lw, w = idx % lw;
        const int p = (int)(w / (C.n + 1));
        const u64 q = C.P[p].q;
        const u64* base = resp + pair * C.k0 * lw + w;
        u64 s = 0;
        for (int j = 0; j < C.k0; j++) s = add_mod(s, base[(size_t)j * lw], q);
        sums[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// launchers (one instantiation per ring size)
// ---------------------------------------------------------------------------
template <int LOGN>
static int ext_grid_t(int sms) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ivp_train<LOGN>, ExtCfg<LOGN>::T,
                                                  ExtCfg<LOGN>::XCHG_BYTES);
    if (occ < 1) occ = 1;
    return occ * sms;
}

int hw_ext_grid(const LaunchInfo& li) {
    switch (li.log_n) {
#define X(L) \
    case L:  \
        return ext_grid_t<L>(li.sm_count);
        HW_FOR_EACH_LOGN(X)
#undef X
    }
    return li.sm_count;
}

cudaError_t launch_ivp_train(const LaunchInfo& li, const uint64_t* rgsw, size_t n, uint64_t* out,
                             uint64_t* acc, int grid, cudaStream_t st) {
    int items = (int)(n * li.k0);
    if (items == 0) return cudaSuccess;
    if (grid > items) grid = items;
    switch (li.log_n) {
#define X(L)                                                                                   \
    case L:                                                                                    \
        k_ivp_train<L><<<grid, ExtCfg<L>::T, ExtCfg<L>::XCHG_BYTES, st>>>(li.dctx, rgsw, items, out, acc); \
        break;
        HW_FOR_EACH_LOGN(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const LaunchInfo& li, uint64_t* model, const uint64_t* out, size_t n,
                              cudaStream_t st) {
    int threads = 256;
    size_t blocks = (li.model_words + threads - 1) / threads;
    if (blocks > (size_t)li.sm_count * 64) blocks = (size_t)li.sm_count * 64;
    k_accumulate<<<(unsigned)blocks, threads, 0, st>>>(li.dctx, model, out, (int)n);
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t launch_vp_infer(const LaunchInfo& li, const uint64_t* model, const uint64_t* rgsw,
                            size_t n, uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st) {
    int items = (int)(n * li.k0 * li.n_classes);
    if (items == 0) return cudaSuccess;
    if (grid > items) grid = items;
    switch (li.log_n) {
#define X(L)                                                                                     \
    case L:                                                                                      \
        k_vp_infer<L><<<grid, ExtCfg<L>::T, ExtCfg<L>::XCHG_BYTES, st>>>(li.dctx, model, rgsw, items, resp, \
                                                                  acc);                          \
        break;
        HW_FOR_EACH_LOGN(X)
#undef X
        default:
            return cudaErrorInvalidValue;
    }
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t launch_class_sums(const LaunchInfo& li, const uint64_t* resp, size_t n, uint64_t* sums,
                              cudaStream_t st) {
    int pairs = (int)(n * li.n_classes);
    if (pairs == 0) return cudaSuccess;
    int threads = 256;
    size_t total = (size_t)pairs * li.lwe_words;
    size_t blocks = (total + threads - 1) / threads;
    if (blocks > (size_t)li.sm_count * 64) blocks = (size_t)li.sm_count * 64;
    k_class_sums<<<(unsigned)blocks, threads, 0, st>>>(li.dctx, resp, pairs, sums);
    (*li.launches)++;
    return cudaGetLastError();
}

cudaError_t hw_wisard_kernels_init() {
    cudaError_t e = cudaSuccess;
#define X(L)                                                                                    \
    if (e == cudaSuccess)                                                                       \
        e = cudaFuncSetAttribute(k_ivp_train<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                 (int)ExtCfg<L>::XCHG_BYTES);                                   \
    if (e == cudaSuccess)                                                                       \
        e = cudaFuncSetAttribute(k_vp_infer<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                 (int)ExtCfg<L>::XCHG_BYTES);
    HW_FOR_EACH_LOGN(X)
#undef X
    return e;
}
