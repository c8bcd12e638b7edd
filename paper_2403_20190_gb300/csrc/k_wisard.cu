// k_wisard.cu -- the accumulation of a training batch into the model and the
// per-class response sums; dispatch of the IVP training (Algorithm 6 via the
// Inverse Vertical Packing of Algorithm 5), VP inference (Algorithm 7 via
// the Vertical Packing of Algorithm 3), clear-model inference and class-count
// kernels of hw_ext.cuh.
#include "hw_internal.cuh"
#include "hw_launch.h"

#include <vector>

// H mod q_i after a training batch's atomic additions (words below
// (n + 1) q_i < 2^64), one word per thread.
__global__ void k_model_reduce(const DevCtx* __restrict__ Cp, u64* __restrict__ model) {
    const DevCtx& C = *Cp;
    const size_t total = C.model_words;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(((idx % C.rlwe_words) / C.n) % C.r);
        model[idx] = reduce64(model[idx], C.P[p]);
    }
}

// counts[w] += sum over the batch of out[i][w] (mod q): the class-count
// ciphertext of dataset balancing, one word per thread.
__global__ void k_add_rlwes(const DevCtx* __restrict__ Cp, u64* __restrict__ counts,
                            const u64* __restrict__ out, int n) {
    const DevCtx& C = *Cp;
    const size_t total = C.rlwe_words;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const u64 q = C.P[(idx / C.n) % C.r].q;
        u64 s = counts[idx];
        for (int i = 0; i < n; i++) s = add_mod(s, out[(size_t)i * total + idx], q);
        counts[idx] = s;
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
// launchers: the external-product kernels go through the context's ExtOps
// ---------------------------------------------------------------------------
// The two parts of a split ring size as one table, part 0 (the default
// first) then part 1.
static std::vector<ExtOps> join_parts(const ExtOps* (*p0)(int*), const ExtOps* (*p1)(int*)) {
    std::vector<ExtOps> t;
    for (auto part : {p0, p1}) {
        int n = 0;
        const ExtOps* x = part(&n);
        t.insert(t.end(), x, x + n);
    }
    return t;
}

const ExtOps* hw_ext_table(int log_n, int* count) {
    *count = 0;
    switch (log_n) {
        case 6: {
            static const std::vector<ExtOps> t = join_parts(hw_ext_table_6_p0, hw_ext_table_6_p1);
            *count = (int)t.size();
            return t.data();
        }
        case 10: {
            static const std::vector<ExtOps> t = join_parts(hw_ext_table_10_p0, hw_ext_table_10_p1);
            *count = (int)t.size();
            return t.data();
        }
        case 12: {
            static const std::vector<ExtOps> t = join_parts(hw_ext_table_12_p0, hw_ext_table_12_p1);
            *count = (int)t.size();
            return t.data();
        }
#define X(L) \
    case L:  \
        return hw_ext_table_##L(count);
        X(7) X(8) X(9) X(11) X(13)
#undef X
    }
    return nullptr;
}

const ExtOps* hw_ext_find(int log_n, int loge, int np, int sm) {
    int count = 0;
    const ExtOps* t = hw_ext_table(log_n, &count);
    for (int k = 0; k < count; k++)
        if (t[k].loge == loge && t[k].np == np && t[k].sm == sm) return &t[k];
    return nullptr;
}

cudaError_t launch_ivp_train(const LaunchInfo& li, const uint64_t* rgsw, size_t n, uint64_t* out,
                             uint64_t* acc, int grid, cudaStream_t st) {
    int items = (int)(n * li.k0);
    if (items == 0) return cudaSuccess;
    if (grid > items) grid = items;
    cudaError_t e = li.ext->ivp(li, rgsw, items, out, acc, grid, st);
    (*li.launches)++;
    return e;
}

cudaError_t launch_model_reduce(const LaunchInfo& li, uint64_t* model, cudaStream_t st) {
    int threads = 256;
    size_t blocks = (li.model_words + threads - 1) / threads;
    if (blocks > (size_t)li.sm_count * 64) blocks = (size_t)li.sm_count * 64;
    k_model_reduce<<<(unsigned)blocks, threads, 0, st>>>(li.dctx, model);
    (*li.launches)++;
    return cudaGetLastError();
}

// Words of the first CMUX's digit transforms: one set of 2 dnum r
// polynomials per (RAM, class); none for the 32-bit external product.
size_t vp_digits_words(const LaunchInfo& li) {
    if (li.ext32) return 0;
    return (size_t)li.k0 * li.n_classes * 2 * li.dnum * li.r * li.n;
}

cudaError_t launch_vp_infer(const LaunchInfo& li, const uint64_t* model, const uint64_t* rgsw,
                            size_t n, uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st,
                            int packed, uint64_t* digits) {
    if (li.z > li.L) packed = 0;  // a tree level is an encrypted address bit: no packing
    const int groups = packed ? (li.n_classes < (1 << li.z) ? li.n_classes : (1 << li.z)) : li.n_classes;
    int items = (int)(n * li.k0 * groups);
    if (items == 0) return cudaSuccess;
    if (vp_digits_words(li) == 0) digits = nullptr;
    if (digits) {
        const int d_items = li.k0 * groups;
        const int d_grid = grid < d_items ? grid : d_items;
        cudaError_t e = li.ext->vp_digits(li, model, d_items, digits, d_grid, packed, st);
        (*li.launches)++;
        if (e != cudaSuccess) return e;
    }
    if (grid > items) grid = items;
    cudaError_t e = li.ext->vp(li, model, rgsw, items, resp, acc, grid, packed, digits, st);
    (*li.launches)++;
    return e;
}

cudaError_t launch_vp_plain(const LaunchInfo& li, const uint64_t* plain, const uint64_t* rgsw, size_t n,
                            uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st) {
    int items = (int)(n * li.k0);
    if (items == 0) return cudaSuccess;
    if (grid > items) grid = items;
    cudaError_t e = li.ext->vp_plain(li, plain, rgsw, items, resp, acc, grid, st);
    (*li.launches)++;
    return e;
}

cudaError_t launch_count_classes(const LaunchInfo& li, uint64_t* counts, const uint64_t* rgsw, size_t n,
                                 uint64_t* out, uint64_t* acc, int grid, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (grid > (int)n) grid = (int)n;
    cudaError_t e = li.ext->count(li, rgsw, (int)n, out, acc, grid, st);
    (*li.launches)++;
    if (e != cudaSuccess) return e;
    const int threads = 256;
    const size_t blocks = (li.rlwe_words + threads - 1) / threads;
    k_add_rlwes<<<(unsigned)blocks, threads, 0, st>>>(li.dctx, counts, out, (int)n);
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
