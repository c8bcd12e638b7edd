// hw_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

struct DevCtx;
struct LaunchInfo;

// Launchers of one external-product geometry (hw_ext.cuh): 2^loge residues
// per thread, np polynomials per transform, `threads` threads per block.
struct ExtOps {
    int loge, np;
    int sm;            // shared-memory mode: 0 none, 1 the accumulator's evaluation form,
                       // 2 the accumulator polynomials of one prime
    int scratch_rlwe;  // per-block RLWE buffers of inference (training adds k1)
    int threads;
    size_t smem, encrypt_smem;  // smem: fixed part (+ r-dependent evaluation form in mode 1)
    cudaError_t (*init)();      // shared-memory attributes of its kernels
    int (*occupancy)(size_t smem);  // resident blocks per SM of the IVP / VP kernels
    cudaError_t (*encrypt)(const LaunchInfo&, const uint64_t* key, const uint8_t* bits,
                           const uint32_t* labels, int slot0, int n_enc, unsigned blocks,
                           uint64_t seed, uint64_t first, uint64_t* out, cudaStream_t);
    cudaError_t (*ivp)(const LaunchInfo&, const uint64_t* rgsw, int items, uint64_t* model,
                       uint64_t* acc, int grid, cudaStream_t);
    cudaError_t (*vp)(const LaunchInfo&, const uint64_t* model, const uint64_t* rgsw, int items,
                      uint64_t* resp, uint64_t* acc, int grid, int packed, const uint64_t* digits,
                      cudaStream_t);
    cudaError_t (*count)(const LaunchInfo&, const uint64_t* rgsw, int items, uint64_t* out,
                         uint64_t* acc, int grid, cudaStream_t);
    cudaError_t (*vp_plain)(const LaunchInfo&, const uint64_t* plain, const uint64_t* rgsw, int items,
                            uint64_t* resp, uint64_t* acc, int grid, cudaStream_t);
    // the first CMUX's digit transforms of every (RAM, class) item of VP
    cudaError_t (*vp_digits)(const LaunchInfo&, const uint64_t* model, int items, uint64_t* digits, int grid,
                             int packed, cudaStream_t);
};

struct LaunchInfo {
    const DevCtx* dctx;  // device copy of the context
    int log_n, n, r, k0, k1, n_classes, n_data, n_slots, L, dnum;
    size_t rlwe_words, lwe_words, rgsw_words, sample_words, model_words;
    int sm_count;
    int small_q;  // every q_i < 2^30: the 32-bit transform tables exist
    int ext32;    // the external product runs in 32-bit words
    const ExtOps* ext;  // the context's external-product geometry
    int ext_grid;       // persistent grid of the IVP / VP kernels
    size_t ext_smem;    // their dynamic shared memory per block
    int ntt_loge;       // hw_ntt_*: 2^ntt_loge residues per thread
    int ntt_limbs;      // hw_ntt_*: 1 = 32-bit arithmetic, 2 = 64-bit
    int z;              // CMUX-tree levels (horizontal packing needs z <= L)
    size_t l2_persist;     // > 0: persisting L2 bytes for the IVP / VP accumulators
    size_t l2_window_max;  // largest access-policy window the device takes
    unsigned long long* launches;  // launch counter
};

// Geometry tables, one per ring size (k_ext_*.cu), and lookup.
#define HW_EXT_TABLE_DECL(L) const ExtOps* hw_ext_table_##L(int* count);
HW_EXT_TABLE_DECL(7) HW_EXT_TABLE_DECL(8) HW_EXT_TABLE_DECL(9)
HW_EXT_TABLE_DECL(11) HW_EXT_TABLE_DECL(13)
#undef HW_EXT_TABLE_DECL
// N = 64, 1024 and 4096 are split in two parts (k_ext_l6a/b.cu, ...).
const ExtOps* hw_ext_table_6_p0(int* count);
const ExtOps* hw_ext_table_6_p1(int* count);
const ExtOps* hw_ext_table_10_p0(int* count);
const ExtOps* hw_ext_table_10_p1(int* count);
const ExtOps* hw_ext_table_12_p0(int* count);
const ExtOps* hw_ext_table_12_p1(int* count);
const ExtOps* hw_ext_table(int log_n, int* count);
const ExtOps* hw_ext_find(int log_n, int loge, int np, int sm);

unsigned ntt_wait_timeouts();
cudaError_t launch_keygen(const LaunchInfo& li, uint64_t seed, uint64_t* key, cudaStream_t st);
cudaError_t launch_encode(const LaunchInfo& li, const uint8_t* values, size_t n, uint8_t* bits,
                          cudaStream_t st);
cudaError_t launch_encrypt(const LaunchInfo& li, const uint64_t* key, const uint8_t* bits,
                           const uint32_t* labels, size_t n, uint64_t seed, uint64_t first,
                           uint64_t* out, cudaStream_t st);
// IVP training adds into the model unreduced; launch_model_reduce brings it
// back below q_i (at most HW_TRAIN_MAX_BATCH(q) samples in between).
cudaError_t launch_ivp_train(const LaunchInfo& li, const uint64_t* rgsw, size_t n, uint64_t* model,
                             uint64_t* acc, int grid, cudaStream_t st);
cudaError_t launch_model_reduce(const LaunchInfo& li, uint64_t* model, cudaStream_t st);
// With `digits` (vp_digits_words of them) the first CMUX of every
// item takes its digit transforms from there, computed once for the batch.
cudaError_t launch_vp_infer(const LaunchInfo& li, const uint64_t* model, const uint64_t* rgsw,
                            size_t n, uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st,
                            int packed = 0, uint64_t* digits = nullptr);
size_t vp_digits_words(const LaunchInfo& li);
// Unencrypted-model inference: the clear counters into plaintext tables, and
// the responses against them.
size_t hw_plain_words_li(const LaunchInfo& li);
cudaError_t launch_plain_load(const LaunchInfo& li, const int64_t* counts, uint64_t* plain, cudaStream_t st);
cudaError_t launch_vp_plain(const LaunchInfo& li, const uint64_t* plain, const uint64_t* rgsw, size_t n,
                            uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st);
cudaError_t launch_count_classes(const LaunchInfo& li, uint64_t* counts, const uint64_t* rgsw, size_t n,
                                 uint64_t* out, uint64_t* acc, int grid, cudaStream_t st);
cudaError_t launch_pdact_balanced(const LaunchInfo& li, const int64_t* counts, const int64_t* class_counts,
                                  size_t n, int64_t* scores, int32_t* labels, cudaStream_t st);
cudaError_t launch_class_sums(const LaunchInfo& li, const uint64_t* resp, size_t n, uint64_t* sums,
                              cudaStream_t st);
cudaError_t launch_decrypt_rlwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                                size_t count, int64_t* out, uint64_t* phase_scratch,
                                size_t chunk, cudaStream_t st);
// Definition 2's counters W[c][j][addr] of a whole model (HW_DEC_MODEL).
cudaError_t launch_decrypt_model(const LaunchInfo& li, const uint64_t* key, const uint64_t* model, int a,
                                 int64_t* out, uint64_t* phase_scratch, size_t chunk, cudaStream_t st);
cudaError_t launch_decrypt_lwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                               size_t count, int64_t* out, cudaStream_t st);
cudaError_t launch_pdact(const LaunchInfo& li, const int64_t* counts, size_t n, int64_t* scores,
                         int32_t* labels, cudaStream_t st);
cudaError_t launch_export_rgsw(const LaunchInfo& li, const uint64_t* rgsw, size_t count,
                               uint64_t* out, cudaStream_t st);
cudaError_t launch_import_rgsw(const LaunchInfo& li, const uint64_t* in, size_t count, uint64_t* rgsw,
                               cudaStream_t st);
cudaError_t launch_ntt_batch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                             cudaStream_t st);
// PackingKeySwitching (k_pack.cu).
size_t hw_pack_scratch_words_li(const LaunchInfo& li, size_t group);
cudaError_t launch_ksk_gen(const LaunchInfo& li, const uint64_t* key, uint64_t seed, uint64_t* ksk,
                           cudaStream_t st);
cudaError_t launch_pack(const LaunchInfo& li, const uint64_t* ksk, const uint64_t* resp, size_t n,
                        uint64_t* packed, uint64_t* scratch, size_t scratch_words, cudaStream_t st);
cudaError_t hw_pack_kernels_init(const LaunchInfo& li);

// Shared-memory attributes of the context's kernels (its ring size, its
// external-product geometry and its batched-NTT variant).
cudaError_t hw_kernels_init(const LaunchInfo& li);
