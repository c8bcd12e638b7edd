// hw_launch.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

struct DevCtx;

struct LaunchInfo {
    const DevCtx* dctx;  // device copy of the context
    int log_n, n, r, k0, k1, n_classes, n_data, n_slots, L, dnum;
    size_t rlwe_words, lwe_words, rgsw_words, sample_words, model_words;
    int sm_count;
    int small_q;  // every q_i < 2^30: the 32-bit transform tables exist
    unsigned long long* launches;  // launch counter
};

// Persistent grid size of the IVP / VP kernels for this context.
int hw_ext_grid(const LaunchInfo& li);

cudaError_t launch_keygen(const LaunchInfo& li, uint64_t seed, uint64_t* key, cudaStream_t st);
cudaError_t launch_encode(const LaunchInfo& li, const uint8_t* values, size_t n, uint8_t* bits,
                          cudaStream_t st);
cudaError_t launch_encrypt(const LaunchInfo& li, const uint64_t* key, const uint8_t* bits,
                           const uint32_t* labels, size_t n, uint64_t seed, uint64_t first,
                           uint64_t* out, cudaStream_t st);
cudaError_t launch_ivp_train(const LaunchInfo& li, const uint64_t* rgsw, size_t n, uint64_t* out,
                             uint64_t* acc, int grid, cudaStream_t st);
cudaError_t launch_accumulate(const LaunchInfo& li, uint64_t* model, const uint64_t* out, size_t n,
                              cudaStream_t st);
cudaError_t launch_vp_infer(const LaunchInfo& li, const uint64_t* model, const uint64_t* rgsw,
                            size_t n, uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st);
cudaError_t launch_class_sums(const LaunchInfo& li, const uint64_t* resp, size_t n, uint64_t* sums,
                              cudaStream_t st);
cudaError_t launch_decrypt_rlwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                                size_t count, int64_t* out, uint64_t* phase_scratch,
                                size_t chunk, cudaStream_t st);
cudaError_t launch_decrypt_lwe(const LaunchInfo& li, const uint64_t* key, const uint64_t* ct,
                               size_t count, int64_t* out, cudaStream_t st);
cudaError_t launch_pdact(const LaunchInfo& li, const int64_t* counts, size_t n, int64_t* scores,
                         int32_t* labels, cudaStream_t st);
cudaError_t launch_export_rgsw(const LaunchInfo& li, const uint64_t* rgsw, size_t count,
                               uint64_t* out, cudaStream_t st);
cudaError_t launch_ntt_batch(const LaunchInfo& li, uint64_t* poly, size_t count, int inverse,
                             cudaStream_t st);
cudaError_t hw_kernels_init(int log_n);
