// noalloc.cu -- encrypted inference for callers that cannot allocate device
// memory.
//
// Some callers have no way to obtain scratch memory on the device: code that
// runs inside a host process whose device memory is owned by another
// allocator it cannot reach, request loops whose latency budget forbids
// cudaMalloc on the hot path, or plug-ins that only ever receive the input
// and output buffers of a request.  hw_infer_static_scratch() serves them:
// it runs the same VP inference kernel as hw_infer(), but the per-block
// accumulators (and their evaluation forms) that hw_infer() takes from the
// caller's scratch buffer live in a fixed array compiled into this library
// instead.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/hwisard.h"
#include "hw_internal.cuh"
#include "hw_launch.h"

// The scratch array: HW_STATIC_SCRATCH_BYTES on every GPU that loads the
// library, held until the process exits.
static __device__ __align__(256) u64 g_static_scratch[HW_STATIC_SCRATCH_BYTES / sizeof(u64)];

// In host code `g_static_scratch` only names the symbol; its device address
// is looked up once per device, with that device current.
#define HW_MAX_DEVICES 64
static std::mutex g_scratch_mu;
static u64* g_scratch_dev[HW_MAX_DEVICES];

// Defined in api.cu: the context's launch information and device.
extern const LaunchInfo* hw_ctx_launch_info(const hw_ctx* ctx);
extern int hw_ctx_device(const hw_ctx* ctx);
extern int hw_ctx_fail(int code, const char* msg);

static int scratch_address(int device, u64** out) {
    if (device < 0 || device >= HW_MAX_DEVICES) return hw_ctx_fail(HW_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            char buf[256];
            snprintf(buf, sizeof(buf), "cudaGetSymbolAddress(static scratch) failed: %s",
                     cudaGetErrorString(e));
            return hw_ctx_fail(HW_ECUDA, buf);
        }
        g_scratch_dev[device] = (u64*)p;
    }
    *out = g_scratch_dev[device];
    return HW_OK;
}

extern "C" int hw_infer_static_scratch(hw_ctx* ctx, const uint64_t* model, const uint64_t* rgsw,
                                       size_t n, uint64_t* resp, uint64_t* sums, void* stream) {
    if (!ctx) return hw_ctx_fail(HW_EINVAL, "hw_infer_static_scratch: null context");
    const int device = hw_ctx_device(ctx);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return hw_ctx_fail(HW_ECUDA, "hw_infer_static_scratch: cudaSetDevice failed");
    if (n == 0) return HW_OK;
    if (!model || !rgsw || !resp || !sums)
        return hw_ctx_fail(HW_EINVAL, "hw_infer_static_scratch: null buffer");
    const LaunchInfo& li = *hw_ctx_launch_info(ctx);
    // each persistent block needs two RLWE accumulators and, unless the
    // geometry keeps it in shared memory, one evaluation-form buffer
    // (scratch_rlwe = 2 or 3 RLWEs)
    const size_t per_block = (size_t)li.ext->scratch_rlwe * li.rlwe_words * sizeof(u64);
    const size_t fit = HW_STATIC_SCRATCH_BYTES / per_block;
    if (fit < 1) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "hw_infer_static_scratch: one block needs %zu bytes of scratch, the static array "
                 "holds %zu (ring too large for this entry point; use hw_infer)",
                 per_block, (size_t)HW_STATIC_SCRATCH_BYTES);
        return hw_ctx_fail(HW_EINVAL, buf);
    }
    if ((double)n * li.k0 * li.n_classes > 2147483647.0)
        return hw_ctx_fail(HW_EINVAL, "hw_infer_static_scratch: batch too large");
    u64* scratch = nullptr;
    int rc = scratch_address(device, &scratch);
    if (rc != HW_OK) return rc;
    int grid = li.ext_grid;
    if ((size_t)grid > fit) grid = (int)fit;
    cudaStream_t st = (cudaStream_t)stream;
    // No part of the array has to start at zero: every block writes each of
    // its accumulators (and their evaluation forms) completely before it
    // reads them.
    e = launch_vp_infer(li, model, rgsw, n, resp, scratch, grid, st);
    if (e == cudaSuccess) e = launch_class_sums(li, resp, n, sums, st);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "hw_infer_static_scratch: launch failed: %s", cudaGetErrorString(e));
        return hw_ctx_fail(HW_ECUDA, buf);
    }
    return HW_OK;
}
