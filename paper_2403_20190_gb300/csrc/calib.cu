// calib.cu -- the integer-issue ceiling of the library's NTT butterflies on
// the GPU it runs on (no counterpart in the paper; it gives the measured
// denominator beside the derived multiply-count peak of the rooflines).
//
// Each thread keeps 16 residues in registers and runs one butterfly form for
// 12 stages per round, with no memory traffic and no barriers, in one
// 512-thread block per SM (the external-product kernels' shape):
//   ct64  lazy Cooley-Tukey with a 64-bit Shoup twiddle (values grow by 2q
//         per stage; one Barrett reduction per 12 stages, as in a 4096-point
//         forward transform)
//   gs64  Harvey Gentleman-Sande (sum reduced below 2q, Shoup product of the
//         difference), as in the inverse transforms
//   ct32 / gs32  the same in 32-bit words (primes below 2^30)
// The values computed are discarded (one XOR per thread is stored so the
// loop is not optimised away).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "hwisard.h"
#include "hw_internal.cuh"

extern int hw_ctx_fail(int code, const char* msg);

namespace {

template <typename W>
__device__ __forceinline__ W shoup_lazy_w(W x, W w, W ws, W q);
template <>
__device__ __forceinline__ u64 shoup_lazy_w<u64>(u64 x, u64 w, u64 ws, u64 q) {
    return shoup_mul_lazy(x, w, ws, q);
}
template <>
__device__ __forceinline__ u32 shoup_lazy_w<u32>(u32 x, u32 w, u32 ws, u32 q) {
    return shoup32_lazy(x, w, ws, q);
}
__device__ __forceinline__ u64 mulhi_w(u64 a, u64 b) { return __umul64hi(a, b); }
__device__ __forceinline__ u32 mulhi_w(u32 a, u32 b) { return __umulhi(a, b); }

template <typename W, int FORM>
__global__ void __launch_bounds__(512, 1) k_bfly_rate(const W* __restrict__ tw, W* __restrict__ out, int rounds) {
    W v[16];
    const W q = tw[8], q2 = 2 * q, mu = tw[9];
#pragma unroll
    for (int e = 0; e < 16; e++) v[e] = (W)(((u64)threadIdx.x * 977u + (u64)e * 131u) % (u64)q);
    W w[4], ws[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        w[i] = tw[2 * i];
        ws[i] = tw[2 * i + 1];
    }
    for (int it = 0; it < rounds; it++) {
#pragma unroll
        for (int s = 0; s < 12; s++) {
            const int h = 1 << (s & 3);
#pragma unroll
            for (int e = 0; e < 16; e++) {
                if (e & h) continue;
                W& X = v[e];
                W& Y = v[e | h];
                if (FORM == 0) {
                    const W t = shoup_lazy_w<W>(Y, w[s & 3], ws[s & 3], q);
                    Y = X + q2 - t;
                    X = X + t;
                } else {
                    W sum = X + Y;
                    sum = sum >= q2 ? sum - q2 : sum;
                    Y = shoup_lazy_w<W>(X + q2 - Y, w[s & 3], ws[s & 3], q);
                    X = sum;
                }
            }
        }
        if (FORM == 0) {
#pragma unroll
            for (int e = 0; e < 16; e++) {
                W r = v[e] - mulhi_w(v[e], mu) * q;
                r = r >= q ? r - q : r;
                v[e] = r >= q ? r - q : r;
            }
        }
    }
    W x = 0;
#pragma unroll
    for (int e = 0; e < 16; e++) x ^= v[e];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <typename W>
int rate(int form, W q, int sms, W* tw_dev, W* out_dev, double* gbfly) {
    W h[10];
    for (int i = 0; i < 4; i++) {
        const W w = (W)((123456789ull * (i + 1)) % (unsigned long long)q);
        h[2 * i] = w;
        h[2 * i + 1] = (W)((((unsigned __int128)w) << (8 * sizeof(W))) / q);
    }
    h[8] = q;
    h[9] = (W)((((unsigned __int128)1) << (8 * sizeof(W))) / q);
    if (cudaMemcpy(tw_dev, h, sizeof(h), cudaMemcpyHostToDevice) != cudaSuccess) return HW_ECUDA;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int rounds = 256;
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(a);
        if (form == 0)
            k_bfly_rate<W, 0><<<sms, 512>>>(tw_dev, out_dev, rounds);
        else
            k_bfly_rate<W, 1><<<sms, 512>>>(tw_dev, out_dev, rounds);
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (cudaGetLastError() != cudaSuccess) return HW_ECUDA;
    *gbfly = (double)sms * 512 * rounds * 12 * 8 / (best * 1e-3) / 1e9;
    return HW_OK;
}

}  // namespace

extern "C" int hw_butterfly_rates(int cuda_device, double* out_host) {
    if (!out_host) return hw_ctx_fail(HW_EINVAL, "hw_butterfly_rates: null output");
    if (cudaSetDevice(cuda_device) != cudaSuccess)
        return hw_ctx_fail(HW_ECUDA, "hw_butterfly_rates: cudaSetDevice failed");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device);
    void* tw = nullptr;
    void* out = nullptr;
    if (cudaMalloc(&tw, 16 * sizeof(u64)) != cudaSuccess ||
        cudaMalloc(&out, (size_t)sms * 512 * sizeof(u64)) != cudaSuccess) {
        cudaFree(tw);
        return hw_ctx_fail(HW_ECUDA, "hw_butterfly_rates: allocation failed");
    }
    // a 50-bit and a 30-bit prime of the workloads' kind (values only set the
    // operands; the instruction sequence is the same for any prime)
    const u64 q64 = 1125899906826241ull;
    const u32 q32 = 1073479681u;
    int rc = rate<u64>(0, q64, sms, (u64*)tw, (u64*)out, &out_host[0]);
    if (rc == HW_OK) rc = rate<u64>(1, q64, sms, (u64*)tw, (u64*)out, &out_host[1]);
    if (rc == HW_OK) rc = rate<u32>(0, q32, sms, (u32*)tw, (u32*)out, &out_host[2]);
    if (rc == HW_OK) rc = rate<u32>(1, q32, sms, (u32*)tw, (u32*)out, &out_host[3]);
    cudaFree(tw);
    cudaFree(out);
    if (rc != HW_OK) return hw_ctx_fail(rc, "hw_butterfly_rates: a measuring launch failed");
    return HW_OK;
}
