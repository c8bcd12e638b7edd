// bfly_ceiling.cu -- integer-issue ceiling of the NTT butterflies on this GPU.
//
// Each thread keeps 16 residues in registers and runs the library's two
// butterfly forms with no memory traffic and no barriers:
//   ct64  lazy Cooley-Tukey (Shoup twiddle, values grow by 2q per stage,
//         one Barrett reduction every 12 stages as in a 4096-point forward
//         transform; the 32-bit form wraps past 2^32 in this loop, which
//         changes no instruction and so no timing)
//   gs64  Harvey Gentleman-Sande (sum reduced below 2q, Shoup product of the
//         difference), as in the inverse transform
//   ct32 / gs32  the same in 32-bit arithmetic (primes below 2^30)
// and reports butterflies per second and per clock per SM (at the clock the
// caller gives).  The result bounds any kernel built from these butterflies:
// a transform or external product cannot run its butterflies faster.
//
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//   bfly_ceiling.cu -o bfly_ceiling && ./bfly_ceiling [sm_mhz]
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>

typedef uint64_t u64;
typedef uint32_t u32;

template <typename W>
struct Wide;
template <>
struct Wide<u64> {
    static __device__ __forceinline__ u64 hi(u64 a, u64 b) { return __umul64hi(a, b); }
};
template <>
struct Wide<u32> {
    static __device__ __forceinline__ u32 hi(u32 a, u32 b) { return __umulhi(a, b); }
};

template <typename W>
__device__ __forceinline__ void ct(W& X, W& Y, W w, W ws, W q, W q2) {
    const W t = Y * w - Wide<W>::hi(Y, ws) * q;
    Y = X + q2 - t;
    X = X + t;
}
template <typename W>
__device__ __forceinline__ void gs(W& U, W& V, W w, W ws, W q, W q2) {
    W s = U + V;
    s = s >= q2 ? s - q2 : s;
    const W d = U + q2 - V;
    V = d * w - Wide<W>::hi(d, ws) * q;
    U = s;
}

// FORM 0: ct, FORM 1: gs.  `rounds` blocks of 12 stages over 8 butterflies.
template <typename W, int FORM>
__global__ void k_bfly(const W* __restrict__ tw, W* __restrict__ out, int rounds, W q) {
    W v[16];
    for (int e = 0; e < 16; e++) v[e] = (W)((threadIdx.x * 977u + e * 131u) % (u32)q);
    W w[4], ws[4];
    for (int i = 0; i < 4; i++) {
        w[i] = tw[2 * i];
        ws[i] = tw[2 * i + 1];
    }
    const W mu = tw[8];  // Barrett constant floor(2^bits / q)
    const W q2 = 2 * q;
    for (int it = 0; it < rounds; it++) {
#pragma unroll
        for (int s = 0; s < 12; s++) {
            const int h = 1 << (s & 3);
#pragma unroll
            for (int e = 0; e < 16; e++) {
                if (e & h) continue;
                if (FORM == 0)
                    ct<W>(v[e], v[e | h], w[s & 3], ws[s & 3], q, q2);
                else
                    gs<W>(v[e], v[e | h], w[s & 3], ws[s & 3], q, q2);
            }
        }
        if (FORM == 0) {
            // the forward transform's single final reduction (Barrett)
#pragma unroll
            for (int e = 0; e < 16; e++) {
                W r = v[e] - Wide<W>::hi(v[e], mu) * q;
                r = r >= q ? r - q : r;
                v[e] = r >= q ? r - q : r;
            }
        }
    }
    W s = 0;
    for (int e = 0; e < 16; e++) s ^= v[e];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename W>
static void run(const char* name, int form, W q, int sms, double mhz, W* out) {
    W h[9];
    for (int i = 0; i < 4; i++) {
        const W w = (W)((123456789ull * (i + 1)) % (u64)q);
        h[2 * i] = w;
        h[2 * i + 1] = (W)((((unsigned __int128)w) << (8 * sizeof(W))) / q);
    }
    h[8] = (W)((((unsigned __int128)1) << (8 * sizeof(W))) / q);
    W* tw;
    cudaMalloc(&tw, sizeof(h));
    cudaMemcpy(tw, h, sizeof(h), cudaMemcpyHostToDevice);
    const int threads = 512, blocks = sms, rounds = 512;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(a);
        if (form == 0)
            k_bfly<W, 0><<<blocks, threads>>>(tw, out, rounds, q);
        else
            k_bfly<W, 1><<<blocks, threads>>>(tw, out, rounds, q);
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    const double bf = (double)blocks * threads * rounds * 12 * 8;
    printf("%-5s %8.1f G butterflies/s  %5.2f per clock per SM at %.0f MHz\n", name, bf / best / 1e6,
           bf / (best * 1e-3) / sms / (mhz * 1e6), mhz);
    cudaFree(tw);
}

int main(int argc, char** argv) {
    const double mhz = argc > 1 ? atof(argv[1]) : 2070.0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    void* out;
    if (cudaMalloc(&out, (size_t)sms * 512 * sizeof(u64)) != cudaSuccess) return 1;
    // one 512-thread block per SM, like the external-product kernels
    run<u64>("ct64", 0, 1125899906826241ull, sms, mhz, (u64*)out);
    run<u64>("gs64", 1, 1125899906826241ull, sms, mhz, (u64*)out);
    run<u32>("ct32", 0, 1073479681u, sms, mhz, (u32*)out);
    run<u32>("gs32", 1, 1073479681u, sms, mhz, (u32*)out);
    const cudaError_t e = cudaGetLastError();
    printf("status: %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
