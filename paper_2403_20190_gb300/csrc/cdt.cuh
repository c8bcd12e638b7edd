// cdt.cuh -- discrete Gaussian sampling for the kernels that encrypt.
#pragma once
#include "cdt_table.h"
#include "hw_internal.cuh"

// The thresholds live in constant memory, statically initialised in every
// translation unit that samples (all threads read the same entry).
static __constant__ u64 c_cdt[HW_CDT_LEN] = {HW_CDT_VALUES};

// Discrete Gaussian G(sigma) by inversion of the cumulative table on the top
// 63 bits of a uniform word: -19 plus the number of thresholds <= u.
__device__ __forceinline__ int gaussian_from_word(u64 w) {
    const u64 u = w >> 1;
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < HW_CDT_LEN; t++) cnt += (u >= c_cdt[t]) ? 1 : 0;
    return cnt - HW_CDT_SUPPORT;
}
