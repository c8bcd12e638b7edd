// hw_ext.cuh -- the kernels built on the external product, templated on the
// context's geometry (2^LOGE residues per thread, NP polynomials per
// transform): RGSW encryption, IVP training, VP inference (with horizontal
// packing), the class-count IVP of dataset balancing and inference against a
// model in clear.  Each ring size's translation unit instantiates its
// geometries and exposes them as a table of launchers (ExtOps) that the
// context picks from.
#pragma once
#include "cdt.cuh"
#include "hw_internal.cuh"
#include "hw_launch.h"

#include <cstring>

// Encrypted bit slot that drives LUT-index bit t of RAM j: label bits first
// (slots 0..L-1), then the RAM's tuple bits; -1 for a constant-0 bit.
__device__ __forceinline__ int bit_slot(const DevCtx& C, int j, int t) {
    return t < C.L ? t : C.ram_slot[(size_t)j * C.a + (t - C.L)];
}

// ---------------------------------------------------------------------------
// EncRGSW.  One block per (sample, bit slot, row).  Row rho < dnum encrypts
// (a, a*s + e + m*g_rho), row dnum+rho encrypts (a + m*g_rho, a*s + e); the
// gadget value g_rho sits at prime rho/dpp only.  a is uniform per prime and
// drawn at its evaluation points (a uniform value at every root of X^N + 1
// is a uniform a): sampling point k, the root psi_min^(2 brv(k) + 1), takes
// two 64-bit words of block k >> 1 -> 128-bit value mod q, so a needs no
// transform.  e is one integer polynomial for all primes, transformed per
// prime.  Rows are stored in evaluation form, Montgomery representation.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP>::T, ExtCfg<LOGN, LOGE, NP>::MINB)
    k_encrypt(const DevCtx* __restrict__ Cp, const u64* __restrict__ key,
              const uint8_t* __restrict__ bits, const uint32_t* __restrict__ labels, int slot0,
              int n_enc_slots, u64 seed, u64 first, u64* __restrict__ out) {
    using X = ExtCfg<LOGN, LOGE, NP>;
    constexpr int N = Ring<LOGN>::N, E = 1 << LOGE, T = X::T;
    extern __shared__ u64 smem[];
    Xchg xc{smem, smem + NP * X::PADDED, X::PADDED, 0};
    u64* A = smem + 2 * NP * X::PADDED;
    int8_t* ebuf = (int8_t*)(A + N);
    const DevCtx& C = *Cp;
    const int r = C.r, tid = threadIdx.x;
    const int rows = 2 * C.dnum;
    const size_t bid = blockIdx.x;
    const int row = (int)(bid % rows);
    const size_t rest = bid / rows;
    const int slot = slot0 + (int)(rest % n_enc_slots);
    const size_t i = rest / n_enc_slots;
    const int bit = slot < C.L ? (int)((labels[i] >> slot) & 1u)
                               : (int)bits[i * C.n_data + (slot - C.L)];
    const u64 stream = (first + i) * (u64)C.n_slots + (u64)slot;
    for (int c0 = tid; c0 < N / 4; c0 += T) {
        Philox4 w = hw_draw(seed, HW_TAG_RGSW_E, (u64)c0, (u64)row, stream);
#pragma unroll
        for (int t = 0; t < 4; t++) ebuf[4 * c0 + t] = (int8_t)gaussian_from_word(w.v[t]);
    }
    const int rho = row % C.dnum;
    const int gi = rho / C.dpp;
    u64* dst_row = out + i * C.sample_words + (size_t)slot * C.rgsw_words + (size_t)row * C.rlwe_words;
    for (int j = 0; j < r; j++) {
        const PrimeConst P = C.P[j];
        const u64 q = P.q;
        __syncthreads();  // ebuf is complete
        // the whole row is computed in Montgomery form (x R mod q, the form
        // it is stored in): a uniform draw hi*2^64 + lo gives
        // a R = hi (R^2 mod q) + lo (R mod q), two products by constants; the
        // transform is linear, so it keeps the form
        const u64 mr = C.mr[j], mr_s = C.mr_s[j], mr2_s = C.mr2_s[j];
        const uint32_t amul = C.a_point_mul[j];
        const u64 gM = (bit && j == gi) ? to_mont(C.gconst[rho], P) : 0;
        const u64* sM = key + (size_t)(r + j) * N;
        u64* da = dst_row + (size_t)(0 * r + j) * N;
        u64* db = dst_row + (size_t)(1 * r + j) * N;
        // a at evaluation positions E*tid + e and E*tid + e + 1 (addresses
        // e*T + tid, thread-major): their points differ by the factor -1, so
        // their sampling points are k and k ^ 1, one Philox block.  a s
        // waits in A (each thread's own addresses) while e is transformed
#pragma unroll
        for (int e = 0; e < E; e += 2) {
            const uint32_t pos = (uint32_t)(E * tid + e);
            const uint32_t x = 2u * (__brev(pos) >> (32 - LOGN)) + 1u;
            const uint32_t y = (amul * x) & (2u * N - 1u);
            const uint32_t k = __brev(y >> 1) >> (32 - LOGN);
            const Philox4 w = hw_draw(seed, HW_TAG_RGSW_A, (u64)(k >> 1), (u64)(row * r + j), stream);
            const int h = 2 * (int)(k & 1u);
            const u64 a0 = add_mod(shoup_mul(w.v[h], P.r2, mr2_s, q), shoup_mul(w.v[h + 1], mr, mr_s, q), q);
            const u64 a1 =
                add_mod(shoup_mul(w.v[2 - h], P.r2, mr2_s, q), shoup_mul(w.v[3 - h], mr, mr_s, q), q);
            const int ad0 = e * T + tid, ad1 = (e + 1) * T + tid;
            A[ad0] = mont_mul(a0, sM[ad0], P);  // REDC(aR * sR) = a s R
            A[ad1] = mont_mul(a1, sM[ad1], P);
            // the evaluation form of the constant polynomial g is g everywhere
            da[ad0] = row < C.dnum ? a0 : add_mod(a0, gM, q);
            da[ad1] = row < C.dnum ? a1 : add_mod(a1, gM, q);
        }
        u64 v[1][E];
#pragma unroll
        for (int kk = 0; kk < E; kk++) {
            const int x = tid + kk * T;
            v[0][kk] = shoup_mul(from_signed((int64_t)ebuf[x], q), mr, mr_s, q);  // e R
        }
        bool done = false;
        if constexpr (LOGN <= 11) {
            if (C.ext32) {  // primes below 2^30: the same transform in 32-bit words
                u32 w[1][E];
#pragma unroll
                for (int kk = 0; kk < E; kk++) w[0][kk] = (u32)v[0][kk];
                fwd_from32<LOGN, LOGE, 1, 0>(w, xc, C.tw32_fwd + (size_t)j * N, (u32)q, 2 * (u32)q);
#pragma unroll
                for (int e = 0; e < E; e++) v[0][e] = w[0][e];  // < 4q, reduced below
                done = true;
            }
        }
        if (!done) ntt_fwd<LOGN, LOGE, 1>(v, xc, C, j);
#pragma unroll
        for (int e = 0; e < E; e++) {
            const int ad = e * T + tid;
            const u64 bM = add_mod(A[ad], reduce_full(v[0][e], P), q);
            db[ad] = row < C.dnum ? add_mod(bM, gM, q) : bM;
        }
    }
}

// ---------------------------------------------------------------------------
// IVP training.  One thread block per work item (sample i, RAM j), persistent
// over items.  For each item: acc = (0, Delta); for each rotation bit t in
// z..L+a-1 with an encrypted control C_t: acc <- acc + C_t [x] (acc X^{2^(t-z)}
// - acc) (BlindRotate with weights -2^k); then the CDEMUX tree over bits
// 0..z-1, level i splitting L_j into (L_j - C_i [x] L_j, C_i [x] L_j).
// Outputs: the item's k1 stored ciphertexts are added into H[j] with 64-bit
// atomic adds of the residues, unreduced (exact integer sums: the order in
// which the batch's items arrive does not change them); the caller reduces
// H mod q_i afterwards and keeps (n + 1) q_i < 2^64.
// Per-block scratch: two accumulators, their evaluation form (outside mode
// 1), the evaluation forms of the k1 tree slots and the k1 tree slots.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP, SM>::T, ExtCfg<LOGN, LOGE, NP, SM>::MINB)
    k_ivp_train(const DevCtx* __restrict__ Cp, const u64* __restrict__ rgsw, int n_items,
                u64* __restrict__ model, u64* __restrict__ scratch) {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, (SM == 1 || SM == 2) ? smem : smem + NP * X::PADDED, X::PADDED, 0};
    if (SM == 2) xc.accs = smem + NP * X::PADDED;
    if (SM == 3) xc.accs = smem + 2 * NP * X::PADDED;
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, T = blockDim.x;
    const size_t rl = C.rlwe_words;
    constexpr int NB = SM == 1 ? 2 : 3;  // per-block RLWE buffers besides the tree
    u64* blk = scratch + (size_t)blockIdx.x * (NB + 2 * C.k1) * rl;
    u64* acc[2] = {blk, blk + rl};
    // one evaluation-form buffer (in shared memory in mode 1), updated in
    // place: the external product reads each thread's own words of a prime
    // before it writes them
    u64* accn = SM == 1 ? smem + NP * X::PADDED : blk + 2 * rl;
    u64* tn = blk + NB * rl;  // evaluation forms of the tree slots
    u64* Lout = tn + (size_t)C.k1 * rl;  // the tree slots (the item's outputs)
    const int kbits = C.L + C.a;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int i = item / C.k0, j = item % C.k0;
        const u64* sample = rgsw + (size_t)i * C.sample_words;
        // last encrypted rotation bit: its CMUX writes straight into slot 0
        int last = -1;
        for (int t = C.z; t < kbits; t++)
            if (bit_slot(C, j, t) >= 0) last = t;
        // acc = trivial RLWE (0, Delta * 1); its evaluation form is Delta everywhere in b
        u64* first_dst = last >= 0 ? acc[0] : Lout;
        u64* first_ntt = last >= 0 ? accn : tn;
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
            u64* dstn = (t == last) ? tn : accn;
            int nslot = -1;  // the next encrypted control (rotation bit or first tree gate)
            for (int t2 = t + 1; t2 < kbits && nslot < 0; t2++) nslot = bit_slot(C, j, t2);
            if (nslot < 0 && C.n_gates > 0) nslot = bit_slot(C, j, C.gate_lvl[0]);
            ext_product<LOGN, LOGE, NP, X::ACC>(
                C, sample + (size_t)slot * C.rgsw_words, acc[cur], w, acc[cur], 0, EXT_ADD, dst, xc,
                ExtNtt{accn, dstn, t - C.z, 0,
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
            ext_product<LOGN, LOGE, NP, X::ACC>(
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
        // the item's stored ciphertexts into H[j] (the last CMUX or gate
        // ended with a barrier, so Lout is complete)
        unsigned long long* Hj = (unsigned long long*)(model + (size_t)j * C.k1 * rl);
        for (size_t w = tid; w < (size_t)C.k1 * rl; w += T) atomicAdd(Hj + w, (unsigned long long)Lout[w]);
        __syncthreads();  // Lout is read before the next item rewrites it
    }
}

// ExtractLWE(ct, k) written by the block: the LWE of coefficient k of the
// phase, a'_y = a_{k-y} for y <= k, -a_{N+k-y} otherwise, b' = b_k (per
// prime, [prime][N a'-coefficients, b']).
__device__ __forceinline__ void extract_lwe_at(const DevCtx& C, const u64* ct, int k, u64* lw) {
    const int tid = threadIdx.x, T = blockDim.x;
    for (int jp = 0; jp < C.r; jp++) {
        const u64 q = C.P[jp].q;
        const u64* pa = ct + (size_t)jp * C.n;
        u64* o = lw + (size_t)jp * (C.n + 1);
        for (int y = tid; y < C.n; y += T) {
            const int x = k - y;
            o[y] = x >= 0 ? pa[x] : neg_mod(pa[x + C.n], q);
        }
        if (tid == 0) o[C.n] = ct[(size_t)(C.r + jp) * C.n + k];
    }
}

// ---------------------------------------------------------------------------
// VP inference.  One thread block per item (sample i, RAM j, class c).
// Label bits are in clear: tree levels driven by label bits select a stored
// ciphertext directly; a tree level driven by an encrypted address bit (z > L)
// is a CMUX(C, L_{v+n}, L_v); label bits among the rotation bits are a plain
// rotation X^-(c >> z).  The encrypted address bits then blind-rotate with
// weights +2^k (X^-2^k) and the last CMUX writes ExtractLWE(., 0) directly.
// Per-block scratch: two accumulators and their evaluation forms.  With
// `digits` (from k_vp_digits) the first CMUX of item (RAM j, class c) --
// the encrypted tree level's when z > L, else the first rotation's -- takes
// its digits' transforms from digits + (j G + c) 2 dnum r N: its source is
// made of stored ciphertexts only, the same for every sample of the batch.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM, int PK>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP, SM>::T, ExtCfg<LOGN, LOGE, NP, SM>::MINB)
    k_vp_infer(const DevCtx* __restrict__ Cp, const u64* __restrict__ model,
               const u64* __restrict__ rgsw, int n_items, u64* __restrict__ resp,
               u64* __restrict__ scratch, const u64* __restrict__ digits) {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, (SM == 1 || SM == 2) ? smem : smem + NP * X::PADDED, X::PADDED, 0};
    if (SM == 2) xc.accs = smem + NP * X::PADDED;
    if (SM == 3) xc.accs = smem + 2 * NP * X::PADDED;
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, T = blockDim.x;
    const size_t rl = C.rlwe_words;
    const int two_n = 2 * C.n;
    u64* blk = scratch + (size_t)blockIdx.x * (SM == 1 ? 2 : 3) * rl;
    u64* acc[2] = {blk, blk + rl};
    // one evaluation-form buffer (in shared memory in mode 1), updated in
    // place (see k_ivp_train)
    u64* accn = SM == 1 ? smem + NP * X::PADDED : blk + 2 * rl;
    const int kbits = C.L + C.a;
    const int l = C.n_classes;
    // PK (horizontal packing, z <= L only): one item per group of classes
    // sharing a stored ciphertext (c = g mod 2^z); their clear label bits
    // above z are not rotated, so class c's lookup is coefficient c >> z of
    // the accumulator
    const int G = PK ? (l < (1 << C.z) ? l : (1 << C.z)) : l;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int c = item % G;  // the class, or the group residue with PK
        const int ij = item / G;
        const int i = ij / C.k0, j = ij % C.k0;
        const u64* sample = rgsw + (size_t)i * C.sample_words;
        const u64* Hj = model + (size_t)j * C.k1 * rl;
        // items run class-fastest (the l classes of a (sample, RAM) share its
        // RGSW bits); responses are stored [sample][class][RAM]
        u64* lwe = resp + (((size_t)i * l + c) * C.k0 + j) * C.lwe_words;
        [[maybe_unused]] const size_t class_stride = (size_t)C.k0 * C.lwe_words;  // next class's response
        const u64* src;
        const u64* srcn = nullptr;  // evaluation form of src, once known
        int e0;
        if (C.z <= C.L) {
            src = Hj + (size_t)C.slot_of[c & ((1 << C.z) - 1)] * rl;
            const int R = PK ? 0 : c >> C.z;  // clear label bits among the rotation bits
            e0 = (two_n - R) % two_n;
        } else {
            // one encrypted tree level (bit z-1, an address bit): CMUX(C, L_{v+n}, L_v)
            const int nn = 1 << (C.z - 1);
            const u64* lo = Hj + (size_t)C.slot_of[c] * rl;
            const u64* hi = Hj + (size_t)C.slot_of[c + nn] * rl;
            const int slot = bit_slot(C, j, C.z - 1);
            if (slot < 0) {
                src = lo;
            } else if (digits) {  // the digits of hi - lo, transformed once per batch
                ext_product<LOGN, LOGE, NP, X::ACC, true>(
                    C, sample + (size_t)slot * C.rgsw_words, hi, 0, lo, 0, EXT_ADD, acc[0], xc,
                    ExtNtt{nullptr, nullptr, -1, 0, nullptr, 0,
                           digits + ((size_t)j * G + c) * (size_t)(2 * C.dnum * C.r) * C.n});
                src = acc[0];
            } else {
                ext_product<LOGN, LOGE, NP, X::ACC>(C, sample + (size_t)slot * C.rgsw_words, hi, 0, lo,
                                                  0, EXT_ADD, acc[0], xc,
                                                  ExtNtt{nullptr, nullptr, -1, 0, nullptr, 0});
                src = acc[0];
            }
            e0 = 0;
        }
        int last = -1;
        for (int t = (C.z > C.L ? C.z : C.L); t < kbits; t++)
            if (bit_slot(C, j, t) >= 0) last = t;
        if constexpr (PK) {
            if (last < 0) {  // nothing encrypted left: extract every class of the group
                for (int cc = c, k = 0; cc < l; cc += 1 << C.z, k++)
                    extract_lwe_at(C, src, k, lwe + (size_t)(cc - c) * class_stride);
                __syncthreads();
                continue;
            }
        }
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
        const u64* dg = (digits && C.z <= C.L)
                            ? digits + ((size_t)j * G + c) * (size_t)(2 * C.dnum * C.r) * C.n
                            : nullptr;
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
            const ExtNtt nt{srcn, t == last ? nullptr : accn, t - C.z, 1,
                            nslot >= 0 ? sample + (size_t)nslot * C.rgsw_words : nullptr, 0, dg};
            const u64* ct = sample + (size_t)slot * C.rgsw_words;
            const bool to_lwe = !PK && t == last;
            u64* dst = to_lwe ? lwe : acc[cur ^ 1];
            const int mode = to_lwe ? EXT_LWE : EXT_ADD;
            if (dg)  // the first CMUX, its digit transforms given
                ext_product<LOGN, LOGE, NP, X::ACC, true>(C, ct, src, eA, src, e0, mode, dst, xc, nt);
            else if (to_lwe)  // the last CMUX, straight into ExtractLWE(., 0)
                ext_product<LOGN, LOGE, NP, X::ACC, false, true>(C, ct, src, eA, src, e0, mode, dst, xc, nt);
            else
                ext_product<LOGN, LOGE, NP, X::ACC>(C, ct, src, eA, src, e0, mode, dst, xc, nt);
            dg = nullptr;
            if (PK && t == last) {
                for (int cc = c, k = 0; cc < l; cc += 1 << C.z, k++)
                    extract_lwe_at(C, acc[cur ^ 1], k, lwe + (size_t)(cc - c) * class_stride);
                __syncthreads();
            } else if (t != last) {
                src = acc[cur ^ 1];
                srcn = accn;
                cur ^= 1;
            }
            e0 = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// The first CMUX's digit transforms of every (RAM j, class c) item of VP:
// its source is the stored ciphertext H[j][c mod 2^z] rotated by the clear
// label bits (z <= L), or the difference of the two stored ciphertexts the
// encrypted tree level selects between (z > L), the same for every sample,
// so the 2 dnum r forward transforms are computed once per batch;
// k_vp_infer reads them.  Item j G + c (G classes, or groups with PK)
// writes digits + item 2 dnum r N.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM, int PK>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP, SM>::T, ExtCfg<LOGN, LOGE, NP, SM>::MINB)
    k_vp_digits(const DevCtx* __restrict__ Cp, const u64* __restrict__ model, int n_items,
                u64* __restrict__ digits) {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, (SM == 1 || SM == 2) ? smem : smem + NP * X::PADDED, X::PADDED, 0};
    const DevCtx& C = *Cp;
    const int two_n = 2 * C.n, l = C.n_classes, kbits = C.L + C.a;
    const size_t rl = C.rlwe_words;
    const int G = PK ? (l < (1 << C.z) ? l : (1 << C.z)) : l;
    const size_t per = (size_t)2 * C.dnum * C.r * C.n;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int c = item % G, j = item / G;
        if (C.z > C.L) {  // the encrypted tree level's CMUX: D = H[j][c + 2^(z-1)] - H[j][c]
            if (bit_slot(C, j, C.z - 1) < 0) continue;  // a constant-0 bit: no CMUX
            const u64* Hj = model + (size_t)j * C.k1 * rl;
            ext_digits<LOGN, LOGE, NP>(C, Hj + (size_t)C.slot_of[c + (1 << (C.z - 1))] * rl, 0,
                                       Hj + (size_t)C.slot_of[c] * rl, 0, xc, digits + (size_t)item * per);
            continue;
        }
        const u64* src = model + (size_t)j * C.k1 * rl + (size_t)C.slot_of[c & ((1 << C.z) - 1)] * rl;
        const int R = PK ? 0 : c >> C.z;
        const int e0 = (two_n - R) % two_n;
        int t0 = -1;
        for (int t = C.L; t < kbits && t0 < 0; t++)
            if (bit_slot(C, j, t) >= 0) t0 = t;
        if (t0 < 0) continue;  // nothing encrypted: VP extracts directly
        const int eA = (e0 + two_n - (1 << (t0 - C.z))) % two_n;
        ext_digits<LOGN, LOGE, NP>(C, src, eA, src, e0, xc, digits + (size_t)item * per);
    }
}

// ---------------------------------------------------------------------------
// Dataset balancing (Section 3.6.1): a small IVP over the label bits of each
// sample.  One block per sample, persistent: acc = (0, Delta); for each label
// bit t: acc <- acc + C_t [x] (acc X^(2^t) - acc) (IVP direction); the result,
// Delta at coefficient = label, goes to out[sample] and a reduction adds the
// batch into the class-count ciphertext.  Per-block scratch as for VP.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP, SM>::T, ExtCfg<LOGN, LOGE, NP, SM>::MINB)
    k_count_classes(const DevCtx* __restrict__ Cp, const u64* __restrict__ rgsw, int n_items,
                    u64* __restrict__ out, u64* __restrict__ scratch) {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    extern __shared__ u64 smem[];
    Xchg xc{smem, (SM == 1 || SM == 2) ? smem : smem + NP * X::PADDED, X::PADDED, 0};
    if (SM == 2) xc.accs = smem + NP * X::PADDED;
    if (SM == 3) xc.accs = smem + 2 * NP * X::PADDED;
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, T = blockDim.x;
    const size_t rl = C.rlwe_words;
    u64* blk = scratch + (size_t)blockIdx.x * (SM == 1 ? 2 : 3) * rl;
    u64* acc[2] = {blk, blk + rl};
    u64* accn = SM == 1 ? smem + NP * X::PADDED : blk + 2 * rl;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const u64* sample = rgsw + (size_t)item * C.sample_words;
        u64* res = out + (size_t)item * rl;
        for (size_t w = tid; w < rl; w += T) {
            const size_t comp = w / ((size_t)C.r * C.n), rem = w % ((size_t)C.r * C.n);
            const int p = (int)(rem / C.n), x = (int)(rem % C.n);
            acc[0][w] = (comp == 1 && x == 0) ? C.delta[p] : 0;
            accn[w] = comp == 1 ? C.delta[p] : 0;
        }
        __syncthreads();
        int cur = 0;
        for (int t = 0; t < C.L; t++) {
            const bool last = t == C.L - 1;
            ext_product<LOGN, LOGE, NP, X::ACC>(
                C, sample + (size_t)t * C.rgsw_words, acc[cur], 1 << t, acc[cur], 0, EXT_ADD,
                last ? res : acc[cur ^ 1], xc,
                ExtNtt{accn, last ? nullptr : accn, t, 0,
                       last ? nullptr : sample + (size_t)(t + 1) * C.rgsw_words, 1});
            cur ^= 1;
        }
    }
}

// Evaluation form of an RLWE (2 r polynomials, fully reduced, thread-major
// positions) written by the block.
template <int LOGN, int LOGE, int NP>
__device__ __forceinline__ void rlwe_to_eval(const DevCtx& C, const u64* src, u64* dstn, Xchg& xc) {
    constexpr int N = Ring<LOGN, LOGE>::N, T = Ring<LOGN, LOGE>::T, E = 1 << LOGE;
    constexpr int NPI = NP < 2 ? NP : 2;  // the two components together
    const int tid = threadIdx.x, r = C.r;
    for (int jp = 0; jp < r; jp++) {
        const PrimeConst P = C.P[jp];
        for (int oc0 = 0; oc0 < 2; oc0 += NPI) {
            u64 v[NPI][E];
#pragma unroll
            for (int pp = 0; pp < NPI; pp++)
#pragma unroll
                for (int kk = 0; kk < E; kk++) v[pp][kk] = src[((size_t)(oc0 + pp) * r + jp) * N + tid + kk * T];
            ntt_fwd<LOGN, LOGE, NPI>(v, xc, C, jp);
#pragma unroll
            for (int pp = 0; pp < NPI; pp++)
#pragma unroll
                for (int e = 0; e < E; e++)
                    dstn[((size_t)(oc0 + pp) * r + jp) * N + e * T + tid] = reduce_full(v[pp][e], P);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Inference against a model in clear (Section 3.6.2).  One block per item
// (sample i, RAM j), persistent over items.  The lookup tables are
// plaintexts, so the blind rotation depends only on the sample:
// R = (0, Delta) rotated by address bits zt..a-1 (zt = max(0, z - L)) with
// weights +2^0, +2^1, ... (X^-2^k), in evaluation form afterwards.  For every
// class c the products R * T_{j,c,v} with its tables (plain: [RAM][class]
// [leaf v < 2^zt][prime][N], evaluation form, Montgomery) give its response:
// zt = 0: ExtractLWE(R * T, 0) -- the a part transformed back, b' = coefficient
// 0 of R_b * T, N^-1 times the sum of its evaluation values;
// zt = 1: ExtractLWE(CMUX(C, R T_1, R T_0), 0) with address bit 0 in control.
// Responses are stored [sample][class][RAM] as VP's.  Per-block scratch as for
// VP: two RLWEs (the rotation, then the two tree inputs) and, outside mode 1,
// the evaluation form of R.
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM>
__global__ void __launch_bounds__(ExtCfg<LOGN, LOGE, NP, SM>::T, ExtCfg<LOGN, LOGE, NP, SM>::MINB)
    k_vp_plain(const DevCtx* __restrict__ Cp, const u64* __restrict__ plain,
               const u64* __restrict__ rgsw, int n_items, u64* __restrict__ resp,
               u64* __restrict__ scratch) {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    constexpr int N = Ring<LOGN>::N, E = 1 << LOGE, T = X::T;
    constexpr int NPI = NP < 2 ? NP : 2;
    extern __shared__ u64 smem[];
    Xchg xc{smem, (SM == 1 || SM == 2) ? smem : smem + NP * X::PADDED, X::PADDED, 0};
    if (SM == 2) xc.accs = smem + NP * X::PADDED;
    if (SM == 3) xc.accs = smem + 2 * NP * X::PADDED;
    const DevCtx& C = *Cp;
    const int tid = threadIdx.x, r = C.r, l = C.n_classes;
    const size_t rl = C.rlwe_words;
    u64* blk = scratch + (size_t)blockIdx.x * (SM == 1 ? 2 : 3) * rl;
    u64* acc[2] = {blk, blk + rl};
    u64* accn = SM == 1 ? smem + NP * X::PADDED : blk + 2 * rl;
    const int zt = C.z > C.L ? C.z - C.L : 0;
    const int nleaf = 1 << zt;
    const int kbits = C.L + C.a;
    const int t0 = C.L + zt;  // LUT-index bit of the first rotation bit
    u64* red = xc.b0;         // block reduction of the b' sums (between transforms)
    constexpr int NR = T >= 32 ? T / 32 : T;  // partial sums per class and prime
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int i = item / C.k0, j = item % C.k0;
        const u64* sample = rgsw + (size_t)i * C.sample_words;
        for (size_t w = tid; w < rl; w += T) {
            const size_t comp = w / ((size_t)r * N), rem = w % ((size_t)r * N);
            const int p = (int)(rem / N), x = (int)(rem % N);
            acc[0][w] = (comp == 1 && x == 0) ? C.delta[p] : 0;
            accn[w] = comp == 1 ? C.delta[p] : 0;
        }
        __syncthreads();
        int cur = 0;
        bool rotated = false;
        for (int t = t0; t < kbits; t++) {
            const int slot = bit_slot(C, j, t);
            if (slot < 0) continue;  // constant-0 address bit: no rotation
            const int k = t - t0;
            int nslot = -1;
            for (int t2 = t + 1; t2 < kbits && nslot < 0; t2++) nslot = bit_slot(C, j, t2);
            if (nslot < 0 && zt > 0) nslot = bit_slot(C, j, C.L);
            ext_product<LOGN, LOGE, NP, X::ACC>(
                C, sample + (size_t)slot * C.rgsw_words, acc[cur], 2 * N - (1 << k), acc[cur], 0, EXT_ADD,
                acc[cur ^ 1], xc,
                ExtNtt{accn, accn, k, 1, nslot >= 0 ? sample + (size_t)nslot * C.rgsw_words : nullptr, 1});
            cur ^= 1;
            rotated = true;
        }
        // with one digit per prime the products kept accn up to date
        if (rotated && !C.diag) rlwe_to_eval<LOGN, LOGE, NP>(C, acc[cur], accn, xc);
        const u64* Tj = plain + (size_t)j * l * nleaf * r * N;
        if (zt == 0) {
            for (int c0 = 0; c0 < l; c0 += NP) {
                // b' = N^-1 sum_k (R_b * T)^_k, per class and prime: per-thread
                // partial sums, reduced over each warp, then over the warps
                __syncthreads();  // the exchange buffer (red) is free
#pragma unroll
                for (int pp = 0; pp < NP; pp++)
                    for (int jp = 0; jp < r; jp++) {
                        const PrimeConst P = C.P[jp];
                        const int c = c0 + pp < l ? c0 + pp : l - 1;
                        const u64* rb = accn + (size_t)(r + jp) * N + tid;
                        const u64* tm = Tj + ((size_t)c * r + jp) * N + tid;
                        u64 sacc = 0;
#pragma unroll
                        for (int e = 0; e < E; e++) sacc = add_mod(sacc, mont_mul(rb[e * T], tm[e * T], P), P.q);
                        if constexpr (T >= 32) {
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1)
                                sacc = add_mod(sacc, __shfl_down_sync(0xffffffffu, sacc, off), P.q);
                            if ((tid & 31) == 0) red[(pp * HW_MAXP + jp) * NR + (tid >> 5)] = sacc;
                        } else {
                            red[(pp * HW_MAXP + jp) * NR + tid] = sacc;
                        }
                    }
                __syncthreads();
                for (int idx = tid; idx < NP * r; idx += T) {
                    const int pp = idx / r, jp = idx % r, c = c0 + pp;
                    if (c < l) {
                        const PrimeConst P = C.P[jp];
                        u64 sacc = 0;
                        for (int w = 0; w < NR; w++) sacc = add_mod(sacc, red[(pp * HW_MAXP + jp) * NR + w], P.q);
                        u64* lw = resp + (((size_t)i * l + c) * C.k0 + j) * C.lwe_words + (size_t)jp * (N + 1);
                        lw[N] = shoup_mul(sacc, C.n_inv[jp], C.n_inv_s[jp], P.q);
                    }
                }
                __syncthreads();  // red is read before the transforms reuse the buffer
                // a': the a parts of NP classes transformed back together
                for (int jp = 0; jp < r; jp++) {
                    const PrimeConst P = C.P[jp];
                    const u64 q = P.q, ninv = C.n_inv[jp], ninv_s = C.n_inv_s[jp];
                    const u64* ra = accn + (size_t)jp * N + tid;
                    u64 v[NP][E];
#pragma unroll
                    for (int pp = 0; pp < NP; pp++) {
                        const int c = c0 + pp < l ? c0 + pp : l - 1;
                        const u64* tm = Tj + ((size_t)c * r + jp) * N + tid;
#pragma unroll
                        for (int e = 0; e < E; e++)
                            v[pp][e] = shoup_mul_lazy(mont_mul(ra[e * T], tm[e * T], P), ninv, ninv_s, q);
                    }
                    ntt_inv<LOGN, LOGE, NP>(v, xc, C, jp);
#pragma unroll
                    for (int pp = 0; pp < NP; pp++) {
                        const int c = c0 + pp;
                        if (c >= l) continue;
                        u64* lw = resp + (((size_t)i * l + c) * C.k0 + j) * C.lwe_words + (size_t)jp * (N + 1);
#pragma unroll
                        for (int kk = 0; kk < E; kk++) {
                            const int x = tid + kk * T;
                            const u64 val = v[pp][kk] >= q ? v[pp][kk] - q : v[pp][kk];
                            if (x == 0)
                                lw[0] = val;
                            else
                                lw[N - x] = neg_mod(val, q);
                        }
                    }
                }
                __syncthreads();
            }
        } else {
            const int tslot = bit_slot(C, j, C.L);  // address bit 0 drives the tree
            for (int c = 0; c < l; c++) {
                u64* lwe = resp + (((size_t)i * l + c) * C.k0 + j) * C.lwe_words;
                // the two leaves R * T_0 -> acc[0], R * T_1 -> acc[1], coefficient form
                for (int v = 0; v < 2; v++)
                    for (int jp = 0; jp < r; jp++) {
                        const PrimeConst P = C.P[jp];
                        const u64 q = P.q, ninv = C.n_inv[jp], ninv_s = C.n_inv_s[jp];
                        const u64* tm = Tj + (((size_t)c * nleaf + v) * r + jp) * N + tid;
                        for (int oc0 = 0; oc0 < 2; oc0 += NPI) {
                            u64 w[NPI][E];
#pragma unroll
                            for (int pp = 0; pp < NPI; pp++) {
                                const u64* rc = accn + ((size_t)(oc0 + pp) * r + jp) * N + tid;
#pragma unroll
                                for (int e = 0; e < E; e++)
                                    w[pp][e] = shoup_mul_lazy(mont_mul(rc[e * T], tm[e * T], P), ninv, ninv_s, q);
                            }
                            ntt_inv<LOGN, LOGE, NPI>(w, xc, C, jp);
#pragma unroll
                            for (int pp = 0; pp < NPI; pp++) {
                                u64* dd = acc[v] + ((size_t)(oc0 + pp) * r + jp) * N;
#pragma unroll
                                for (int kk = 0; kk < E; kk++)
                                    dd[tid + kk * T] = w[pp][kk] >= q ? w[pp][kk] - q : w[pp][kk];
                            }
                        }
                    }
                __syncthreads();
                if (tslot < 0) {  // constant-0 control: the CMUX keeps leaf 0
                    extract_lwe_at(C, acc[0], 0, lwe);
                    __syncthreads();
                } else {
                    ext_product<LOGN, LOGE, NP, X::ACC>(C, sample + (size_t)tslot * C.rgsw_words, acc[1], 0,
                                                      acc[0], 0, EXT_LWE, lwe, xc,
                                                      ExtNtt{nullptr, nullptr, -1, 0, nullptr, 0});
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launch table of one geometry
// ---------------------------------------------------------------------------
template <int LOGN, int LOGE, int NP, int SM>
struct ExtVariant {
    using X = ExtCfg<LOGN, LOGE, NP, SM>;
    using XE = ExtCfg<LOGN, LOGE, NP, 0>;  // encryption keeps nothing else in shared memory
    static constexpr size_t ENC_SMEM = XE::XCHG_BYTES + (size_t)Ring<LOGN>::N * 9;
    static constexpr int MAX_SMEM = 227 * 1024;

    static cudaError_t init() {
        cudaError_t e = cudaFuncSetAttribute(k_encrypt<LOGN, LOGE, NP>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ENC_SMEM);
        const int smem = SM == 1 ? MAX_SMEM : (int)X::FIXED_BYTES;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_ivp_train<LOGN, LOGE, NP, SM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_vp_infer<LOGN, LOGE, NP, SM, 0>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_vp_infer<LOGN, LOGE, NP, SM, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_vp_digits<LOGN, LOGE, NP, SM, 0>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_vp_digits<LOGN, LOGE, NP, SM, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_count_classes<LOGN, LOGE, NP, SM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_vp_plain<LOGN, LOGE, NP, SM>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        return e;
    }
    // resident blocks per SM of the persistent kernels (the smaller of the
    // two) at `smem` bytes of dynamic shared memory per block
    static int occupancy(size_t smem) {
        int a = 0, b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_ivp_train<LOGN, LOGE, NP, SM>, X::T, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_vp_infer<LOGN, LOGE, NP, SM, 0>, X::T, smem);
        int o = a < b ? a : b;
        return o < 1 ? 1 : o;
    }
    static cudaError_t encrypt(const LaunchInfo& li, const uint64_t* key, const uint8_t* bits,
                               const uint32_t* labels, int slot0, int n_enc, unsigned blocks,
                               uint64_t seed, uint64_t first, uint64_t* out, cudaStream_t st) {
        k_encrypt<LOGN, LOGE, NP><<<blocks, X::T, ENC_SMEM, st>>>(li.dctx, key, bits, labels, slot0, n_enc,
                                                                 seed, first, out);
        return cudaGetLastError();
    }
    // Launch configuration; with li.l2_persist the launch carries an access-
    // policy window over the first `window` bytes of the per-block scratch.
    struct Launch {
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute attr;
        Launch(const LaunchInfo& li, int grid, cudaStream_t st, void* scratch, size_t window) {
            memset(&cfg, 0, sizeof(cfg));
            memset(&attr, 0, sizeof(attr));
            cfg.gridDim = dim3(grid);
            cfg.blockDim = dim3(X::T);
            cfg.dynamicSmemBytes = li.ext_smem;
            cfg.stream = st;
            if (li.l2_persist > 0 && window > 0) {
                if (window > li.l2_window_max) window = li.l2_window_max;
                attr.id = cudaLaunchAttributeAccessPolicyWindow;
                attr.val.accessPolicyWindow.base_ptr = scratch;
                attr.val.accessPolicyWindow.num_bytes = window;
                const double ratio = (double)li.l2_persist / (double)window;
                attr.val.accessPolicyWindow.hitRatio = ratio < 1.0 ? (float)ratio : 1.0f;
                attr.val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
                attr.val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
                cfg.attrs = &attr;
                cfg.numAttrs = 1;
            }
        }
    };
    static constexpr int SCRATCH_RLWE = SM == 1 ? 2 : 3;  // per-block RLWE buffers (inference)
    static cudaError_t ivp(const LaunchInfo& li, const uint64_t* rgsw, int items, uint64_t* out,
                           uint64_t* acc, int grid, cudaStream_t st) {
        // per-block scratch: two accumulators, (their evaluation form,) the tree
        // slots' evaluation forms and the tree slots
        Launch L(li, grid, st, acc, (size_t)grid * (SCRATCH_RLWE + 2 * li.k1) * li.rlwe_words * sizeof(u64));
        return cudaLaunchKernelEx(&L.cfg, k_ivp_train<LOGN, LOGE, NP, SM>, li.dctx, (const u64*)rgsw, items,
                                  (u64*)out, (u64*)acc);
    }
    static cudaError_t vp(const LaunchInfo& li, const uint64_t* model, const uint64_t* rgsw, int items,
                          uint64_t* resp, uint64_t* acc, int grid, int packed, const uint64_t* digits,
                          cudaStream_t st) {
        Launch L(li, grid, st, acc, (size_t)grid * SCRATCH_RLWE * li.rlwe_words * sizeof(u64));
        if (packed)
            return cudaLaunchKernelEx(&L.cfg, k_vp_infer<LOGN, LOGE, NP, SM, 1>, li.dctx, (const u64*)model,
                                      (const u64*)rgsw, items, (u64*)resp, (u64*)acc, (const u64*)digits);
        return cudaLaunchKernelEx(&L.cfg, k_vp_infer<LOGN, LOGE, NP, SM, 0>, li.dctx, (const u64*)model,
                                  (const u64*)rgsw, items, (u64*)resp, (u64*)acc, (const u64*)digits);
    }
    static cudaError_t vp_digits(const LaunchInfo& li, const uint64_t* model, int items, uint64_t* digits,
                                 int grid, int packed, cudaStream_t st) {
        Launch L(li, grid, st, nullptr, 0);
        if (packed)
            return cudaLaunchKernelEx(&L.cfg, k_vp_digits<LOGN, LOGE, NP, SM, 1>, li.dctx, (const u64*)model,
                                      items, (u64*)digits);
        return cudaLaunchKernelEx(&L.cfg, k_vp_digits<LOGN, LOGE, NP, SM, 0>, li.dctx, (const u64*)model,
                                  items, (u64*)digits);
    }
    static cudaError_t vp_plain(const LaunchInfo& li, const uint64_t* plain, const uint64_t* rgsw, int items,
                                uint64_t* resp, uint64_t* acc, int grid, cudaStream_t st) {
        Launch L(li, grid, st, acc, (size_t)grid * SCRATCH_RLWE * li.rlwe_words * sizeof(u64));
        return cudaLaunchKernelEx(&L.cfg, k_vp_plain<LOGN, LOGE, NP, SM>, li.dctx, (const u64*)plain,
                                  (const u64*)rgsw, items, (u64*)resp, (u64*)acc);
    }
    static cudaError_t count(const LaunchInfo& li, const uint64_t* rgsw, int items, uint64_t* out,
                             uint64_t* acc, int grid, cudaStream_t st) {
        Launch L(li, grid, st, acc, 0);
        return cudaLaunchKernelEx(&L.cfg, k_count_classes<LOGN, LOGE, NP, SM>, li.dctx, (const u64*)rgsw,
                                  items, (u64*)out, (u64*)acc);
    }
    static ExtOps ops() {
        return ExtOps{LOGE, NP, SM, SCRATCH_RLWE, X::T, X::FIXED_BYTES, ENC_SMEM, &init, &occupancy,
                      &encrypt, &ivp, &vp, &count, &vp_plain, &vp_digits};
    }
};

#define HW_EXT_VARIANT(L, E, P, M) ExtVariant<L, E, P, M>::ops(),
// Defines hw_ext_table_<L>: the geometries instantiated for N = 2^L.
#define HW_EXT_TABLE(L, LIST)                                 \
    const ExtOps* hw_ext_table_##L(int* count) {              \
        static const ExtOps table[] = {LIST};                 \
        *count = (int)(sizeof(table) / sizeof(table[0]));     \
        return table;                                         \
    }
// Defines hw_ext_table_<L>_p<PART>: one part of the geometries of N = 2^L,
// for ring sizes whose instantiations are split over translation units so
// that they compile in parallel (k_wisard.cu joins the parts, part 0 first).
#define HW_EXT_TABLE_PART(L, PART, LIST)                      \
    const ExtOps* hw_ext_table_##L##_p##PART(int* count) {    \
        static const ExtOps table[] = {LIST};                 \
        *count = (int)(sizeof(table) / sizeof(table[0]));     \
        return table;                                         \
    }
