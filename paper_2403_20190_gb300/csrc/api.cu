// api.cu -- host implementation of the C ABI declared in include/hwisard.h.
//
// hw_create derives every parameter of a context (Section 2.4 Setup, read
// as an RNS modulus; Definition 2 for the model shape), builds the transform
// tables, pi_r and the H3 matrix on the host, and uploads them once.  All
// per-sample work runs in the kernels of k_crypto.cu and k_wisard.cu.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hwisard.h"
#include "hw_internal.cuh"
#include "hw_launch.h"

typedef unsigned __int128 u128;

static thread_local std::string g_last_error;

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CUDA_TRY(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(HW_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                              \
    } while (0)

// FNV-1a over a byte range (the context self-check's fingerprint).
static uint64_t fnv1a(const unsigned char* p, size_t n) {
    uint64_t h = 0xcbf29ce484222325ULL;
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 0x100000001b3ULL;
    }
    return h;
}

// Host-side fault injection for tests: with HW_FAULT_ALLOC=k in the
// environment, the k-th device allocation of each hw_create fails as if the
// device were out of memory (the allocation is not attempted).
static cudaError_t ctx_malloc(void** p, size_t bytes, int* nth) {
    ++*nth;
    const char* f = getenv("HW_FAULT_ALLOC");
    if (f && atoi(f) == *nth) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

struct hw_ctx {
    hw_params prm;
    hw_sizes sz;
    int device;
    DevCtx host;          // host copy (device pointers filled in)
    DevCtx* dctx;         // device copy
    void* tables;         // one device block for all tables
    size_t tables_bytes;  // its size, and the FNV-1a hash of what was uploaded
    uint64_t tables_hash;
    u64* phase_scratch;   // decryption phases, chunk * r * N words
    size_t phase_chunk;
    LaunchInfo li;
    hw_geometry geom;     // resolved kernel geometry
    unsigned long long launches;
    std::vector<int32_t> ram_slot;
};

// ----------------------------------------------------------------- host math
static u64 hmul(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 hpow(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = hmul(r, b, q);
        b = hmul(b, b, q);
        e >>= 1;
    }
    return r;
}
static u64 hinv(u64 a, u64 q) { return hpow(a, q - 2, q); }

static bool miller_rabin(u64 n) {
    if (n < 2) return false;
    const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        s++;
    }
    for (u64 a : small) {
        u64 x = hpow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int k = 1; k < s && witness; k++) {
            x = hmul(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// A primitive 2N-th root of unity: the first odd x >= 3 whose power
// x^((q-1)/2N) squares to -1 after log_n doublings.  Any such root gives the
// same coefficient-domain results; it only fixes the evaluation order.
static u64 find_root(u64 q, int log_n) {
    const u64 n = (u64)1 << log_n;
    for (u64 x = 3; x < q; x += 2) {
        u64 w = hpow(x, (q - 1) / (2 * n), q);
        if (hpow(w, n, q) == q - 1) return w;
    }
    return 0;
}

static int brv(int x, int bits) {
    int y = 0;
    for (int b = 0; b < bits; b++) y |= ((x >> b) & 1) << (bits - 1 - b);
    return y;
}

static u64 shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// little-endian multi-limb helpers
static void lmul_small(u64* a, u64 m) {
    u128 carry = 0;
    for (int t = 0; t < HW_LIMBS; t++) {
        u128 v = (u128)a[t] * m + carry;
        a[t] = (u64)v;
        carry = v >> 64;
    }
}
static u64 lmod(const u64* a, u64 q) {
    u128 r = 0;
    for (int t = HW_LIMBS - 1; t >= 0; t--) r = ((r << 64) | a[t]) % q;
    return (u64)r;
}
static void lshr(const u64* a, int s, u64* out) {  // 0 < s < 64
    for (int t = 0; t < HW_LIMBS; t++) {
        u64 hi = t + 1 < HW_LIMBS ? a[t + 1] : 0;
        out[t] = (a[t] >> s) | (hi << (64 - s));
    }
}

static int ilog2_ceil(int l) {
    int L = 0;
    while ((1 << L) < l) L++;
    return L;
}

// ------------------------------------------------------------------ create
// Fills the defaults of a geometry and checks it against what is built.
static int resolve_geometry(const hw_params* p, const hw_geometry* g, hw_geometry* out) {
    hw_geometry G;
    memset(&G, 0, sizeof(G));
    if (g) G = *g;
    const int log_n = p->log_n;
    const bool small_q = p->prime_bits <= 30;
    if (G.ext_loge == 0) G.ext_loge = default_ext_loge(log_n);
    if (G.ext_np == 0) G.ext_np = default_ext_np(log_n);
    if (G.ntt_loge == 0) G.ntt_loge = 4;
    if (G.ntt_limbs == 0) G.ntt_limbs = small_q ? 1 : 2;
    if (G.ext_smem < 0 || G.ext_smem > 3) return fail(HW_EINVAL, "ext_smem must be 0, 1, 2 or 3");
    const ExtOps* ops = hw_ext_find(log_n, G.ext_loge, G.ext_np, G.ext_smem);
    if (!ops)
        return fail(HW_EINVAL,
                    "external-product geometry (loge %d, np %d, smem mode %d) is not built for log_n %d",
                    G.ext_loge, G.ext_np, G.ext_smem, log_n);
    if (ops->sm == 1) {
        const size_t rl_bytes = (size_t)2 * p->n_primes * ((size_t)1 << log_n) * sizeof(u64);
        if (ops->smem + rl_bytes > (size_t)227 * 1024)
            return fail(HW_EINVAL, "the evaluation form (%zu bytes) does not fit in shared memory beside "
                        "the exchange buffer (%zu bytes)", rl_bytes, ops->smem);
    }
    if (G.ext_blocks_per_sm < 0 || G.ext_blocks_per_sm > 32)
        return fail(HW_EINVAL, "ext_blocks_per_sm must be 0..32");
    if (G.ntt_loge != 3 && G.ntt_loge != 4) return fail(HW_EINVAL, "ntt_loge must be 3 or 4");
    if (G.ntt_limbs != 1 && G.ntt_limbs != 2) return fail(HW_EINVAL, "ntt_limbs must be 1 or 2");
    if (G.ntt_limbs == 1 && !small_q)
        return fail(HW_EINVAL, "32-bit transform arithmetic needs every prime below 2^30");
    if (G.l2_persist != 0 && G.l2_persist != 1) return fail(HW_EINVAL, "l2_persist must be 0 or 1");
    *out = G;
    return HW_OK;
}

extern "C" int hw_create(const hw_params* p, int cuda_device, hw_ctx** out) {
    return hw_create_tuned(p, nullptr, cuda_device, out);
}

extern "C" int hw_create_tuned(const hw_params* p, const hw_geometry* g, int cuda_device,
                               hw_ctx** out) {
    if (!p || !out) return fail(HW_EINVAL, "hw_create: null argument");
    *out = nullptr;
    if (p->log_n < 6 || p->log_n > 13) return fail(HW_EINVAL, "log_n must be in [6, 13]");
    if (p->n_primes < 1 || p->n_primes > 3) return fail(HW_EINVAL, "n_primes must be 1..3");
    if (p->prime_bits < 20 || p->prime_bits > 55) return fail(HW_EINVAL, "prime_bits must be 20..55");
    if (p->log_beta < 0 || p->log_beta > 30) return fail(HW_EINVAL, "log_beta must be 0..30");
    if (p->log_p < 1 || p->log_p > 30) return fail(HW_EINVAL, "log_p must be 1..30");
    if (p->n_classes < 2 || p->n_classes > 64) return fail(HW_EINVAL, "n_classes must be 2..64");
    if (p->n_values < 1 || p->therm_bits < 1 || p->therm_bits > 16)
        return fail(HW_EINVAL, "bad n_values / therm_bits");
    if (p->addr_bits < 1 || p->addr_bits > 20) return fail(HW_EINVAL, "addr_bits must be 1..20");
    if (p->hash_h3 && (p->tuple_bits < 1 || p->tuple_bits > 32))
        return fail(HW_EINVAL, "tuple_bits must be 1..32");
    if (p->act < 0 || p->act > 2) return fail(HW_EINVAL, "act must be HW_ACT_*");
    hw_geometry G;
    if (int rc = resolve_geometry(p, g, &G)) return rc;
    const int ext_loge = G.ext_loge;

    hw_ctx* c = new hw_ctx();
    memset(&c->host, 0, sizeof(DevCtx));
    c->prm = *p;
    c->device = cuda_device;
    c->launches = 0;
    DevCtx& H = c->host;
    hw_sizes& S = c->sz;
    memset(&S, 0, sizeof(S));

    const int log_n = p->log_n, n = 1 << log_n, r = p->n_primes;
    const int L = ilog2_ceil(p->n_classes);
    const int a = p->addr_bits;
    const int s = p->n_values * p->therm_bits;
    int k0, n_data;
    if (p->hash_h3) {
        k0 = (s + p->tuple_bits - 1) / p->tuple_bits;
        n_data = k0 * a;
    } else {
        k0 = (s + a - 1) / a;
        n_data = s;
    }
    int z = L + a - log_n;
    if (z < 0) z = 0;
    if (z > HW_MAX_Z) {
        delete c;
        return fail(HW_EINVAL, "tree depth z = %d exceeds %d", z, HW_MAX_Z);
    }
    if (z - L > 1) {
        delete c;
        return fail(HW_EINVAL, "more than one encrypted CMUX-tree level (z - L = %d)", z - L);
    }
    const int dpp = p->log_beta ? (p->prime_bits + p->log_beta - 1) / p->log_beta : 1;
    const int dnum = r * dpp;
    if (dnum > HW_MAX_DNUM) {
        delete c;
        return fail(HW_EINVAL, "too many gadget rows (%d)", dnum);
    }

    // primes: the r largest q < 2^bits with q = 1 mod 2N, descending
    std::vector<u64> q;
    {
        const u64 m = (u64)2 << log_n;
        u64 cand = (((u64)1 << p->prime_bits) - 2) / m * m + 1;
        while ((int)q.size() < r && cand > m) {
            if (miller_rabin(cand)) q.push_back(cand);
            cand -= m;
        }
        if ((int)q.size() < r) {
            delete c;
            return fail(HW_EINVAL, "not enough NTT-friendly primes");
        }
    }

    // tree: stored ciphertext indices V, slots and the pruned gate list
    std::vector<int> V;
    {
        std::vector<char> in(1 << z, 0);
        int xs = z > L ? 1 << (z - L) : 1;
        for (int cl = 0; cl < p->n_classes; cl++)
            for (int x = 0; x < xs; x++) in[(cl + (x << L)) % (1 << z)] = 1;
        for (int v = 0; v < (1 << z); v++) {
            H.slot_of[v] = -1;
            if (in[v]) {
                H.slot_of[v] = (int8_t)V.size();
                V.push_back(v);
            }
        }
        int ng = 0;
        for (int i = 0; i < z; i++)
            for (int j = 0; j < (1 << i); j++) {
                bool need = false;
                for (int v : V)
                    if (v % (1 << (i + 1)) == j + (1 << i)) need = true;
                if (need) {
                    H.gate_lvl[ng] = (int8_t)i;
                    H.gate_j[ng] = (int8_t)j;
                    ng++;
                }
            }
        H.n_gates = ng;
    }
    const int k1 = (int)V.size();

    H.log_n = log_n;
    H.n = n;
    H.r = r;
    H.dnum = dnum;
    H.dpp = dpp;
    H.log_beta = p->log_beta;
    H.L = L;
    H.a = a;
    H.k0 = k0;
    H.k1 = k1;
    H.z = z;
    H.n_data = n_data;
    H.n_slots = L + n_data;
    H.s = s;
    H.n_classes = p->n_classes;
    H.therm_bits = p->therm_bits;
    H.tuple_bits = p->tuple_bits;
    H.hash_h3 = p->hash_h3;
    H.n_values = p->n_values;
    H.log_p = p->log_p;
    H.act = p->act;
    H.act_arg = p->act_arg;
    H.rlwe_words = (size_t)2 * r * n;
    H.lwe_words = (size_t)r * (n + 1);
    H.rgsw_words = (size_t)2 * dnum * H.rlwe_words;
    H.sample_words = (size_t)H.n_slots * H.rgsw_words;
    H.model_words = (size_t)k0 * k1 * H.rlwe_words;

    // modulus Q, Delta = floor(Q/p), CRT constants
    u64 Q[HW_LIMBS] = {1, 0, 0, 0};
    for (int i = 0; i < r; i++) lmul_small(Q, q[i]);
    u64 delta[HW_LIMBS];
    lshr(Q, p->log_p, delta);
    lshr(Q, 1, H.halfQ);
    memcpy(H.Q, Q, sizeof(Q));
    for (int i = 0; i < r; i++) {
        PrimeConst& P = H.P[i];
        P.q = q[i];
        u64 inv = q[i];  // Newton iteration for q^-1 mod 2^64
        for (int it = 0; it < 6; it++) inv *= 2 - q[i] * inv;
        P.qneg = (u64)0 - inv;
        u64 t = ((u64)0 - q[i]) % q[i];  // 2^64 mod q
        P.r2 = hmul(t, t, q[i]);
        P.mu = ~(u64)0 / q[i];
        H.delta[i] = lmod(delta, q[i]);
        u64 Mi[HW_LIMBS] = {1, 0, 0, 0};
        for (int k = 0; k < r; k++)
            if (k != i) lmul_small(Mi, q[k]);
        memcpy(H.M[i], Mi, sizeof(Mi));
        u64 y = hinv(lmod(Mi, q[i]), q[i]);
        H.yM[i] = (u64)(((u128)y << 64) % q[i]);
        H.n_inv[i] = hinv((u64)n % q[i], q[i]);
        H.n_inv_s[i] = shoup(H.n_inv[i], q[i]);
        H.mr[i] = t;
        H.mr_s[i] = shoup(t, q[i]);
        H.mr2_s[i] = shoup(P.r2, q[i]);
        S.q[i] = q[i];
    }
    for (int rho = 0; rho < dnum; rho++) {
        int i = rho / dpp, k = rho % dpp;
        H.gconst[rho] = p->log_beta ? hpow((u64)1 << p->log_beta, (u64)k, q[i]) : 1;
    }

    // transform tables: interleaved (w, Shoup(w)) pairs, [prime][N]
    std::vector<u64> tw((size_t)4 * r * n);
    u64* tw_fwd = tw.data();
    u64* tw_inv = tw_fwd + (size_t)2 * r * n;
    for (int i = 0; i < r; i++) {
        u64 psi = find_root(q[i], log_n);
        if (!psi) {
            delete c;
            return fail(HW_EINVAL, "no 2N-th root of unity");
        }
        u64 psi_inv = hinv(psi, q[i]);
        // RGSW masks are drawn at the points psi_min^(2 brv(k) + 1), psi_min
        // the smallest primitive 2N-th root: psi_min = psi^u for the odd u
        // whose power is smallest, and position pos of this order (the point
        // psi^(2 brv(pos) + 1)) is sampling point u^-1 (2 brv(pos) + 1) mod 2N
        {
            const u64 two_n = 2 * (u64)n, step = hmul(psi, psi, q[i]);
            u64 x = psi, best = psi, u = 1;
            for (u64 e = 1; e < two_n; e += 2) {
                if (x < best) {
                    best = x;
                    u = e;
                }
                x = hmul(x, step, q[i]);
            }
            u64 uinv = 1;
            while ((u * uinv) % two_n != 1) uinv += 2;
            H.a_point_mul[i] = (uint32_t)uinv;
        }
        for (int k = 0; k < n; k++) {
            int e = brv(k, log_n);
            u64 w = hpow(psi, (u64)e, q[i]), wi = hpow(psi_inv, (u64)e, q[i]);
            size_t o = 2 * ((size_t)i * n + k);
            tw_fwd[o] = w;
            tw_fwd[o + 1] = shoup(w, q[i]);
            tw_inv[o] = wi;
            tw_inv[o + 1] = shoup(wi, q[i]);
        }
    }
    // rotation tables (Psi^(+-2^t) - 1 and inverses), interleaved with Shoup
    // companions; X^e evaluates to psi^((2 brv(pos) + 1) e) at position pos
    std::vector<u64> rot((size_t)2 * r * 2 * log_n * n), rinv((size_t)2 * r * 2 * log_n * n);
    {
        std::vector<u64> dv((size_t)2 * log_n * n), pre((size_t)2 * log_n * n);
        for (int i = 0; i < r; i++) {
            u64 psi = find_root(q[i], log_n), psi_inv = hinv(psi, q[i]);
            for (int pos = 0; pos < n; pos++) {
                u64 ev = 2 * (u64)brv(pos, log_n) + 1;
                for (int sg = 0; sg < 2; sg++) {
                    u64 x = hpow(sg ? psi_inv : psi, ev, q[i]);
                    for (int t = 0; t < log_n; t++) {
                        dv[((size_t)sg * log_n + t) * n + pos] = (x + q[i] - 1) % q[i];
                        x = hmul(x, x, q[i]);
                    }
                }
            }
            // batch inversion: one Fermat inverse for the whole table
            u64 run = 1;
            for (size_t k = 0; k < dv.size(); k++) {
                pre[k] = run;
                run = hmul(run, dv[k], q[i]);
            }
            u64 inv = hinv(run, q[i]);
            for (size_t k = dv.size(); k-- > 0;) {
                u64 dk = hmul(inv, pre[k], q[i]);
                inv = hmul(inv, dv[k], q[i]);
                // thread-major: position pos of a row sits at eval_addr(pos)
                const size_t row = k / n;
                const int pos = (int)(k % n);
                size_t o = 2 * ((size_t)i * 2 * log_n * n + row * n + eval_addr(pos, log_n, ext_loge));
                rot[o] = dv[k];
                rot[o + 1] = shoup(dv[k], q[i]);
                rinv[o] = dk;
                rinv[o + 1] = shoup(dk, q[i]);
            }
        }
    }
    H.diag = p->log_beta == 0 ? 1 : 0;

    // 32-bit transform tables when every prime is below 2^30
    const bool small_q = p->prime_bits <= 30;
    std::vector<uint32_t> tw32(small_q ? (size_t)4 * r * n : 1, 0);
    if (small_q)
        for (int i = 0; i < r; i++) {
            const uint32_t qi = (uint32_t)q[i];
            for (int k = 0; k < n; k++) {
                const u64* f = &tw[2 * ((size_t)i * n + k)];
                const u64* b = &tw[(size_t)2 * r * n + 2 * ((size_t)i * n + k)];
                size_t o = 2 * ((size_t)i * n + k);
                tw32[o] = (uint32_t)f[0];
                tw32[o + 1] = (uint32_t)((f[0] << 32) / qi);
                tw32[(size_t)2 * r * n + o] = (uint32_t)b[0];
                tw32[(size_t)2 * r * n + o + 1] = (uint32_t)((b[0] << 32) / qi);
            }
            u64 ni = hinv((u64)n % q[i], q[i]);
            H.n_inv32[i] = (uint32_t)ni;
            H.n_inv32_s[i] = (uint32_t)((ni << 32) / qi);
        }

    // 32-bit external product: 30-bit primes, several digits per prime, a
    // MAC sum of 2 dnum products (q - 1)^2 that fits 64 bits, and a ring the
    // 32-bit path is compiled for (N <= 2048)
    H.ext32 = 0;
    if (small_q && !H.diag && log_n <= 11) {
        unsigned __int128 bound = 0;
        for (int i = 0; i < r; i++) {
            const unsigned __int128 m = (unsigned __int128)(q[i] - 1) * (q[i] - 1) * (2 * (u64)dnum);
            if (m > bound) bound = m;
        }
        H.ext32 = bound < ((unsigned __int128)1 << 64) ? 1 : 0;
    }

    // digits must lift without reduction: |d| <= (q_i - 1)/2 < q_j
    for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++)
            if ((q[i] - 1) / 2 >= q[j]) {
                delete c;
                return fail(HW_EINVAL, "primes too far apart for the RNS gadget");
            }

    // pi_r (Fisher-Yates from the top with the PERM stream), H3 rows, RAM slots
    std::vector<int32_t> perm(s);
    for (int k = 0; k < s; k++) perm[k] = k;
    for (int j = s - 1; j >= 1; j--) {
        Philox4 w = hw_draw(p->model_seed, HW_TAG_PERM, (u64)j >> 2, 0, 0);
        int k = (int)(w.v[j & 3] % (u64)(j + 1));
        std::swap(perm[j], perm[k]);
    }
    std::vector<u64> h3(p->hash_h3 ? p->tuple_bits : 1, 0);
    if (p->hash_h3)
        for (int i = 0; i < p->tuple_bits; i++) {
            Philox4 w = hw_draw(p->model_seed, HW_TAG_H3, (u64)i >> 2, 0, 0);
            h3[i] = w.v[i & 3] & (((u64)1 << a) - 1);
        }
    c->ram_slot.assign((size_t)k0 * a, -1);
    for (int j = 0; j < k0; j++)
        for (int i = 0; i < a; i++) {
            if (p->hash_h3)
                c->ram_slot[(size_t)j * a + i] = L + j * a + i;
            else if (j * a + i < s)
                c->ram_slot[(size_t)j * a + i] = L + perm[j * a + i];
        }

    // upload
    size_t bytes_tw = tw.size() * 8, bytes_rs = c->ram_slot.size() * 4, bytes_perm = perm.size() * 4,
           bytes_h3 = h3.size() * 8, bytes_rot = rot.size() * 8, bytes_tw32 = tw32.size() * 4;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t total = al(bytes_tw) + al(bytes_rs) + al(bytes_perm) + al(bytes_h3) + 2 * al(bytes_rot) +
                   al(bytes_tw32) + al(sizeof(DevCtx));
    c->phase_chunk = 64;
    c->tables = nullptr;
    c->phase_scratch = nullptr;
    int n_alloc = 0;
    cudaError_t e = cudaSetDevice(cuda_device);
    if (e == cudaSuccess) e = ctx_malloc(&c->tables, total, &n_alloc);
    if (e == cudaSuccess)
        e = ctx_malloc((void**)&c->phase_scratch, c->phase_chunk * (size_t)r * n * sizeof(u64), &n_alloc);
    if (e != cudaSuccess) {
        if (c->tables) cudaFree(c->tables);
        delete c;
        return fail(HW_ECUDA, "device allocation failed: %s", cudaGetErrorString(e));
    }
    char* base = (char*)c->tables;
    size_t off = 0;
    cudaMemset(base, 0, total);  // padding between tables hashes as zeros
    auto put = [&](const void* src, size_t nb) {
        char* d = base + off;
        cudaMemcpy(d, src, nb, cudaMemcpyHostToDevice);
        off += al(nb);
        return d;
    };
    char* d_tw = put(tw.data(), bytes_tw);
    H.tw_fwd = (const ulonglong2*)d_tw;
    H.tw_inv = H.tw_fwd + (size_t)r * n;
    H.ram_slot = (const int32_t*)put(c->ram_slot.data(), bytes_rs);
    H.perm = (const int32_t*)put(perm.data(), bytes_perm);
    H.h3 = (const u64*)put(h3.data(), bytes_h3);
    H.rot_tab = (const ulonglong2*)put(rot.data(), bytes_rot);
    H.rot_inv = (const ulonglong2*)put(rinv.data(), bytes_rot);
    {
        const uint2* t32 = (const uint2*)put(tw32.data(), bytes_tw32);
        H.tw32_fwd = small_q ? t32 : nullptr;
        H.tw32_inv = small_q ? t32 + (size_t)r * n : nullptr;
    }
    H.ext_loge = G.ext_loge;
    H.ext_np = G.ext_np;
    c->dctx = (DevCtx*)put(&H, sizeof(DevCtx));
    c->tables_bytes = total;
    c->tables_hash = 0;
    {
        std::vector<unsigned char> img(total);
        if (cudaMemcpy(img.data(), base, total, cudaMemcpyDeviceToHost) == cudaSuccess)
            c->tables_hash = fnv1a(img.data(), total);
    }
    LaunchInfo& li = c->li;
    li.log_n = log_n;
    li.ext = hw_ext_find(log_n, G.ext_loge, G.ext_np, G.ext_smem);
    li.ext_smem = li.ext->smem + (li.ext->sm == 1 ? (size_t)H.rlwe_words * sizeof(u64) : 0);
    li.ntt_loge = G.ntt_loge;
    li.ntt_limbs = G.ntt_limbs;
    e = hw_kernels_init(li);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(c->tables);
        cudaFree(c->phase_scratch);
        delete c;
        return fail(HW_ECUDA, "context upload failed: %s", cudaGetErrorString(e));
    }

    // sizes
    S.n = n;
    S.r = r;
    S.L = L;
    S.a = a;
    S.s = s;
    S.k0 = k0;
    S.k1 = k1;
    S.z = z;
    S.dpp = dpp;
    S.dnum = dnum;
    S.n_data = n_data;
    S.n_slots = H.n_slots;
    S.rlwe_words = H.rlwe_words;
    S.lwe_words = H.lwe_words;
    S.rgsw_words = H.rgsw_words;
    S.key_words = (size_t)2 * r * n;
    S.model_words = H.model_words;
    S.sample_words = H.sample_words;
    S.resp_words = (size_t)p->n_classes * k0 * H.lwe_words;
    S.sums_words = (size_t)p->n_classes * H.lwe_words;
    S.word_bits = H.ext32 ? 32 : 64;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device);
    li.dctx = c->dctx;
    li.log_n = log_n;
    li.n = n;
    li.r = r;
    li.k0 = k0;
    li.k1 = k1;
    li.n_classes = p->n_classes;
    li.n_data = n_data;
    li.n_slots = H.n_slots;
    li.L = L;
    li.dnum = dnum;
    li.z = z;
    li.rlwe_words = H.rlwe_words;
    li.lwe_words = H.lwe_words;
    li.rgsw_words = H.rgsw_words;
    li.sample_words = H.sample_words;
    li.model_words = H.model_words;
    li.sm_count = sms;
    li.small_q = p->prime_bits <= 30 ? 1 : 0;
    li.ext32 = H.ext32;
    li.launches = &c->launches;
    {
        int occ = li.ext->occupancy(li.ext_smem);
        if (G.ext_blocks_per_sm > 0 && G.ext_blocks_per_sm < occ) occ = G.ext_blocks_per_sm;
        G.ext_blocks_per_sm = occ;
        li.ext_grid = occ * sms;
    }
    li.l2_persist = 0;
    li.l2_window_max = 0;
    if (G.l2_persist) {
        // persisting set-aside of this process's context, sized to the
        // inference kernel's accumulators (two RLWEs and their evaluation
        // forms per resident block) and capped by the device; it ends with
        // the context
        int max_persist = 0, max_window = 0;
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, cuda_device);
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, cuda_device);
        size_t want = (size_t)li.ext_grid * li.ext->scratch_rlwe * H.rlwe_words * sizeof(u64);
        if (want > (size_t)max_persist) want = (size_t)max_persist;
        size_t cur = 0;
        cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
        if (want > cur && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess) {
            cudaGetLastError();
            want = cur;
        }
        if (want > 0 && max_window > 0) {
            li.l2_persist = want;
            li.l2_window_max = (size_t)max_window;
        } else {
            G.l2_persist = 0;  // not available here: report it off
        }
    }
    c->geom = G;
    *out = c;
    return HW_OK;
}

extern "C" int hw_get_geometry(const hw_ctx* c, hw_geometry* out) {
    if (!c || !out) return fail(HW_EINVAL, "hw_get_geometry: null argument");
    *out = c->geom;
    return HW_OK;
}

extern "C" int hw_list_geometries(const hw_params* p, hw_geometry* out, size_t max, size_t* count) {
    if (!p || !count) return fail(HW_EINVAL, "hw_list_geometries: null argument");
    if (p->log_n < 6 || p->log_n > 13) return fail(HW_EINVAL, "log_n must be in [6, 13]");
    int nt = 0;
    const ExtOps* t = hw_ext_table(p->log_n, &nt);
    const int d_loge = default_ext_loge(p->log_n), d_np = default_ext_np(p->log_n);
    size_t k = 0;
    auto emit = [&](int loge, int np, int sm) {
        if (out && k < max) {
            memset(&out[k], 0, sizeof(hw_geometry));
            out[k].ext_loge = loge;
            out[k].ext_np = np;
            out[k].ext_smem = sm;
        }
        k++;
    };
    emit(d_loge, d_np, 0);
    for (int i = 0; i < nt; i++)
        if (!(t[i].loge == d_loge && t[i].np == d_np && t[i].sm == 0)) emit(t[i].loge, t[i].np, t[i].sm);
    *count = k;
    return HW_OK;
}

extern "C" int hw_destroy(hw_ctx* c) {
    if (!c) return HW_OK;
    cudaSetDevice(c->device);
    cudaFree(c->tables);
    cudaFree(c->phase_scratch);
    delete c;
    return HW_OK;
}

extern "C" int hw_check_context(const hw_ctx* c) {
    if (!c) return fail(HW_EINVAL, "hw_check_context: null context");
    cudaSetDevice(c->device);
    std::vector<unsigned char> img(c->tables_bytes);
    cudaError_t e = cudaMemcpy(img.data(), c->tables, c->tables_bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(HW_ECUDA, "hw_check_context: copy failed: %s", cudaGetErrorString(e));
    if (fnv1a(img.data(), img.size()) != c->tables_hash)
        return fail(HW_EMISMATCH, "hw_check_context: the context's device tables changed since creation");
    const unsigned to = ntt_wait_timeouts();
    if (to == ~0u) return fail(HW_ECUDA, "hw_check_context: the transform's wait counter cannot be read");
    if (to) return fail(HW_ETIMEOUT, "hw_check_context: %u bulk-copy waits of the batched transform ran out", to);
    return HW_OK;
}

extern "C" int hw_get_sizes(const hw_ctx* c, hw_sizes* out) {
    if (!c || !out) return fail(HW_EINVAL, "hw_get_sizes: null argument");
    *out = c->sz;
    return HW_OK;
}

extern "C" int hw_get_ram_slots(const hw_ctx* c, int32_t* dst, size_t n) {
    if (!c || !dst) return fail(HW_EINVAL, "hw_get_ram_slots: null argument");
    if (n < c->ram_slot.size()) return fail(HW_ENOMEM, "hw_get_ram_slots: need %zu entries", c->ram_slot.size());
    memcpy(dst, c->ram_slot.data(), c->ram_slot.size() * sizeof(int32_t));
    return HW_OK;
}

extern "C" uint64_t hw_launch_count(const hw_ctx* c) { return c ? c->launches : 0; }

// Accessors for entry points defined in other translation units.
const LaunchInfo* hw_ctx_launch_info(const hw_ctx* c) { return &c->li; }
int hw_ctx_device(const hw_ctx* c) { return c->device; }
int hw_ctx_fail(int code, const char* msg) { return fail(code, "%s", msg); }

extern "C" const char* hw_last_error(void) { return g_last_error.c_str(); }

// Persistent-grid scratch per block: two accumulators and, unless it lives in
// shared memory, one evaluation-form buffer (inference), plus the k1 tree
// slots and their evaluation forms (training; the items add their slots into
// the model themselves, so nothing grows with the batch).
extern "C" size_t hw_train_scratch_words(const hw_ctx* c, size_t n) {
    if (!c) return 0;
    (void)n;
    return (size_t)c->li.ext_grid * (c->li.ext->scratch_rlwe + 2 * (size_t)c->sz.k1) * c->sz.rlwe_words;
}

// Training samples per IVP launch: the model's words grow by < q_i per
// sample between reductions and must stay below 2^64.
static size_t train_chunk(const hw_ctx* c) {
    u64 qmax = 0;
    for (int i = 0; i < c->sz.r; i++) qmax = c->sz.q[i] > qmax ? c->sz.q[i] : qmax;
    const u64 lim = (~(u64)0) / qmax - 1;  // (lim + 1) q <= 2^64 - 1
    const size_t per_launch = (size_t)0x7fffffff / (size_t)c->sz.k0;  // items fit an int
    return lim < per_launch ? (size_t)lim : per_launch;
}

// Inference scratch: the persistent blocks' accumulators, then (batches of
// two or more samples) the first CMUX's digit transforms shared by the batch.
static size_t infer_block_words(const hw_ctx* c) {
    return (size_t)c->li.ext_grid * c->li.ext->scratch_rlwe * c->sz.rlwe_words;
}

static size_t infer_digit_words(const hw_ctx* c, size_t n) { return n >= 2 ? vp_digits_words(c->li) : 0; }

extern "C" size_t hw_infer_scratch_words(const hw_ctx* c, size_t n) {
    if (!c) return 0;
    return infer_block_words(c) + infer_digit_words(c, n);
}

#define CHECK_CTX(c)                                                   \
    do {                                                               \
        if (!(c)) return fail(HW_EINVAL, "%s: null context", __func__); \
        cudaSetDevice((c)->device);                                    \
    } while (0)

extern "C" int hw_keygen(hw_ctx* c, uint64_t seed, uint64_t* key, void* stream) {
    CHECK_CTX(c);
    if (!key) return fail(HW_EINVAL, "hw_keygen: null key buffer");
    CUDA_TRY(launch_keygen(c->li, seed, key, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_encode(hw_ctx* c, const uint8_t* values, size_t n, uint8_t* bits, void* stream) {
    CHECK_CTX(c);
    if (n && (!values || !bits)) return fail(HW_EINVAL, "hw_encode: null buffer");
    CUDA_TRY(launch_encode(c->li, values, n, bits, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_encrypt_sample(hw_ctx* c, const uint64_t* key, const uint8_t* bits,
                                 const uint32_t* labels, size_t n, uint64_t seed, uint64_t first,
                                 uint64_t* rgsw, void* stream) {
    CHECK_CTX(c);
    if (n && (!key || !bits || !rgsw)) return fail(HW_EINVAL, "hw_encrypt_sample: null buffer");
    CUDA_TRY(launch_encrypt(c->li, key, bits, labels, n, seed, first, rgsw, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_train_accumulate(hw_ctx* c, uint64_t* model, const uint64_t* rgsw, size_t n,
                                   uint64_t* scratch, size_t scratch_words, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!model || !rgsw || !scratch) return fail(HW_EINVAL, "hw_train_accumulate: null buffer");
    size_t need = hw_train_scratch_words(c, n);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_train_accumulate: scratch has %zu words, needs %zu", scratch_words, need);
    const int grid = c->li.ext_grid;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t chunk = train_chunk(c);
    for (size_t s0 = 0; s0 < n; s0 += chunk) {
        const size_t m = n - s0 < chunk ? n - s0 : chunk;
        CUDA_TRY(launch_ivp_train(c->li, rgsw + s0 * c->sz.sample_words, m, model, scratch, grid, st));
        CUDA_TRY(launch_model_reduce(c->li, model, st));
    }
    return HW_OK;
}

extern "C" int hw_infer(hw_ctx* c, const uint64_t* model, const uint64_t* rgsw, size_t n,
                        uint64_t* resp, uint64_t* sums, uint64_t* scratch, size_t scratch_words,
                        void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!model || !rgsw || !resp || !sums || !scratch) return fail(HW_EINVAL, "hw_infer: null buffer");
    size_t need = hw_infer_scratch_words(c, n);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_infer: scratch has %zu words, needs %zu", scratch_words, need);
    int grid = c->li.ext_grid;
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* digits = infer_digit_words(c, n) ? scratch + infer_block_words(c) : nullptr;
    CUDA_TRY(launch_vp_infer(c->li, model, rgsw, n, resp, scratch, grid, st, 0, digits));
    CUDA_TRY(launch_class_sums(c->li, resp, n, sums, st));
    return HW_OK;
}

extern "C" int hw_infer_packed(hw_ctx* c, const uint64_t* model, const uint64_t* rgsw, size_t n,
                               uint64_t* resp, uint64_t* sums, uint64_t* scratch, size_t scratch_words,
                               void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!model || !rgsw || !resp || !sums || !scratch)
        return fail(HW_EINVAL, "hw_infer_packed: null buffer");
    size_t need = hw_infer_scratch_words(c, n);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_infer_packed: scratch has %zu words, needs %zu", scratch_words, need);
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* digits = infer_digit_words(c, n) ? scratch + infer_block_words(c) : nullptr;
    CUDA_TRY(launch_vp_infer(c->li, model, rgsw, n, resp, scratch, c->li.ext_grid, st, 1, digits));
    CUDA_TRY(launch_class_sums(c->li, resp, n, sums, st));
    return HW_OK;
}

extern "C" size_t hw_plain_model_words(const hw_ctx* c) { return c ? hw_plain_words_li(c->li) : 0; }

extern "C" int hw_plain_model_load(hw_ctx* c, const int64_t* counts, uint64_t* plain, void* stream) {
    CHECK_CTX(c);
    if (!counts || !plain) return fail(HW_EINVAL, "hw_plain_model_load: null buffer");
    CUDA_TRY(launch_plain_load(c->li, counts, plain, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_infer_plain(hw_ctx* c, const uint64_t* plain, const uint64_t* rgsw, size_t n, uint64_t* resp,
                              uint64_t* sums, uint64_t* scratch, size_t scratch_words, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!plain || !rgsw || !resp || !sums || !scratch) return fail(HW_EINVAL, "hw_infer_plain: null buffer");
    size_t need = infer_block_words(c);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_infer_plain: scratch has %zu words, needs %zu", scratch_words, need);
    if (n * (size_t)c->sz.k0 > 0x7fffffff) return fail(HW_EINVAL, "hw_infer_plain: batch too large");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(launch_vp_plain(c->li, plain, rgsw, n, resp, scratch, c->li.ext_grid, st));
    CUDA_TRY(launch_class_sums(c->li, resp, n, sums, st));
    return HW_OK;
}

extern "C" int hw_decrypt(hw_ctx* c, const uint64_t* key, int what, const uint64_t* obj,
                          size_t count, int64_t* out, void* stream) {
    CHECK_CTX(c);
    if (count == 0) return HW_OK;
    if (!key || !obj || !out) return fail(HW_EINVAL, "hw_decrypt: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    if (what == HW_DEC_RLWE) {
        CUDA_TRY(launch_decrypt_rlwe(c->li, key, obj, count, out, c->phase_scratch, c->phase_chunk, st));
    } else if (what == HW_DEC_LWE) {
        CUDA_TRY(launch_decrypt_lwe(c->li, key, obj, count, out, st));
    } else if (what == HW_DEC_MODEL) {
        if (count != 1) return fail(HW_EINVAL, "hw_decrypt: HW_DEC_MODEL decrypts one model (count = 1)");
        CUDA_TRY(launch_decrypt_model(c->li, key, obj, c->sz.a, out, c->phase_scratch, c->phase_chunk, st));
    } else {
        return fail(HW_EINVAL, "hw_decrypt: unknown object kind %d", what);
    }
    return HW_OK;
}

extern "C" int hw_pdact(hw_ctx* c, const int64_t* counts, size_t n, int64_t* scores, int32_t* labels,
                        void* stream) {
    CHECK_CTX(c);
    if (n && (!counts || !scores || !labels)) return fail(HW_EINVAL, "hw_pdact: null buffer");
    CUDA_TRY(launch_pdact(c->li, counts, n, scores, labels, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" size_t hw_count_scratch_words(const hw_ctx* c, size_t n) {
    if (!c) return 0;
    return n * c->sz.rlwe_words + (size_t)c->li.ext_grid * c->li.ext->scratch_rlwe * c->sz.rlwe_words;
}

extern "C" int hw_count_classes(hw_ctx* c, uint64_t* counts, const uint64_t* rgsw, size_t n, uint64_t* scratch,
                                size_t scratch_words, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!counts || !rgsw || !scratch) return fail(HW_EINVAL, "hw_count_classes: null buffer");
    const size_t need = hw_count_scratch_words(c, n);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_count_classes: scratch needs %zu words, got %zu", need, scratch_words);
    if (n > 0x7fffffff) return fail(HW_EINVAL, "hw_count_classes: batch too large");
    u64* out = scratch;
    u64* acc = scratch + n * c->sz.rlwe_words;
    CUDA_TRY(launch_count_classes(c->li, counts, rgsw, n, out, acc, c->li.ext_grid, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_pdact_balanced(hw_ctx* c, const int64_t* counts, const int64_t* class_counts, size_t n,
                                 int64_t* scores, int32_t* labels, void* stream) {
    CHECK_CTX(c);
    if (n && (!counts || !class_counts || !scores || !labels))
        return fail(HW_EINVAL, "hw_pdact_balanced: null buffer");
    CUDA_TRY(launch_pdact_balanced(c->li, counts, class_counts, n, scores, labels, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" size_t hw_ksk_words(const hw_ctx* c) {
    return c ? (size_t)c->sz.n * c->sz.dnum * c->sz.rlwe_words : 0;
}

extern "C" int hw_ksk_gen(hw_ctx* c, const uint64_t* key, uint64_t seed, uint64_t* ksk, void* stream) {
    CHECK_CTX(c);
    if (!key || !ksk) return fail(HW_EINVAL, "hw_ksk_gen: null buffer");
    CUDA_TRY(launch_ksk_gen(c->li, key, seed, ksk, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" size_t hw_pack_scratch_words(const hw_ctx* c, size_t n) {
    return c ? hw_pack_scratch_words_li(c->li, n) : 0;
}

extern "C" int hw_pack_responses(hw_ctx* c, const uint64_t* ksk, const uint64_t* resp, size_t n,
                                 uint64_t* packed, uint64_t* scratch, size_t scratch_words, void* stream) {
    CHECK_CTX(c);
    if (n == 0) return HW_OK;
    if (!ksk || !resp || !packed || !scratch) return fail(HW_EINVAL, "hw_pack_responses: null buffer");
    if ((size_t)c->sz.k0 * c->prm.n_classes > (size_t)c->sz.n)
        return fail(HW_EINVAL, "hw_pack_responses: %d responses per sample exceed N = %d",
                    c->sz.k0 * c->prm.n_classes, c->sz.n);
    const size_t need = hw_pack_scratch_words_li(c->li, 1);
    if (scratch_words < need)
        return fail(HW_ENOMEM, "hw_pack_responses: scratch needs at least %zu words, got %zu", need, scratch_words);
    CUDA_TRY(launch_pack(c->li, ksk, resp, n, packed, scratch, scratch_words, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_export_rgsw(hw_ctx* c, const uint64_t* rgsw, size_t count, uint64_t* out,
                              void* stream) {
    CHECK_CTX(c);
    if (count && (!rgsw || !out)) return fail(HW_EINVAL, "hw_export_rgsw: null buffer");
    if (rgsw == out) return fail(HW_EINVAL, "hw_export_rgsw: output must not alias input");
    CUDA_TRY(launch_export_rgsw(c->li, rgsw, count, out, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_import_rgsw(hw_ctx* c, const uint64_t* canonical, size_t count, uint64_t* rgsw,
                              void* stream) {
    CHECK_CTX(c);
    if (count && (!canonical || !rgsw)) return fail(HW_EINVAL, "hw_import_rgsw: null buffer");
    CUDA_TRY(launch_import_rgsw(c->li, canonical, count, rgsw, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_ntt_forward(hw_ctx* c, uint64_t* poly, size_t count, void* stream) {
    CHECK_CTX(c);
    if (count && !poly) return fail(HW_EINVAL, "hw_ntt_forward: null buffer");
    CUDA_TRY(launch_ntt_batch(c->li, poly, count, 0, (cudaStream_t)stream));
    return HW_OK;
}

extern "C" int hw_ntt_inverse(hw_ctx* c, uint64_t* poly, size_t count, void* stream) {
    CHECK_CTX(c);
    if (count && !poly) return fail(HW_EINVAL, "hw_ntt_inverse: null buffer");
    CUDA_TRY(launch_ntt_batch(c->li, poly, count, 1, (cudaStream_t)stream));
    return HW_OK;
}

// ------------------------------------------------------------------ model
// Definition 2's model H as a caller buffer: creation (H <- {0}), and the
// canonical words with a header naming the parameter set, for saving a
// model and resuming training elsewhere (the model is additive,
// Section 3.6.2).

static void digest_word(uint64_t* h, uint64_t v) {
    for (int b = 0; b < 8; b++) {
        *h ^= (v >> (8 * b)) & 0xff;
        *h *= 0x100000001b3ULL;
    }
}

extern "C" int hw_params_digest(const hw_params* p, uint64_t* out) {
    if (!p || !out) return fail(HW_EINVAL, "hw_params_digest: null argument");
    uint64_t h = 0xcbf29ce484222325ULL;
    const int32_t f[] = {p->log_n,     p->n_primes,   p->prime_bits, p->log_beta, p->log_p,
                         p->n_classes, p->n_values,   p->therm_bits, p->tuple_bits, p->addr_bits,
                         p->hash_h3,   p->act,        p->act_arg};
    for (int32_t v : f) digest_word(&h, (uint64_t)(int64_t)v);
    digest_word(&h, p->model_seed);
    *out = h;
    return HW_OK;
}

extern "C" size_t hw_model_words(const hw_ctx* c) { return c ? c->sz.model_words : 0; }

extern "C" int hw_model_zero(hw_ctx* c, uint64_t* model, void* stream) {
    CHECK_CTX(c);
    if (!model) return fail(HW_EINVAL, "hw_model_zero: null buffer");
    CUDA_TRY(cudaMemsetAsync(model, 0, c->sz.model_words * sizeof(u64), (cudaStream_t)stream));
    return HW_OK;
}

extern "C" size_t hw_model_export_words(const hw_ctx* c) {
    return c ? HW_MODEL_HEADER_WORDS + c->sz.model_words : 0;
}

extern "C" int hw_model_header_check(const hw_params* p, const uint64_t* in, size_t n_words,
                                     uint64_t* samples) {
    if (!p || !in) return fail(HW_EINVAL, "hw_model_header_check: null argument");
    if (n_words < HW_MODEL_HEADER_WORDS || in[0] != HW_MODEL_MAGIC)
        return fail(HW_EINVAL, "hw_model_header_check: not an exported model");
    if (in[1] != HW_MODEL_VERSION)
        return fail(HW_EINVAL, "hw_model_header_check: format version %llu, this library reads %d",
                    (unsigned long long)in[1], HW_MODEL_VERSION);
    uint64_t d = 0;
    hw_params_digest(p, &d);
    if (in[2] != d) return fail(HW_EMISMATCH, "hw_model_header_check: model made for another parameter set");
    if (in[8] != (uint64_t)(n_words - HW_MODEL_HEADER_WORDS))
        return fail(HW_EINVAL, "hw_model_header_check: %zu model words follow the header, it announces %llu",
                    n_words - HW_MODEL_HEADER_WORDS, (unsigned long long)in[8]);
    if (samples) *samples = in[3];
    return HW_OK;
}

extern "C" int hw_model_export(hw_ctx* c, const uint64_t* model, uint64_t samples, uint64_t* out,
                               size_t n_words, void* stream) {
    CHECK_CTX(c);
    if (!model || !out) return fail(HW_EINVAL, "hw_model_export: null buffer");
    const size_t need = HW_MODEL_HEADER_WORDS + c->sz.model_words;
    if (n_words < need) return fail(HW_ENOMEM, "hw_model_export: needs %zu words, got %zu", need, n_words);
    uint64_t d = 0;
    hw_params_digest(&c->prm, &d);
    const uint64_t head[HW_MODEL_HEADER_WORDS] = {HW_MODEL_MAGIC, HW_MODEL_VERSION, d, samples,
                                                  (uint64_t)c->sz.k0, (uint64_t)c->sz.k1, (uint64_t)c->sz.r,
                                                  (uint64_t)c->sz.n, (uint64_t)c->sz.model_words};
    memcpy(out, head, sizeof(head));
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(out + HW_MODEL_HEADER_WORDS, model, c->sz.model_words * sizeof(u64),
                             cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return HW_OK;
}

extern "C" int hw_model_import(hw_ctx* c, const uint64_t* in, size_t n_words, uint64_t* model,
                               uint64_t* samples, void* stream) {
    CHECK_CTX(c);
    if (!in || !model) return fail(HW_EINVAL, "hw_model_import: null buffer");
    uint64_t smp = 0;
    int rc = hw_model_header_check(&c->prm, in, n_words, &smp);
    if (rc != HW_OK) return rc;
    if (in[4] != (uint64_t)c->sz.k0 || in[5] != (uint64_t)c->sz.k1 || in[6] != (uint64_t)c->sz.r ||
        in[7] != (uint64_t)c->sz.n || in[8] != (uint64_t)c->sz.model_words)
        return fail(HW_EMISMATCH, "hw_model_import: model shape differs from this context's");
    // every word is a residue of its prime: [RAM][slot][component][prime][N]
    const u64* w = in + HW_MODEL_HEADER_WORDS;
    const size_t n = (size_t)c->sz.n, r = (size_t)c->sz.r;
    for (size_t i = 0; i < c->sz.model_words; i++)
        if (w[i] >= c->sz.q[(i / n) % r])
            return fail(HW_EINVAL, "hw_model_import: word %zu is not reduced mod its prime", i);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(model, w, c->sz.model_words * sizeof(u64), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (samples) *samples = smp;
    return HW_OK;
}
