// tune.cu -- hw_autotune: measures the built kernel geometries of a
// parameter set on a probe step and picks the fastest.  Host code over the
// public entry points; the probe inputs are synthetic and every geometry
// computes the same results, so only time differs.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "../../include/hwisard.h"

int hw_ctx_fail(int code, const char* msg);

namespace {

struct DevBuf {
    void* p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 8) == cudaSuccess; }
    template <typename T>
    T* as() const {
        return (T*)p;
    }
};

struct Events {
    cudaEvent_t ev[4];
    Events() {
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~Events() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
    double ms(int a, int b) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
};

const double kUnset = -1.0;

void entry_init(hw_tune_entry* e, const hw_geometry& g) {
    memset(e, 0, sizeof(*e));
    e->geometry = g;
    e->ms_encrypt = e->ms_train = e->ms_infer = e->ms_ntt = kUnset;
}

double keep_min(double best, double t) { return best < 0 || t < best ? t : best; }

// One step of n training and n test samples: encrypt both, train, infer.
int probe_step(const hw_params* p, const hw_geometry& g, int dev, size_t n, int reps,
               cudaStream_t st, hw_tune_entry* out) {
    entry_init(out, g);
    hw_ctx* c = nullptr;
    int rc = hw_create_tuned(p, &g, dev, &c);
    if (rc != HW_OK) return out->status = rc;
    hw_get_geometry(c, &out->geometry);
    hw_sizes S;
    hw_get_sizes(c, &S);
    const size_t w_tr = hw_train_scratch_words(c, n), w_inf = hw_infer_scratch_words(c, n);
    const size_t bytes = 8 * (S.key_words + 2 * n * S.sample_words + S.model_words + w_tr + w_inf +
                              n * (S.resp_words + S.sums_words)) +
                         n * ((size_t)S.n_data + 4);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if (bytes + ((size_t)1 << 30) > free_b) {
        hw_destroy(c);
        return out->status = HW_ENOMEM;
    }
    DevBuf key, bits, labels, rg_tr, rg_te, model, scr_tr, scr_inf, resp, sums;
    bool ok = key.alloc(8 * S.key_words) && bits.alloc(n * S.n_data) && labels.alloc(4 * n) &&
              rg_tr.alloc(8 * n * S.sample_words) && rg_te.alloc(8 * n * S.sample_words) &&
              model.alloc(8 * S.model_words) && scr_tr.alloc(8 * w_tr) && scr_inf.alloc(8 * w_inf) &&
              resp.alloc(8 * n * S.resp_words) && sums.alloc(8 * n * S.sums_words);
    if (!ok) {
        hw_destroy(c);
        return out->status = HW_ENOMEM;
    }
    // synthetic bits (a fixed xorshift pattern) and labels i mod l
    std::vector<uint8_t> hb(n * S.n_data);
    uint64_t x = 0x9E3779B97F4A7C15ULL;
    for (auto& b : hb) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        b = (uint8_t)(x & 1);
    }
    std::vector<uint32_t> hl(n);
    for (size_t i = 0; i < n; i++) hl[i] = (uint32_t)(i % (size_t)p->n_classes);
    cudaMemcpy(bits.p, hb.data(), hb.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(labels.p, hl.data(), 4 * n, cudaMemcpyHostToDevice);
    cudaMemsetAsync(model.p, 0, 8 * S.model_words, st);
    rc = hw_keygen(c, 1, key.as<uint64_t>(), st);
    Events E;
    for (int it = 0; it <= reps && rc == HW_OK; it++) {  // iteration 0 warms up
        cudaEventRecord(E.ev[0], st);
        rc = hw_encrypt_sample(c, key.as<uint64_t>(), bits.as<uint8_t>(), labels.as<uint32_t>(), n, 7, 0,
                               rg_tr.as<uint64_t>(), st);
        if (rc == HW_OK)
            rc = hw_encrypt_sample(c, key.as<uint64_t>(), bits.as<uint8_t>(), nullptr, n, 8, 0,
                                   rg_te.as<uint64_t>(), st);
        cudaEventRecord(E.ev[1], st);
        if (rc == HW_OK)
            rc = hw_train_accumulate(c, model.as<uint64_t>(), rg_tr.as<uint64_t>(), n, scr_tr.as<uint64_t>(),
                                     w_tr, st);
        cudaEventRecord(E.ev[2], st);
        if (rc == HW_OK)
            rc = hw_infer(c, model.as<uint64_t>(), rg_te.as<uint64_t>(), n, resp.as<uint64_t>(),
                          sums.as<uint64_t>(), scr_inf.as<uint64_t>(), w_inf, st);
        cudaEventRecord(E.ev[3], st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = HW_ECUDA;
        if (rc == HW_OK && it > 0) {
            out->ms_encrypt = keep_min(out->ms_encrypt, E.ms(0, 1));
            out->ms_train = keep_min(out->ms_train, E.ms(1, 2));
            out->ms_infer = keep_min(out->ms_infer, E.ms(2, 3));
        }
    }
    hw_destroy(c);
    return out->status = rc;
}

// Forward + inverse batched transform of polynomials filling 256 MiB.
int probe_ntt(const hw_params* p, const hw_geometry& g, int dev, int reps, cudaStream_t st,
              hw_tune_entry* out) {
    entry_init(out, g);
    hw_ctx* c = nullptr;
    int rc = hw_create_tuned(p, &g, dev, &c);
    if (rc != HW_OK) return out->status = rc;
    hw_get_geometry(c, &out->geometry);
    hw_sizes S;
    hw_get_sizes(c, &S);
    size_t count = ((size_t)256 << 20) / (8 * (size_t)S.n);
    count -= count % (size_t)S.r;
    if (count == 0) count = S.r;
    DevBuf poly;
    if (!poly.alloc(8 * count * S.n)) {
        hw_destroy(c);
        return out->status = HW_ENOMEM;
    }
    cudaMemsetAsync(poly.p, 0, 8 * count * S.n, st);
    Events E;
    for (int it = 0; it <= reps && rc == HW_OK; it++) {
        cudaEventRecord(E.ev[0], st);
        rc = hw_ntt_forward(c, poly.as<uint64_t>(), count, st);
        if (rc == HW_OK) rc = hw_ntt_inverse(c, poly.as<uint64_t>(), count, st);
        cudaEventRecord(E.ev[1], st);
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = HW_ECUDA;
        if (rc == HW_OK && it > 0) out->ms_ntt = keep_min(out->ms_ntt, E.ms(0, 1));
    }
    hw_destroy(c);
    return out->status = rc;
}

}  // namespace

extern "C" int hw_autotune(const hw_params* p, int dev, size_t n_probe, int32_t reps, hw_geometry* best,
                           hw_tune_entry* entries, size_t max_entries, size_t* n_entries) {
    if (!p || !best) return hw_ctx_fail(HW_EINVAL, "hw_autotune: null argument");
    if (n_probe == 0) n_probe = 1;
    if (reps < 1) reps = 1;
    size_t ng = 0;
    int rc = hw_list_geometries(p, nullptr, 0, &ng);
    if (rc != HW_OK) return rc;
    std::vector<hw_geometry> ext(ng);
    hw_list_geometries(p, ext.data(), ng, &ng);
    if (cudaSetDevice(dev) != cudaSuccess) return hw_ctx_fail(HW_ECUDA, "hw_autotune: cudaSetDevice failed");
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return hw_ctx_fail(HW_ECUDA, "hw_autotune: cudaStreamCreate failed");

    std::vector<hw_tune_entry> all;
    // external-product geometries, each at full occupancy and, where more than
    // one block fits per SM, at half of it
    int best_step = -1;
    double best_ms = 0;
    for (const hw_geometry& g0 : ext) {
        hw_tune_entry e;
        probe_step(p, g0, dev, n_probe, reps, st, &e);
        all.push_back(e);
        const int occ = e.geometry.ext_blocks_per_sm;
        if (e.status == HW_OK && occ >= 2) {
            hw_geometry g1 = g0;
            g1.ext_blocks_per_sm = occ / 2;
            probe_step(p, g1, dev, n_probe, reps, st, &e);
            all.push_back(e);
        }
    }
    for (size_t k = 0; k < all.size(); k++) {
        const hw_tune_entry& e = all[k];
        if (e.status != HW_OK) continue;
        const double t = e.ms_encrypt + e.ms_train + e.ms_infer;
        if (best_step < 0 || t < best_ms) {
            best_step = (int)k;
            best_ms = t;
        }
    }
    // the best step geometry again with its accumulators persisting in L2;
    // the set-aside it takes is given back afterwards.  It changes a
    // context-wide cache setting, so it is kept only when it is at least 2 %
    // faster (timing noise alone must not switch it on)
    if (best_step >= 0) {
        size_t prev = 0;
        cudaDeviceGetLimit(&prev, cudaLimitPersistingL2CacheSize);
        hw_geometry g = all[best_step].geometry;
        g.l2_persist = 1;
        hw_tune_entry e;
        probe_step(p, g, dev, n_probe, reps, st, &e);
        cudaCtxResetPersistingL2Cache();
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, prev);
        cudaGetLastError();
        if (e.status == HW_OK && e.geometry.l2_persist == 1) {
            all.push_back(e);
            const double t = e.ms_encrypt + e.ms_train + e.ms_infer;
            if (t < 0.98 * best_ms) {
                best_step = (int)all.size() - 1;
                best_ms = t;
            }
        }
    }
    // batched-transform variants (radix 8 / 16, 64-bit and, for primes
    // below 2^30, 32-bit arithmetic) with the default step geometry
    const size_t first_ntt = all.size();
    for (int limbs = 1; limbs <= 2; limbs++) {
        if (limbs == 1 && p->prime_bits > 30) continue;
        for (int loge = 3; loge <= 4; loge++) {
            hw_geometry g;
            memset(&g, 0, sizeof(g));
            g.ntt_loge = loge;
            g.ntt_limbs = limbs;
            hw_tune_entry e;
            probe_ntt(p, g, dev, reps, st, &e);
            all.push_back(e);
        }
    }
    int best_ntt = -1;
    for (size_t k = first_ntt; k < all.size(); k++) {
        if (all[k].status != HW_OK) continue;
        if (best_ntt < 0 || all[k].ms_ntt < all[best_ntt].ms_ntt) best_ntt = (int)k;
    }
    cudaStreamDestroy(st);
    if (n_entries) *n_entries = all.size();
    if (entries)
        for (size_t k = 0; k < all.size() && k < max_entries; k++) entries[k] = all[k];
    if (best_step < 0) {
        for (const hw_tune_entry& e : all)
            if (e.status != HW_OK) return e.status == HW_ENOMEM ? hw_ctx_fail(HW_ENOMEM, "hw_autotune: probe does not fit in device memory")
                                                                 : hw_ctx_fail(e.status, "hw_autotune: every geometry failed");
        return hw_ctx_fail(HW_EINVAL, "hw_autotune: no geometry");
    }
    *best = all[best_step].geometry;
    if (best_ntt >= 0) {
        best->ntt_loge = all[best_ntt].geometry.ntt_loge;
        best->ntt_limbs = all[best_ntt].geometry.ntt_limbs;
    }
    return HW_OK;
}
