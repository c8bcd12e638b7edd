/*
 * hwisard.h -- C ABI of the GB300 (sm_103a) homomorphic WiSARD hot path.
 *
 * The library implements encrypted training and inference of an Integer
 * WiSARD (Neumann, Guimaraes, Aranha, Borin, "Homomorphic WiSARDs",
 * PoPETs 2024) over RLWE/RGSW ciphertexts with an RNS modulus
 * Q = q_0 ... q_{r-1}.  Every step runs in CUDA kernels on one GPU; there is
 * no CPU fallback.
 *
 * Conventions
 * -----------
 * - All calls return HW_OK (0) or a negative HW_E* code; the message of the
 *   last failure of the calling thread is in hw_last_error().  The library
 *   never aborts the process.
 * - Arrays passed as "device" pointers live in device memory of the context's
 *   GPU and are owned by the caller; the library never frees them.  "host"
 *   pointers are ordinary host memory (pinned memory makes copies faster).
 * - Calls that take a `stream` (a cudaStream_t, NULL = default stream) only
 *   enqueue work and return; the caller synchronises.  Calls without a stream
 *   are synchronous.
 * - Word = 64-bit unsigned residue.  Polynomials have N = 2^log_n
 *   coefficients; an RNS polynomial is [prime 0..r-1][coefficient 0..N-1].
 * - Canonical (coefficient-domain) layouts:
 *     RLWE   (a, b)       [component a=0,b=1][prime][N], residues in [0, q_i)
 *     LWE    (a', b')     [prime][N a-coefficients, then b]   (r*(N+1) words)
 *     model  H            [RAM k0][ciphertext k1][RLWE]       (Definition 2)
 *   RGSW ciphertexts and the secret key are kept in an internal evaluation
 *   form; hw_export_rgsw() returns the canonical coefficient form
 *   [row 0..2*dnum-1][RLWE].
 */
#ifndef HWISARD_H
#define HWISARD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HW_OK 0
#define HW_EINVAL (-1)    /* bad argument, size or parameter */
#define HW_ENOMEM (-2)    /* a caller buffer is too small */
#define HW_ECUDA (-3)     /* a CUDA call failed; see hw_last_error() */
#define HW_ETIMEOUT (-4)  /* a bounded device-side wait ran out (see hw_check_context) */
#define HW_EMISMATCH (-5) /* object made for other parameters */

/* PD-act activations (Section 3.2): floor(log2(x+1)), min(floor(log2(x+1)),
 * act_arg), and [x > act_arg]. */
#define HW_ACT_LOG 0
#define HW_ACT_BLOG 1
#define HW_ACT_BIN 2

/* What hw_decrypt decrypts. */
#define HW_DEC_RLWE 0  /* count RLWE ciphertexts -> count*N values */
#define HW_DEC_LWE 1   /* count LWE ciphertexts  -> count values */
#define HW_DEC_MODEL 2 /* one model H -> its l*k0*2^a counters W[c][j][addr] */

typedef struct hw_params {
    int32_t log_n;      /* ring dimension N = 2^log_n, 10 <= log_n <= 13 */
    int32_t n_primes;   /* r, 1..3 */
    int32_t prime_bits; /* q_i < 2^prime_bits, q_i = 1 mod 2N, 20 <= bits <= 55 */
    int32_t log_beta;   /* gadget base 2^log_beta; 0 = one digit per prime */
    int32_t log_p;      /* plaintext modulus p = 2^log_p, 1..30 */
    int32_t n_classes;  /* l, 2..64 */
    int32_t n_values;   /* uint8 input values per sample */
    int32_t therm_bits; /* thermometer width T, 1..16 */
    int32_t tuple_bits; /* bits per tuple before hashing (= addr_bits if not hashed) */
    int32_t addr_bits;  /* a, RAM address bits, 1..20 */
    int32_t hash_h3;    /* 1: client hashes each tuple to addr_bits with H3 */
    int32_t act;        /* HW_ACT_* for hw_pdact */
    int32_t act_arg;    /* bound (blog) or threshold (bin) */
    int32_t reserved;
    uint64_t model_seed; /* seeds the bit permutation pi_r and the H3 matrix */
} hw_params;

typedef struct hw_ctx hw_ctx;

/* Derived sizes (words are 64-bit). */
typedef struct hw_sizes {
    int32_t n, r, L, a, s, k0, k1, z, dpp, dnum, n_data, n_slots;
    uint64_t q[4];          /* the RNS primes, descending */
    size_t rlwe_words;      /* 2 r N */
    size_t lwe_words;       /* r (N + 1) */
    size_t rgsw_words;      /* 2 dnum rlwe_words */
    size_t key_words;       /* device secret key buffer */
    size_t model_words;     /* k0 k1 rlwe_words */
    size_t sample_words;    /* n_slots rgsw_words: one encrypted sample */
    size_t resp_words;      /* l k0 lwe_words: responses of one test sample */
    size_t sums_words;      /* l lwe_words: class sums of one test sample */
    int32_t word_bits;      /* 32: external products and encryption transforms run in 32-bit
                               words (every q_i < 2^30, several gadget digits per prime,
                               N <= 2048); 64 otherwise.  Results are the same either way. */
    int32_t reserved;
} hw_sizes;

/* Create a context on `cuda_device` for the given parameters: finds the
 * primes, roots of unity, transform tables, pi_r and (if hashed) the H3
 * matrix, and uploads them.  The RNS modulus and noise distribution are the
 * readings of Section 2.4 (Setup) listed with the project's design notes. */
int hw_create(const hw_params* params, int cuda_device, hw_ctx** out);
/* (Testing hook: with HW_FAULT_ALLOC=k in the environment, the k-th device
 * allocation of each hw_create fails as if the device were out of memory;
 * the call returns HW_ECUDA having freed what it allocated.) */
int hw_destroy(hw_ctx* ctx);

/* Kernel geometry of a context.  It has no counterpart in the paper and
 * changes no result: every geometry produces the same canonical
 * ciphertexts, models, responses and transforms (only the internal
 * evaluation layout of RGSW rows and keys follows ext_loge, so those are
 * valid only within contexts of the same geometry).  0 in a field means the
 * library's default. */
typedef struct hw_geometry {
    int32_t ext_loge;          /* external product: 2^ext_loge residues per thread (radix of the
                                  in-register transform stages); 3 or 4 */
    int32_t ext_np;            /* external product: polynomials transformed together per block, 1 or 2 */
    int32_t ext_blocks_per_sm; /* resident blocks per SM of the persistent training / inference
                                  kernels; 0 = as many as fit (resolved on return) */
    int32_t ntt_loge;          /* hw_ntt_forward/inverse: 2^ntt_loge residues per thread; 3 or 4 */
    int32_t ntt_limbs;         /* hw_ntt_forward/inverse: 32-bit words per residue in the arithmetic:
                                  1 (only when every q_i < 2^30) or 2 */
    int32_t ext_smem;          /* what else the training / inference kernels keep in shared
                                  memory beside one exchange buffer (instead of two): 0 nothing;
                                  1 the accumulator's evaluation form (2*r*N words; HW_EINVAL
                                  where it does not fit); 2 the accumulator polynomials of the
                                  prime being processed (2*N words, off the registers);
                                  3 two exchange buffers plus the first of those two
                                  accumulator polynomials (N words; the second stays in
                                  registers) */
    int32_t l2_persist;        /* 1: the training / inference kernels mark their per-block
                                  accumulators persisting in L2 (an access-policy window on each
                                  launch and a persisting set-aside of this process's context,
                                  sized to those accumulators); 0: off (default) */
    int32_t reserved;
} hw_geometry;

/* hw_create with a chosen geometry (NULL = defaults).  HW_EINVAL if the
 * (ext_loge, ext_np) pair is not built for this ring size or a field is
 * out of range; hw_list_geometries() gives the pairs that are built. */
int hw_create_tuned(const hw_params* params, const hw_geometry* geometry, int cuda_device,
                    hw_ctx** out);
/* Self-check (no counterpart in the paper): HW_OK while the context's device
 * tables (transform, rotation and index tables and the device copy of the
 * context) are byte for byte what hw_create uploaded, HW_EMISMATCH if
 * anything has written into them since, HW_ETIMEOUT if a bounded wait of
 * the batched transform ran out on this device since the library was
 * loaded.  Synchronous; copies the tables back (a few MB).  Lets a
 * long-running caller detect a stray write before it launches work on a
 * damaged context. */
int hw_check_context(const hw_ctx* ctx);
/* The context's geometry with every default resolved. */
int hw_get_geometry(const hw_ctx* ctx, hw_geometry* out);
/* The external-product geometries built for params->log_n (ext_loge,
 * ext_np, ext_smem set; other fields 0), default first; a listed
 * geometry with ext_smem = 1 may still not fit a parameter set.  Host only: needs no GPU.
 * Writes min(*count, max) entries; *count = the number available. */
int hw_list_geometries(const hw_params* params, hw_geometry* out_host, size_t max, size_t* count);

/* One measured candidate of hw_autotune (milliseconds; -1 = not measured). */
typedef struct hw_tune_entry {
    hw_geometry geometry;
    double ms_encrypt; /* encrypt n_probe training + n_probe test samples */
    double ms_train;   /* hw_train_accumulate of n_probe samples */
    double ms_infer;   /* hw_infer of n_probe samples */
    double ms_ntt;     /* forward + inverse transform of the probe polynomials */
    int32_t status;    /* HW_OK, or the error this candidate met */
    int32_t reserved;
} hw_tune_entry;

/* Autotuner (no counterpart in the paper): times every built external-
 * product geometry (and, where it matters, a halved resident-block count;
 * then the fastest one again with l2_persist, kept only when at least 2 %
 * faster) on one step of n_probe training and n_probe test samples -- encryption,
 * training, inference -- and every batched-NTT variant on a batch of
 * polynomials larger than L2, each `reps` times (best time kept), on
 * synthetic inputs in buffers it allocates and frees itself.  *best gets
 * the fastest step geometry combined with the fastest NTT variant;
 * entries_host (may be NULL) gets up to max_entries candidates and
 * *n_entries their number.  Synchronous; uses the whole GPU while it runs.
 * HW_ENOMEM if the probe does not fit in device memory. */
int hw_autotune(const hw_params* params, int cuda_device, size_t n_probe, int32_t reps,
                hw_geometry* best, hw_tune_entry* entries_host, size_t max_entries,
                size_t* n_entries);
int hw_get_sizes(const hw_ctx* ctx, hw_sizes* out);
/* Host copy of the server's index tables: ram_slot[k0*a] gives, for RAM j and
 * address bit i, the encrypted bit slot it reads (-1: constant 0). */
int hw_get_ram_slots(const hw_ctx* ctx, int32_t* ram_slot_host, size_t n);

/* Scratch words hw_train_accumulate / hw_infer need for a batch of n samples:
 * buffers per resident block of the persistent kernels, and for hw_infer at
 * n >= 2 one set of the first CMUX's digit transforms per (RAM, class)
 * (2 dnum r N words each; that CMUX's source is made of stored ciphertexts
 * only, shared by the batch; none when the external product runs in 32-bit
 * words).  Neither grows further with n.  hw_infer_packed needs what
 * hw_infer needs; hw_infer_plain needs hw_infer_scratch_words(ctx, 1). */
size_t hw_train_scratch_words(const hw_ctx* ctx, size_t n);
size_t hw_infer_scratch_words(const hw_ctx* ctx, size_t n);

/* SecretKeyGen (Section 2.4): a ternary RLWE key S_1 drawn from `seed`
 * (coefficient k from word k of the KEY stream, w mod 3 -> 0,+1,-1).
 * key_dev: key_words device words, written. */
int hw_keygen(hw_ctx* ctx, uint64_t seed, uint64_t* key_dev, void* stream);

/* Client pre-processing (Sections 2.3.1-2.3.2, 3.4): quantise each uint8
 * value to level (v*(T+1))>>8, thermometer-encode it; hashed contexts also
 * apply pi_r and H3 per tuple.  values_dev: n*n_values bytes; bits_dev:
 * n*n_data bytes (0/1), written. */
int hw_encode(hw_ctx* ctx, const uint8_t* values_dev, size_t n, uint8_t* bits_dev, void* stream);

/* EncRGSW of every bit of n samples (Section 3.4: samples and labels are
 * encrypted bit by bit).  Slot b < L is label bit b (LSB first), slot L+d is
 * data bit d.  labels_dev: n uint32 labels, or NULL to skip the label slots
 * (inference).  Sample i uses stream index (first_sample+i)*n_slots+slot of
 * the RGSW_A / RGSW_E streams keyed by `seed`.  rgsw_dev: n*sample_words
 * device words, written (label slots untouched when labels_dev is NULL). */
int hw_encrypt_sample(hw_ctx* ctx, const uint64_t* key_dev, const uint8_t* bits_dev,
                      const uint32_t* labels_dev, size_t n, uint64_t seed, uint64_t first_sample,
                      uint64_t* rgsw_dev, void* stream);

/* Homomorphic training (Algorithm 6): for each sample and RAM j, the Inverse
 * Vertical Packing (Algorithm 5) of b = [label bits, tuple bits of RAM j] and
 * the trivial RLWE (0, Delta) is added into H[j] (mod q_i).  model_dev:
 * model_words device words, updated in place: each (sample, RAM) item adds
 * its stored ciphertexts with 64-bit atomic adds (exact integer sums, so the
 * result does not depend on the order the items finish in), then one pass
 * reduces H mod q_i; batches larger than 2^64 / max q_i - 2 samples are
 * split into such passes.  No other work may read or write the model while
 * the call runs.  scratch_dev: at least hw_train_scratch_words(ctx, n)
 * device words. */
int hw_train_accumulate(hw_ctx* ctx, uint64_t* model_dev, const uint64_t* rgsw_dev, size_t n,
                        uint64_t* scratch_dev, size_t scratch_words, void* stream);

/* Homomorphic inference with PD-act (Algorithm 7): for each sample, RAM j and
 * class c, the Vertical Packing (Algorithm 3) of H[j] with the label bits of c
 * in clear, then ExtractLWE(., 0).  resp_dev: n*resp_words words, laid out
 * [sample][class][RAM][LWE]; sums_dev: n*sums_words words, [sample][class][LWE],
 * the per-class sums over RAMs (mod q_i).  Both written. */
int hw_infer(hw_ctx* ctx, const uint64_t* model_dev, const uint64_t* rgsw_dev, size_t n,
             uint64_t* resp_dev, uint64_t* sums_dev, uint64_t* scratch_dev, size_t scratch_words,
             void* stream);

/* hw_infer with horizontal packing (Section 6): the classes that share a
 * stored ciphertext (c = g mod 2^z) and differ only in clear label bits
 * above z are answered by one VP -- the accumulator is not rotated by those
 * bits, and class c's response is ExtractLWE(acc, c >> z).  It needs
 * min(l, 2^z) VPs per (sample, RAM) instead of l (cfg1: 1 instead of 2).
 * Same buffers and layouts as hw_infer; the responses are different
 * ciphertexts that decrypt to the same counters.  When a tree level is an
 * encrypted address bit (z > L) nothing can be packed and it runs hw_infer. */
int hw_infer_packed(hw_ctx* ctx, const uint64_t* model_dev, const uint64_t* rgsw_dev, size_t n,
                    uint64_t* resp_dev, uint64_t* sums_dev, uint64_t* scratch_dev, size_t scratch_words,
                    void* stream);

/* Inference against a model in clear (Section 3.6.2 remarks that inference
 * is faster when the model is not encrypted; the algorithm is this
 * library's reading).  The lookup tables of RAM j, class c are plaintext
 * polynomials T_{j,c,v}, v < 2^zt with zt = max(0, z - L): coefficient k of
 * T_{j,c,v} is the counter of address v + 2^zt k.  The blind rotation then
 * depends on the sample only: R = (0, Delta) rotated by address bits
 * zt..a-1 with weights X^-(2^0), X^-(2^1), ... runs once per (sample, RAM),
 * and class c's response is ExtractLWE(R * T_{j,c,0}, 0) (zt = 0) or
 * ExtractLWE(CMUX(C_{bit 0}, R * T_{j,c,1}, R * T_{j,c,0}), 0) (zt = 1):
 * coefficient 0 of Delta X^-addr T(X) is Delta T[addr].  The noise of R is
 * multiplied by the table's coefficient sum (the number of training samples
 * of the class for a trained model).
 * hw_plain_model_load: counts_dev [l][k0][2^a] int64 (Algorithm 4's W, as
 * hw_decrypt gives a model back), reduced mod q_i -> plain_dev, the
 * hw_plain_model_words(ctx) words of tables in the internal evaluation form
 * (valid for contexts of the same geometry).
 * hw_infer_plain: responses and sums laid out as hw_infer's (they decrypt to
 * the same counters; the ciphertexts differ); scratch of
 * hw_infer_scratch_words(ctx, 1) words whatever n. */
size_t hw_plain_model_words(const hw_ctx* ctx);
int hw_plain_model_load(hw_ctx* ctx, const int64_t* counts_dev, uint64_t* plain_dev, void* stream);
int hw_infer_plain(hw_ctx* ctx, const uint64_t* plain_dev, const uint64_t* rgsw_dev, size_t n,
                   uint64_t* resp_dev, uint64_t* sums_dev, uint64_t* scratch_dev, size_t scratch_words,
                   void* stream);

/* DecRLWE / DecLWE (Section 2.4): phase b - a*s combined over the primes by
 * the CRT and rounded, m = floor((p*phi + floor(Q/2)) / Q) mod p.  what =
 * HW_DEC_RLWE: obj_dev holds count RLWEs, out_dev gets count*N values;
 * HW_DEC_LWE: count LWEs, count values; HW_DEC_MODEL: obj_dev is one model
 * (count = 1), out_dev gets its l*k0*2^a counters [class][RAM][address]
 * (see hw_model_words).  out_dev: int64 device array. */
int hw_decrypt(hw_ctx* ctx, const uint64_t* key_dev, int what, const uint64_t* obj_dev,
               size_t count, int64_t* out_dev, void* stream);

/* The model H of Definition 2: k0 RAMs x k1 stored RLWEs (the LUT index
 * m = c + 2^L addr of class c, address addr -- label bits low, as
 * Algorithm 6 orders the bits -- is coefficient m >> z of stored ciphertext
 * slot(m mod 2^z); only the slots a label < l reaches are stored).  The
 * model is a caller buffer of hw_model_words(ctx) device words.
 * hw_model_zero: H <- {0} (Algorithm 6's initial model: trivial encryptions
 * of 0), on the stream.
 * hw_decrypt(..., HW_DEC_MODEL, model_dev, 1, out_dev, ...) writes the
 * l * k0 * 2^a counters [class c][RAM j][address] (Algorithm 4's W after
 * homomorphic training), int64 in [0, p). */
size_t hw_model_words(const hw_ctx* ctx);
int hw_model_zero(hw_ctx* ctx, uint64_t* model_dev, void* stream);

/* Exported model (no counterpart in the paper; the model is additive,
 * Section 3.6.2, so training can stop after any batch and resume from the
 * saved model with bit-identical results).  Layout, uint64 words:
 *   [0] HW_MODEL_MAGIC  [1] HW_MODEL_VERSION  [2] hw_params_digest
 *   [3] samples trained (the caller's count, stored as given)
 *   [4] k0  [5] k1  [6] r  [7] N  [8] model words M
 *   then the M canonical words of H ([RAM][slot][RLWE], residues < q_i).
 * hw_model_export: model_dev -> out_host (hw_model_export_words(ctx)
 * words); synchronous (waits for the stream).
 * hw_model_import: in_host -> model_dev after checking the header (magic,
 * version, the parameter digest: HW_EMISMATCH for another parameter set,
 * the shape) and that every word is reduced mod its prime (HW_EINVAL);
 * *samples gets the stored count.  Synchronous.
 * hw_model_header_check: the header checks alone, host only (no context,
 * no GPU): HW_EINVAL (not a model, other version, word count),
 * HW_EMISMATCH (other parameters).
 * hw_params_digest: FNV-1a 64 over every hw_params field but `reserved`
 * (each as a little-endian 64-bit word, model_seed last); host only. */
#define HW_MODEL_MAGIC 0x3144524153495748ULL /* "HWISARD1" little-endian */
#define HW_MODEL_VERSION 1
#define HW_MODEL_HEADER_WORDS 9
int hw_params_digest(const hw_params* params, uint64_t* out);
size_t hw_model_export_words(const hw_ctx* ctx);
int hw_model_export(hw_ctx* ctx, const uint64_t* model_dev, uint64_t samples, uint64_t* out_host,
                    size_t n_words, void* stream);
int hw_model_import(hw_ctx* ctx, const uint64_t* in_host, size_t n_words, uint64_t* model_dev,
                    uint64_t* samples, void* stream);
int hw_model_header_check(const hw_params* params, const uint64_t* in_host, size_t n_words,
                          uint64_t* samples);

/* PD-act (Section 3.5.1): counts_dev [n][l][k0] decrypted responses ->
 * scores_dev [n][l] (sum of activated counts) and labels_dev [n] (arg-max,
 * ties to the lowest class). */
int hw_pdact(hw_ctx* ctx, const int64_t* counts_dev, size_t n, int64_t* scores_dev,
             int32_t* labels_dev, void* stream);

/* hw_infer without caller scratch (the paper has no counterpart; this is a
 * library convenience).  For callers that cannot allocate device memory --
 * a request loop that may not call cudaMalloc, or a plug-in that only sees
 * the input and output buffers -- the per-block accumulators of the
 * inference kernel (and their evaluation forms) come from a static device
 * array of
 * HW_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Results are identical to hw_infer().
 * - The first call on a device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 * - All calls share the array: calls whose work overlaps on the GPU (other
 *   streams, other threads, other contexts on the same device) race.  Order
 *   them, e.g. on one stream.
 * - Each resident block of the inference kernel takes S * rlwe_words * 8
 *   bytes of the array, S = 2 when the context's geometry keeps the
 *   accumulator's evaluation form in shared memory (ext_smem = 1) and 3
 *   otherwise.  Rings where one block does not fit are rejected with
 *   HW_EINVAL; the number of resident blocks is capped so that all of them
 *   fit (fewer blocks: the same results, more slowly).
 * - Nothing is allocated or freed: no cudaMalloc, cudaFree or allocating
 *   library call. */
#define HW_STATIC_SCRATCH_BYTES (48u << 20)
int hw_infer_static_scratch(hw_ctx* ctx, const uint64_t* model_dev, const uint64_t* rgsw_dev,
                            size_t n, uint64_t* resp_dev, uint64_t* sums_dev, void* stream);

/* PackingKeySwitching (Section 2.4; Algorithm 7 returns its result for
 * PD-act): packs the l * k0 responses of each test sample into one RLWE
 * encrypting sum_i u_i X^i, i = c * k0 + j (the response order), so a
 * client receives one RLWE per sample instead of l * k0 LWEs.
 * Key: hw_ksk_words(ctx) device words, N * dnum RLWE rows encrypting
 * s_x * g_rho (x < N, gadget row rho) under the secret key, made by
 * hw_ksk_gen from key_dev and `seed` (KSK_A / KSK_E streams).
 * Packing: C = sum_i X^i (0, b_i) - sum_{x,rho} KS_{x,rho} * D_{x,rho}(X),
 * D_{x,rho}(X) = sum_i Dec_rho(a_{i,x}) X^i (the RGSW gadget).
 * resp_dev: n * resp_words (as hw_infer writes them); packed_dev: n *
 * rlwe_words, canonical RLWEs (decrypt with HW_DEC_RLWE: coefficient i is
 * u_i); scratch_dev: scratch_words device words, at least
 * hw_pack_scratch_words(ctx, 1); hw_pack_responses packs as many samples per
 * pass as the scratch holds (hw_pack_scratch_words(ctx, n): all n in one
 * pass, four launches), so a larger scratch means fewer, fuller launches.
 * HW_EINVAL when l * k0 > N. */
size_t hw_ksk_words(const hw_ctx* ctx);
int hw_ksk_gen(hw_ctx* ctx, const uint64_t* key_dev, uint64_t seed, uint64_t* ksk_dev, void* stream);
size_t hw_pack_scratch_words(const hw_ctx* ctx, size_t n);
int hw_pack_responses(hw_ctx* ctx, const uint64_t* ksk_dev, const uint64_t* resp_dev, size_t n,
                      uint64_t* packed_dev, uint64_t* scratch_dev, size_t scratch_words, void* stream);

/* Dataset balancing (Section 3.6.1): for each of n encrypted training
 * samples (the same rgsw_dev as hw_train_accumulate), a small IVP over its
 * label bits -- BlindRotate from (0, Delta) with weights X^(+2^t) over the
 * L label slots -- gives an RLWE with Delta at coefficient = label; the
 * batch is added (mod q_i) into counts_dev (rlwe_words, caller-zeroed
 * before the first batch), whose coefficient c then decrypts
 * (hw_decrypt, HW_DEC_RLWE) to the number of class-c samples.
 * scratch_dev: hw_count_scratch_words(ctx, n) device words. */
size_t hw_count_scratch_words(const hw_ctx* ctx, size_t n);
int hw_count_classes(hw_ctx* ctx, uint64_t* counts_dev, const uint64_t* rgsw_dev, size_t n,
                     uint64_t* scratch_dev, size_t scratch_words, void* stream);

/* PD-act with the balancing rescale (Section 3.6.1 leaves the rule open;
 * this library's reading): class_counts_dev [l] (the decrypted counts),
 * counters of class c scaled by n_ref / n_c with floor division before the
 * activation (n_ref = the largest count; classes with n_c = 0 unchanged) --
 * the same as training on a set where every class is repeated up to n_ref
 * samples.  Layouts as hw_pdact. */
int hw_pdact_balanced(hw_ctx* ctx, const int64_t* counts_dev, const int64_t* class_counts_dev, size_t n,
                      int64_t* scores_dev, int32_t* labels_dev, void* stream);

/* Canonical coefficient form of count RGSW ciphertexts (for checks). */
int hw_export_rgsw(hw_ctx* ctx, const uint64_t* rgsw_dev, size_t count, uint64_t* out_dev,
                   void* stream);

/* The inverse of hw_export_rgsw: count RGSW ciphertexts in canonical
 * coefficient form ([row 0..2*dnum-1][RLWE], words reduced mod q_i on
 * entry) into this context's internal evaluation form, as hw_train_accumulate
 * and hw_infer read it.  No counterpart in the paper: it lets ciphertexts
 * made elsewhere (another implementation, or a context of another geometry,
 * via hw_export_rgsw) be used here.  canonical_dev and rgsw_dev may be the
 * same buffer. */
int hw_import_rgsw(hw_ctx* ctx, const uint64_t* canonical_dev, size_t count, uint64_t* rgsw_dev,
                   void* stream);

/* Batched forward / inverse negacyclic transform of count polynomials in
 * place, polynomial t using prime (t mod r).  The forward output is in the
 * library's evaluation order; inverse(forward(x)) = x.  In 32-bit
 * arithmetic (ntt_limbs = 1) with a 16-byte aligned poly_dev, a persistent
 * grid streams the polynomials through shared memory with bulk asynchronous
 * copies (one in flight per block while it transforms the previous one);
 * its waits are bounded, and one that runs out (not expected) stops the
 * block and makes hw_check_context return HW_ETIMEOUT.  Otherwise one
 * block transforms one polynomial. */
int hw_ntt_forward(hw_ctx* ctx, uint64_t* poly_dev, size_t count, void* stream);
int hw_ntt_inverse(hw_ctx* ctx, uint64_t* poly_dev, size_t count, void* stream);

/* Integer-issue ceiling of the library's butterfly forms on `cuda_device`
 * (no counterpart in the paper: the measured denominator beside the
 * derived multiply-count peak).  Register-only loops, one 512-thread block
 * per SM; out_host[0..3] = G butterflies/s of the 64-bit lazy Cooley-Tukey,
 * the 64-bit Harvey Gentleman-Sande, and their 32-bit forms.  Synchronous;
 * takes about a second of the whole GPU. */
int hw_butterfly_rates(int cuda_device, double* out_host);

/* Number of kernel launches the library has issued since the context was
 * created (all calls). */
uint64_t hw_launch_count(const hw_ctx* ctx);

const char* hw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HWISARD_H */
