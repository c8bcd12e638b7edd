/*
 * oracle.c -- plain, slow CPU reference of the homomorphic WiSARD hot path
 * (Neumann, Guimaraes, Aranha, Borin: "Homomorphic WiSARDs", PoPETs 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, table
 * or constant generator with the CUDA library; the two meet only through the
 * seeded raw inputs of the synthdata package and the published definition of
 * the Philox4x64-10 generator, which each side implements on its own.
 *
 * Every routine is written for a reader checking it against the paper:
 * modular products are computed as (a*b) mod q with 128-bit integers, the
 * number-theoretic transform is the textbook twisted radix-2 Cooley-Tukey
 * transform (pinned against the schoolbook negacyclic product), and the
 * algorithms follow the paper's step order.
 *
 * Representation: an RLWE ciphertext (a, b) is stored in the coefficient
 * domain as [component a,b][prime 0..r-1][coefficient 0..N-1] residues in
 * [0, q_i).  An RGSW ciphertext is [row 0..2*dnum-1][component][prime][N];
 * the oracle keeps its rows in its own evaluation (NTT) order, a cache of
 * the coefficient form that or_rgsw_export() inverts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;
typedef unsigned __int128 u128;

#define OR_MAXP 4
#define OR_CDT_LEN 38 /* support -19..19, 39 values, 38 thresholds */

/* ------------------------------------------------------------------ */
/* Modular arithmetic on residues in [0, q).                           */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : (u64)((u128)a + q - b); }
static u64 negmod(u64 a, u64 q) { return a == 0 ? 0 : q - a; }

static u64 powmod(u64 base, u64 e, u64 q) {
    u64 r = 1 % q, b = base % q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* Fermat inverse, q prime. */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

/* A signed integer reduced into [0, q). */
static u64 from_signed(long long v, u64 q) {
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) + 1; /* |v| without overflow */
    m %= q;
    return m == 0 ? 0 : q - m;
}

/* ------------------------------------------------------------------ */
/* Primes: deterministic Miller-Rabin for 64-bit inputs.               */
/* ------------------------------------------------------------------ */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int k = 1; k < s; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* The r largest primes q < 2^bits with q = 1 (mod 2N), descending. */
int or_find_primes(int log_n, int bits, int r, u64 *out) {
    u64 m = (u64)2 << log_n;              /* 2N */
    u64 top = ((u64)1 << bits) - 1;       /* largest value below 2^bits */
    u64 q = (top - 1) / m * m + 1;        /* largest value = 1 mod 2N */
    int found = 0;
    while (found < r && q > m) {
        if (or_is_prime(q)) out[found++] = q;
        q -= m;
    }
    return found == r ? 0 : -1;
}

/* A primitive 2N-th root of unity: psi = x^((q-1)/2N) for the smallest
 * x >= 2 whose power satisfies psi^N = -1 (so psi has order exactly 2N). */
u64 or_find_psi(u64 q, int log_n) {
    u64 n = (u64)1 << log_n;
    for (u64 x = 2; x < q; x++) {
        u64 psi = powmod(x, (q - 1) / (2 * n), q);
        if (powmod(psi, n, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11).                  */
/* ------------------------------------------------------------------ */
void or_philox(const u64 ctr[4], const u64 key[2], u64 out[4]) {
    const u64 M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const u64 W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    u64 x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    u64 k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        u128 p0 = (u128)M0 * x0, p1 = (u128)M1 * x2;
        u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0;
        u64 hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;
        x0 = hi1 ^ x1 ^ k0;
        x1 = lo1;
        x2 = hi0 ^ x3 ^ k1;
        x3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags, carried in the second key word. */
enum { TAG_KEY = 1, TAG_RGSW_A = 2, TAG_RGSW_E = 3, TAG_PERM = 4, TAG_H3 = 5, TAG_KSK_A = 7, TAG_KSK_E = 8 };

static void draw(u64 seed, u64 tag, u64 c0, u64 c1, u64 c2, u64 out[4]) {
    u64 ctr[4] = {c0, c1, c2, 0};
    u64 key[2] = {seed, tag};
    or_philox(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* Context.                                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int log_n, n, r;
    int log_beta;   /* 0: one digit per prime (the digit is the centred residue) */
    int dpp;        /* digits per prime */
    int dnum;       /* r * dpp gadget rows per half of an RGSW */
    u64 q[OR_MAXP];
    u64 psi[OR_MAXP];
    u64 cdt[OR_CDT_LEN];
} or_ctx;

or_ctx *or_ctx_new(int log_n, int r, const u64 *q, const u64 *psi, int log_beta, int dpp,
                   const u64 *cdt) {
    if (r < 1 || r > OR_MAXP) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->log_n = log_n;
    c->n = 1 << log_n;
    c->r = r;
    c->log_beta = log_beta;
    c->dpp = dpp;
    c->dnum = r * dpp;
    for (int i = 0; i < r; i++) { c->q[i] = q[i]; c->psi[i] = psi[i]; }
    memcpy(c->cdt, cdt, sizeof(c->cdt));
    return c;
}

void or_ctx_free(or_ctx *c) { free(c); }

size_t or_rlwe_words(const or_ctx *c) { return (size_t)2 * c->r * c->n; }
size_t or_rgsw_words(const or_ctx *c) { return (size_t)2 * c->dnum * or_rlwe_words(c); }

/* ------------------------------------------------------------------ */
/* Ring R_q = Z_q[X]/(X^N+1).                                          */
/* ------------------------------------------------------------------ */

/* Schoolbook negacyclic product: X^N = -1 (the ring's definition). */
void or_poly_mul_schoolbook(const u64 *a, const u64 *b, u64 *out, int n, u64 q) {
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < n) out[k] = addmod(out[k], p, q);
            else out[k - n] = submod(out[k - n], p, q);
        }
}

static void bit_reverse(u64 *a, int log_n) {
    int n = 1 << log_n;
    for (int i = 0; i < n; i++) {
        int j = 0;
        for (int b = 0; b < log_n; b++) j |= ((i >> b) & 1) << (log_n - 1 - b);
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* Forward negacyclic NTT: out[k] = sum_i a[i] * psi^((2k+1) i), i.e. the
 * evaluation of a at the odd powers of psi.  Textbook form: twist by psi^i,
 * then the iterative radix-2 Cooley-Tukey cyclic transform with omega=psi^2. */
void or_ntt_fwd(u64 *a, int log_n, u64 q, u64 psi) {
    int n = 1 << log_n;
    u64 tw = 1;
    for (int i = 0; i < n; i++) { a[i] = mulmod(a[i], tw, q); tw = mulmod(tw, psi, q); }
    bit_reverse(a, log_n);
    u64 omega = mulmod(psi, psi, q);
    for (int len = 2; len <= n; len <<= 1) {
        u64 wlen = powmod(omega, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 w = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + len / 2], w, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
}

/* Inverse of or_ntt_fwd: cyclic inverse transform with omega^-1, scale by
 * N^-1, then untwist by psi^-i. */
void or_ntt_inv(u64 *a, int log_n, u64 q, u64 psi) {
    int n = 1 << log_n;
    bit_reverse(a, log_n);
    u64 omega_inv = invmod(mulmod(psi, psi, q), q);
    for (int len = 2; len <= n; len <<= 1) {
        u64 wlen = powmod(omega_inv, (u64)(n / len), q);
        for (int i = 0; i < n; i += len) {
            u64 w = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j], v = mulmod(a[i + j + len / 2], w, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
    u64 n_inv = invmod((u64)n % q, q), psi_inv = invmod(psi, q), tw = n_inv;
    for (int i = 0; i < n; i++) { a[i] = mulmod(a[i], tw, q); tw = mulmod(tw, psi_inv, q); }
}

/* Negacyclic product through the transform. */
void or_poly_mul(const u64 *a, const u64 *b, u64 *out, int log_n, u64 q, u64 psi) {
    int n = 1 << log_n;
    u64 *ta = (u64 *)malloc(sizeof(u64) * n), *tb = (u64 *)malloc(sizeof(u64) * n);
    memcpy(ta, a, sizeof(u64) * n);
    memcpy(tb, b, sizeof(u64) * n);
    or_ntt_fwd(ta, log_n, q, psi);
    or_ntt_fwd(tb, log_n, q, psi);
    for (int k = 0; k < n; k++) out[k] = mulmod(ta[k], tb[k], q);
    or_ntt_inv(out, log_n, q, psi);
    free(ta);
    free(tb);
}

/* c * X^e for e in [0, 2N): coefficient i moves to i+e; wrapping past N
 * flips its sign because X^N = -1.  Applied to both components. */
void or_rlwe_rotate(const or_ctx *c, const u64 *in, long long e, u64 *out) {
    int n = c->n;
    long long two_n = 2LL * n;
    e %= two_n;
    if (e < 0) e += two_n;
    for (int comp = 0; comp < 2; comp++)
        for (int j = 0; j < c->r; j++) {
            const u64 *src = in + ((size_t)comp * c->r + j) * n;
            u64 *dst = out + ((size_t)comp * c->r + j) * n;
            u64 q = c->q[j];
            for (int i = 0; i < n; i++) {
                long long t = i + e;
                int neg = 0;
                while (t >= n) { t -= n; neg ^= 1; }
                dst[t] = neg ? negmod(src[i], q) : src[i];
            }
        }
}

void or_rlwe_add(const or_ctx *c, u64 *acc, const u64 *x) {
    for (int comp = 0; comp < 2; comp++)
        for (int j = 0; j < c->r; j++) {
            size_t off = ((size_t)comp * c->r + j) * c->n;
            for (int i = 0; i < c->n; i++) acc[off + i] = addmod(acc[off + i], x[off + i], c->q[j]);
        }
}

/* ct * T for a plaintext polynomial T with integer coefficients (reduced
 * into each prime): both components multiplied by T in R_q, so the phase is
 * multiplied by T exactly -- (b T) - (a T) s = (b - a s) T.  Used by the
 * unencrypted-model inference, whose lookup tables are plaintexts. */
void or_rlwe_mul_plain(const or_ctx *c, const u64 *ct, const long long *t, u64 *out) {
    int n = c->n;
    u64 *tq = (u64 *)malloc(sizeof(u64) * n);
    for (int j = 0; j < c->r; j++) {
        for (int i = 0; i < n; i++) tq[i] = from_signed(t[i], c->q[j]);
        for (int comp = 0; comp < 2; comp++) {
            size_t off = ((size_t)comp * c->r + j) * n;
            or_poly_mul(ct + off, tq, out + off, c->log_n, c->q[j], c->psi[j]);
        }
    }
    free(tq);
}

void or_rlwe_sub(const or_ctx *c, u64 *acc, const u64 *x) {
    for (int comp = 0; comp < 2; comp++)
        for (int j = 0; j < c->r; j++) {
            size_t off = ((size_t)comp * c->r + j) * c->n;
            for (int i = 0; i < c->n; i++) acc[off + i] = submod(acc[off + i], x[off + i], c->q[j]);
        }
}

/* ------------------------------------------------------------------ */
/* Sampling (Section 2.1: uniform U and Gaussian G(sigma)).            */
/* ------------------------------------------------------------------ */

/* Ternary secret key S_1, one coefficient per 64-bit word: w mod 3 in
 * {0,1,2} -> {0,+1,-1}. */
void or_keygen(const or_ctx *c, u64 seed, int8_t *s) {
    for (int k = 0; k < c->n; k++) {
        u64 w[4];
        draw(seed, TAG_KEY, (u64)k >> 2, 0, 0, w);
        u64 v = w[k & 3] % 3;
        s[k] = v == 0 ? 0 : (v == 1 ? 1 : -1);
    }
}

/* Discrete Gaussian by inversion of the cumulative table: u is a 63-bit
 * uniform integer and the sample is -19 plus the number of thresholds <= u. */
static long long gaussian(const or_ctx *c, u64 w) {
    u64 u = w >> 1;
    int cnt = 0;
    for (int i = 0; i < OR_CDT_LEN; i++) cnt += (u >= c->cdt[i]);
    return (long long)cnt - 19;
}

long long or_gaussian(const or_ctx *c, u64 w) { return gaussian(c, w); }

/* ------------------------------------------------------------------ */
/* RGSW encryption (Section 2.4, EncRGSW): 2*dnum RLWE encryptions of   */
/* zero plus m*G.  Gadget rows follow the RNS reading: row rho = i*dpp  */
/* + k carries g = beta^k at prime i and 0 at the other primes (for     */
/* beta = q_i this is the CRT idempotent, residue 1 at prime i).        */
/* Rows 0..dnum-1 add m*g to b, rows dnum.. add m*g to a.               */
/*                                                                      */
/* The mask a ~ U(R_q) (Section 2.4 fixes no domain for it) is drawn    */
/* by its values at the N roots of X^N + 1: the evaluation map is a     */
/* bijection of R_q, so uniform values are a uniform a.  Sampling index */
/* k is the value at zeta_k = psi_min^(2 brv(k) + 1), psi_min the       */
/* smallest primitive 2N-th root of unity mod q and brv the log2(N)-bit */
/* reversal; its word pair is that of coefficient k before.             */
/* ------------------------------------------------------------------ */

static int brv_int(int x, int log_n) {
    int y = 0;
    for (int b = 0; b < log_n; b++) y |= ((x >> b) & 1) << (log_n - 1 - b);
    return y;
}

/* The odd exponent v with psi^v = psi_min: the odd powers of a primitive
 * 2N-th root are all of them, so psi_min is the smallest of those. */
static u64 min_root_exponent(u64 q, u64 psi, int n) {
    u64 step = mulmod(psi, psi, q), x = psi, best = psi, v = 1;
    for (u64 e = 1; e < 2 * (u64)n; e += 2) {
        if (x < best) { best = x; v = e; }
        x = mulmod(x, step, q);
    }
    return v;
}

/* a's coefficients from its values U[k] = a(zeta_k): zeta_k is this
 * oracle's evaluation point psi^(2m+1) for m = (v (2 brv(k) + 1) mod 2N -
 * 1) / 2, the slot m of its natural evaluation order; then the inverse
 * transform. */
static void mask_from_points(const or_ctx *c, int j, const u64 *U, u64 *a) {
    int n = c->n, log_n = c->log_n;
    u64 v = min_root_exponent(c->q[j], c->psi[j], n);
    for (int k = 0; k < n; k++) {
        u64 y = (v * (2 * (u64)brv_int(k, log_n) + 1)) % (2 * (u64)n);
        a[(y - 1) / 2] = U[k];
    }
    or_ntt_inv(a, log_n, c->q[j], c->psi[j]);
}
void or_encrypt_rgsw(const or_ctx *c, const int8_t *s, u64 seed, u64 stream_idx, int bit,
                     int trivial, u64 *rgsw_ntt) {
    int n = c->n, r = c->r;
    u64 *spoly = (u64 *)malloc(sizeof(u64) * n), *U = (u64 *)malloc(sizeof(u64) * n);
    u64 *a = (u64 *)malloc(sizeof(u64) * n), *b = (u64 *)malloc(sizeof(u64) * n);
    long long *e = (long long *)malloc(sizeof(long long) * n);
    size_t rlwe = or_rlwe_words(c);
    for (int row = 0; row < 2 * c->dnum; row++) {
        for (int k = 0; k < n; k++) {
            u64 w[4];
            draw(seed, TAG_RGSW_E, (u64)k >> 2, (u64)row, stream_idx, w);
            e[k] = trivial ? 0 : gaussian(c, w[k & 3]);
        }
        int rho = row % c->dnum, gi = rho / c->dpp, gk = rho % c->dpp;
        for (int j = 0; j < r; j++) {
            u64 q = c->q[j];
            for (int k = 0; k < n; k++) spoly[k] = from_signed(s[k], q);
            for (int k = 0; k < n; k++) {
                u64 w[4];
                draw(seed, TAG_RGSW_A, (u64)k >> 1, (u64)row * r + j, stream_idx, w);
                u64 hi = w[2 * (k & 1)], lo = w[2 * (k & 1) + 1];
                U[k] = (u64)((((u128)hi << 64) | lo) % q);
            }
            if (trivial)
                memset(a, 0, sizeof(u64) * n);
            else
                mask_from_points(c, j, U, a);
            or_poly_mul(a, spoly, b, c->log_n, q, c->psi[j]);
            for (int k = 0; k < n; k++) b[k] = addmod(b[k], from_signed(e[k], q), q);
            if (bit && j == gi) {
                u64 g = c->log_beta ? powmod((u64)1 << c->log_beta, (u64)gk, q) : 1;
                if (row < c->dnum) b[0] = addmod(b[0], g, q);
                else a[0] = addmod(a[0], g, q);
            }
            u64 *dst_a = rgsw_ntt + (size_t)row * rlwe + (size_t)(0 * r + j) * n;
            u64 *dst_b = rgsw_ntt + (size_t)row * rlwe + (size_t)(1 * r + j) * n;
            memcpy(dst_a, a, sizeof(u64) * n);
            memcpy(dst_b, b, sizeof(u64) * n);
            or_ntt_fwd(dst_a, c->log_n, q, c->psi[j]);
            or_ntt_fwd(dst_b, c->log_n, q, c->psi[j]);
        }
    }
    free(spoly); free(U); free(a); free(b); free(e);
}

/* Coefficient form of an RGSW held in the oracle's evaluation order. */
void or_rgsw_export(const or_ctx *c, const u64 *rgsw_ntt, u64 *out) {
    size_t total = or_rgsw_words(c);
    memcpy(out, rgsw_ntt, sizeof(u64) * total);
    for (int row = 0; row < 2 * c->dnum; row++)
        for (int comp = 0; comp < 2; comp++)
            for (int j = 0; j < c->r; j++)
                or_ntt_inv(out + ((size_t)(row * 2 + comp) * c->r + j) * c->n, c->log_n, c->q[j],
                           c->psi[j]);
}

/* RLWE encryption of a message polynomial already scaled by Delta (given as
 * residues m_scaled[r][N]), under the RGSW_A/RGSW_E streams of row 0.  Used by
 * tests to build RLWE inputs. */
void or_encrypt_rlwe(const or_ctx *c, const int8_t *s, u64 seed, u64 stream_idx,
                     const u64 *m_scaled, int trivial, u64 *out) {
    int n = c->n, r = c->r;
    u64 *spoly = (u64 *)malloc(sizeof(u64) * n);
    long long *e = (long long *)malloc(sizeof(long long) * n);
    for (int k = 0; k < n; k++) {
        u64 w[4];
        draw(seed, TAG_RGSW_E, (u64)k >> 2, 0, stream_idx, w);
        e[k] = trivial ? 0 : gaussian(c, w[k & 3]);
    }
    for (int j = 0; j < r; j++) {
        u64 q = c->q[j];
        u64 *a = out + (size_t)(0 * r + j) * n, *b = out + (size_t)(1 * r + j) * n;
        for (int k = 0; k < n; k++) spoly[k] = from_signed(s[k], q);
        for (int k = 0; k < n; k++) {
            u64 w[4];
            draw(seed, TAG_RGSW_A, (u64)k >> 1, (u64)j, stream_idx, w);
            u64 hi = w[2 * (k & 1)], lo = w[2 * (k & 1) + 1];
            a[k] = trivial ? 0 : (u64)((((u128)hi << 64) | lo) % q);
        }
        or_poly_mul(a, spoly, b, c->log_n, q, c->psi[j]);
        for (int k = 0; k < n; k++)
            b[k] = addmod(addmod(b[k], from_signed(e[k], q), q), m_scaled[(size_t)j * n + k], q);
    }
    free(spoly); free(e);
}

/* Phase b - a*s of an RLWE, residues [r][N]. */
void or_rlwe_phase(const or_ctx *c, const int8_t *s, const u64 *ct, u64 *phase) {
    int n = c->n, r = c->r;
    u64 *spoly = (u64 *)malloc(sizeof(u64) * n), *as = (u64 *)malloc(sizeof(u64) * n);
    for (int j = 0; j < r; j++) {
        u64 q = c->q[j];
        for (int k = 0; k < n; k++) spoly[k] = from_signed(s[k], q);
        or_poly_mul(ct + (size_t)(0 * r + j) * n, spoly, as, c->log_n, q, c->psi[j]);
        for (int k = 0; k < n; k++) phase[(size_t)j * n + k] = submod(ct[(size_t)(1 * r + j) * n + k], as[k], q);
    }
    free(spoly); free(as);
}

/* ------------------------------------------------------------------ */
/* Gadget decomposition (the inverse of G in EncRGSW, Section 2.4).     */
/* For source prime i the residue x_i is centred into (-q_i/2, q_i/2]   */
/* and split into dpp signed base-beta digits in [-beta/2, beta/2),     */
/* least significant first; the last digit keeps the remaining carry.   */
/* With log_beta = 0 the single digit is the centred residue itself.    */
/* Digit rho = i*dpp + k of every coefficient, lifted to each prime j.  */
/* ------------------------------------------------------------------ */
static void decompose(const or_ctx *c, const u64 *comp_res /* [r][N] */, int rho,
                      u64 *digit /* [r][N] */) {
    int n = c->n, i = rho / c->dpp, k = rho % c->dpp;
    u64 qi = c->q[i];
    for (int x = 0; x < n; x++) {
        u64 v = comp_res[(size_t)i * n + x];
        long long cen = v > (qi - 1) / 2 ? (long long)v - (long long)qi : (long long)v;
        long long d = cen;
        if (c->log_beta) {
            long long beta = 1LL << c->log_beta, half = beta / 2;
            for (int t = 0; t <= k; t++) {
                if (t == c->dpp - 1) { d = cen; break; }
                long long m = cen % beta;
                if (m < 0) m += beta;
                if (m >= half) m -= beta;
                d = m;
                cen = (cen - m) / beta;
            }
        }
        for (int j = 0; j < c->r; j++) digit[(size_t)j * n + x] = from_signed(d, c->q[j]);
    }
}

/* Exported for the recomposition test: digit rho of one component. */
void or_decompose(const or_ctx *c, const u64 *comp_res, int rho, u64 *digit) {
    decompose(c, comp_res, rho, digit);
}

/* ------------------------------------------------------------------ */
/* PackingKeySwitching (Section 2.4).  Key: for every LWE key coefficient */
/* x < N and gadget row rho < dnum (row = x*dnum + rho), an RLWE         */
/* (a, a*s + e + s_x * g_rho) with g_rho the gadget value at prime       */
/* rho / dpp (0 at the others); a from TAG_KSK_A (two words per          */
/* coefficient, counter (k>>1, row*r + j, 0)), e from TAG_KSK_E (counter */
/* (k>>2, row, 0)).  Stored in coefficient form, rows in order.          */
/* ------------------------------------------------------------------ */
void or_ksk_gen(const or_ctx *c, const int8_t *s, u64 seed, int trivial, u64 *ksk) {
    int n = c->n, r = c->r;
    size_t rlwe = or_rlwe_words(c);
    u64 *spoly = (u64 *)malloc(sizeof(u64) * n);
    long long *e = (long long *)malloc(sizeof(long long) * n);
    for (int x = 0; x < n; x++) {
        for (int rho = 0; rho < c->dnum; rho++) {
            const u64 row = (u64)x * c->dnum + rho;
            int gi = rho / c->dpp, gk = rho % c->dpp;
            for (int k = 0; k < n; k++) {
                u64 w[4];
                draw(seed, TAG_KSK_E, (u64)k >> 2, row, 0, w);
                e[k] = trivial ? 0 : gaussian(c, w[k & 3]);
            }
            u64 *out = ksk + row * rlwe;
            for (int j = 0; j < r; j++) {
                u64 q = c->q[j];
                u64 *a = out + (size_t)(0 * r + j) * n, *b = out + (size_t)(1 * r + j) * n;
                for (int k = 0; k < n; k++) spoly[k] = from_signed(s[k], q);
                for (int k = 0; k < n; k++) {
                    u64 w[4];
                    draw(seed, TAG_KSK_A, (u64)k >> 1, row * r + j, 0, w);
                    u64 hi = w[2 * (k & 1)], lo = w[2 * (k & 1) + 1];
                    a[k] = trivial ? 0 : (u64)((((u128)hi << 64) | lo) % q);
                }
                or_poly_mul(a, spoly, b, c->log_n, q, c->psi[j]);
                for (int k = 0; k < n; k++) b[k] = addmod(b[k], from_signed(e[k], q), q);
                if (j == gi) {
                    u64 g = c->log_beta ? powmod((u64)1 << c->log_beta, (u64)gk, q) : 1;
                    b[0] = addmod(b[0], mulmod(from_signed(s[x], q), g, q), q);
                }
            }
        }
    }
    free(spoly); free(e);
}

/* Packing of k <= N LWE ciphertexts (each [prime][N a', then b']) into one
 * RLWE encrypting sum_i m_i X^i:
 *   C = sum_i X^i (0, b_i) - sum_{x, rho} KSK_{x,rho} * D_{x,rho}(X),
 *   D_{x,rho}(X) = sum_i Dec_rho(a'_{i,x}) X^i, digits lifted to every prime. */
void or_pack_keyswitch(const or_ctx *c, const u64 *ksk, const u64 *lwes, int k, u64 *out) {
    int n = c->n, r = c->r;
    size_t rlwe = or_rlwe_words(c), lw = (size_t)r * (n + 1);
    u64 *A = (u64 *)malloc(sizeof(u64) * (size_t)r * n);
    u64 *D = (u64 *)malloc(sizeof(u64) * (size_t)r * n);
    u64 *t = (u64 *)malloc(sizeof(u64) * n);
    memset(out, 0, sizeof(u64) * rlwe);
    for (int i = 0; i < k; i++)
        for (int j = 0; j < r; j++) out[(size_t)(r + j) * n + i] = lwes[i * lw + (size_t)j * (n + 1) + n];
    for (int x = 0; x < n; x++) {
        memset(A, 0, sizeof(u64) * (size_t)r * n);
        for (int i = 0; i < k; i++)
            for (int j = 0; j < r; j++) A[(size_t)j * n + i] = lwes[i * lw + (size_t)j * (n + 1) + x];
        for (int rho = 0; rho < c->dnum; rho++) {
            decompose(c, A, rho, D);
            const u64 *row = ksk + ((size_t)x * c->dnum + rho) * rlwe;
            for (int comp = 0; comp < 2; comp++)
                for (int j = 0; j < r; j++) {
                    u64 q = c->q[j];
                    or_poly_mul(row + (size_t)(comp * r + j) * n, D + (size_t)j * n, t, c->log_n, q, c->psi[j]);
                    u64 *o = out + (size_t)(comp * r + j) * n;
                    for (int y = 0; y < n; y++) o[y] = submod(o[y], t[y], q);
                }
        }
    }
    free(A); free(D); free(t);
}

/* External product C [x] c (Section 2.4): sum over gadget rows of
 * Dec(b)_rho * row_rho + Dec(a)_rho * row_{dnum+rho}; each ring product is
 * taken through the transform, summed in evaluation form, then inverted. */
void or_ext_product(const or_ctx *c, const u64 *rgsw_ntt, const u64 *in, u64 *out) {
    int n = c->n, r = c->r;
    size_t rlwe = or_rlwe_words(c);
    u64 *acc = (u64 *)calloc(rlwe, sizeof(u64));
    u64 *dig = (u64 *)malloc(sizeof(u64) * (size_t)r * n);
    for (int src = 0; src < 2; src++) {           /* 0: a, 1: b */
        const u64 *comp = in + (size_t)src * r * n;
        for (int rho = 0; rho < c->dnum; rho++) {
            int row = src == 1 ? rho : c->dnum + rho;
            decompose(c, comp, rho, dig);
            for (int j = 0; j < r; j++) {
                u64 q = c->q[j];
                u64 *dj = dig + (size_t)j * n;
                or_ntt_fwd(dj, c->log_n, q, c->psi[j]);
                for (int oc = 0; oc < 2; oc++) {
                    const u64 *rw = rgsw_ntt + (size_t)row * rlwe + (size_t)(oc * r + j) * n;
                    u64 *dst = acc + (size_t)(oc * r + j) * n;
                    for (int x = 0; x < n; x++) dst[x] = addmod(dst[x], mulmod(dj[x], rw[x], q), q);
                }
            }
        }
    }
    for (int oc = 0; oc < 2; oc++)
        for (int j = 0; j < r; j++) or_ntt_inv(acc + (size_t)(oc * r + j) * n, c->log_n, c->q[j], c->psi[j]);
    memcpy(out, acc, sizeof(u64) * rlwe);
    free(acc);
    free(dig);
}

/* CMUX(C, c1, c0) = c0 + C [x] (c1 - c0): selects c1 when C encrypts 1. */
void or_cmux(const or_ctx *c, const u64 *rgsw_ntt, const u64 *c1, const u64 *c0, u64 *out) {
    size_t rlwe = or_rlwe_words(c);
    u64 *d = (u64 *)malloc(sizeof(u64) * rlwe), *t = (u64 *)malloc(sizeof(u64) * rlwe);
    memcpy(d, c1, sizeof(u64) * rlwe);
    or_rlwe_sub(c, d, c0);
    or_ext_product(c, rgsw_ntt, d, t);
    if (out != c0) memcpy(out, c0, sizeof(u64) * rlwe);
    or_rlwe_add(c, out, t);
    free(d);
    free(t);
}

/* BlindRotate (Section 2.4) with weights I_t = sign * 2^t over the given
 * bits, in list order: acc <- CMUX(C_t, acc * X^(-I_t), acc).  A bit given
 * in clear (rgsw[t] == NULL) rotates exactly when it is 1 and is skipped
 * when it is 0.  sign = +1 is the VP direction (X^-2^t), sign = -1 the IVP
 * direction (X^+2^t). */
void or_blind_rotate(const or_ctx *c, u64 *acc, const u64 *const *rgsw, const int *clear,
                     int nbits, int sign) {
    size_t rlwe = or_rlwe_words(c);
    u64 *rot = (u64 *)malloc(sizeof(u64) * rlwe);
    for (int t = 0; t < nbits; t++) {
        long long e = -(long long)sign * (1LL << t);
        if (rgsw[t] == NULL) {
            if (clear[t]) {
                or_rlwe_rotate(c, acc, e, rot);
                memcpy(acc, rot, sizeof(u64) * rlwe);
            }
            continue;
        }
        or_rlwe_rotate(c, acc, e, rot);
        or_cmux(c, rgsw[t], rot, acc, acc);
    }
    free(rot);
}

/* ExtractLWE(c, 0): a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0, per prime; the
 * LWE is stored as [prime][N a-coefficients, then b]. */
void or_extract_lwe0(const or_ctx *c, const u64 *ct, u64 *lwe) {
    int n = c->n;
    for (int j = 0; j < c->r; j++) {
        const u64 *a = ct + (size_t)(0 * c->r + j) * n, *b = ct + (size_t)(1 * c->r + j) * n;
        u64 *dst = lwe + (size_t)j * (n + 1);
        dst[0] = a[0];
        for (int x = 1; x < n; x++) dst[x] = negmod(a[n - x], c->q[j]);
        dst[n] = b[0];
    }
}

/* Phase b' - <a', s> of an LWE, per prime. */
void or_lwe_phase(const or_ctx *c, const int8_t *s, const u64 *lwe, u64 *phase) {
    int n = c->n;
    for (int j = 0; j < c->r; j++) {
        u64 q = c->q[j], acc = 0;
        const u64 *src = lwe + (size_t)j * (n + 1);
        for (int x = 0; x < n; x++) acc = addmod(acc, mulmod(src[x], from_signed(s[x], q), q), q);
        phase[j] = submod(src[n], acc, q);
    }
}

void or_lwe_add(const or_ctx *c, u64 *acc, const u64 *x) {
    for (int j = 0; j < c->r; j++)
        for (int t = 0; t <= c->n; t++) {
            size_t o = (size_t)j * (c->n + 1) + t;
            acc[o] = addmod(acc[o], x[o], c->q[j]);
        }
}

/* ------------------------------------------------------------------ */
/* CDEMUX gate and Inverse Vertical Packing (Section 3.3, Algorithm 5). */
/* ------------------------------------------------------------------ */

/* CDEMUX(C, d) = (d - C [x] d, C [x] d): d is replaced by its first output,
 * the second output is written to hi. */
void or_cdemux(const or_ctx *c, const u64 *rgsw_ntt, u64 *d, u64 *hi) {
    or_ext_product(c, rgsw_ntt, d, hi);
    or_rlwe_sub(c, d, hi);
}

/* IVP over k bits b_0..b_{k-1} (NULL rgsw = bit given in clear): blind
 * rotation of lhat by bits b_z..b_{k-1} with weights -2^0, -2^1, ...,
 * then the CDEMUX tree over b_0..b_{z-1}: level i (offset n = 2^i) splits
 * L_j into (L_j, L_{j+n}) for j in [0, n).  gate[i * 2^(z-1) + j] says
 * whether the gate is evaluated; a gate that is not evaluated leaves L_j in
 * place.  L must hold 2^z RLWE buffers; they are overwritten. */
void or_ivp(const or_ctx *c, const u64 *lhat, const u64 *const *rgsw, const int *clear, int k,
            int z, const uint8_t *gate, u64 *L) {
    size_t rlwe = or_rlwe_words(c);
    int nl = 1 << z;
    memset(L, 0, sizeof(u64) * rlwe * nl);
    memcpy(L, lhat, sizeof(u64) * rlwe);
    or_blind_rotate(c, L, rgsw + z, clear + z, k - z, -1);
    int half = nl / 2 > 0 ? nl / 2 : 1;
    for (int i = 0; i < z; i++) {
        int n = 1 << i;
        for (int j = 0; j < n; j++) {
            if (!gate[i * half + j]) continue;
            u64 *lo = L + (size_t)j * rlwe, *hi = L + (size_t)(j + n) * rlwe;
            if (rgsw[i] != NULL) {
                or_cdemux(c, rgsw[i], lo, hi);
            } else if (clear[i]) {
                memcpy(hi, lo, sizeof(u64) * rlwe);
                memset(lo, 0, sizeof(u64) * rlwe);
            } else {
                memset(hi, 0, sizeof(u64) * rlwe);
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Vertical Packing (Section 2.4.2, Algorithm 3).                       */
/* ------------------------------------------------------------------ */

/* VP over k bits: CMUX tree on b_0..b_{z-1} starting from the largest
 * offset (n = 2^(z-1), control b_{log2 n}), L_j <- CMUX(b, L_{j+n}, L_j) for
 * j in [0, n); then blind rotation of L_0 by b_z..b_{k-1} with weights
 * +2^0, +2^1, ...; then ExtractLWE(., 0).  Lin holds 2^z RLWE pointers,
 * NULL meaning an all-zero ciphertext. */
/* The accumulator of VP before ExtractLWE: the tree, then BlindRotate over
 * bits z..k-1 (clear bits rotate exactly or are skipped); used by horizontal
 * packing, which extracts several coefficients of one accumulator. */
void or_vp_rlwe(const or_ctx *c, const u64 *const *Lin, const u64 *const *rgsw, const int *clear,
                int k, int z, u64 *out) {
    size_t rlwe = or_rlwe_words(c);
    int nl = 1 << z;
    u64 *L = (u64 *)calloc(rlwe * nl, sizeof(u64));
    for (int v = 0; v < nl; v++)
        if (Lin[v]) memcpy(L + (size_t)v * rlwe, Lin[v], sizeof(u64) * rlwe);
    for (int lvl = z - 1; lvl >= 0; lvl--) {
        int n = 1 << lvl;
        for (int j = 0; j < n; j++) {
            u64 *lo = L + (size_t)j * rlwe, *hi = L + (size_t)(j + n) * rlwe;
            if (rgsw[lvl] != NULL) or_cmux(c, rgsw[lvl], hi, lo, lo);
            else if (clear[lvl]) memcpy(lo, hi, sizeof(u64) * rlwe);
        }
    }
    or_blind_rotate(c, L, rgsw + z, clear + z, k - z, +1);
    memcpy(out, L, sizeof(u64) * rlwe);
    free(L);
}

void or_vp(const or_ctx *c, const u64 *const *Lin, const u64 *const *rgsw, const int *clear,
           int k, int z, u64 *lwe) {
    size_t rlwe = or_rlwe_words(c);
    int nl = 1 << z;
    u64 *L = (u64 *)calloc(rlwe * nl, sizeof(u64));
    for (int v = 0; v < nl; v++)
        if (Lin[v]) memcpy(L + (size_t)v * rlwe, Lin[v], sizeof(u64) * rlwe);
    for (int lvl = z - 1; lvl >= 0; lvl--) {
        int n = 1 << lvl;
        for (int j = 0; j < n; j++) {
            u64 *lo = L + (size_t)j * rlwe, *hi = L + (size_t)(j + n) * rlwe;
            if (rgsw[lvl] != NULL) or_cmux(c, rgsw[lvl], hi, lo, lo);
            else if (clear[lvl]) memcpy(lo, hi, sizeof(u64) * rlwe);
        }
    }
    or_blind_rotate(c, L, rgsw + z, clear + z, k - z, +1);
    or_extract_lwe0(c, L, lwe);
    free(L);
}
