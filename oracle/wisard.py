"""Plain (unencrypted) WiSARD pieces of the oracle.  TEST INFRASTRUCTURE ONLY.

* client pre-processing: linear quantisation (Section 2.3.1), thermometer
  encoding T_T (Section 2.3.2), the bit permutation pi_r of Definition 1 and,
  for hashed workloads, an H3 hash of each tuple (a client-side,
  dataset-independent pre-processing step as Section 3.4 allows);
* the Integer WiSARD of Algorithm 4 and the evaluation of Algorithm 2;
* the activations of Section 3.2 and post-decryption activation (PD-act,
  Section 3.5.1): activate each decrypted RAM response, add per class,
  arg-max with ties going to the lowest class index.
"""
import ctypes

import numpy as np

from ._lib import lib, u64p

TAG_PERM = 4
TAG_H3 = 5


def _philox(seed: int, tag: int, c0: int):
    ctr = (ctypes.c_uint64 * 4)(c0, 0, 0, 0)
    key = (ctypes.c_uint64 * 2)(seed, tag)
    out = (ctypes.c_uint64 * 4)()
    lib().or_philox(ctypes.cast(ctr, u64p), ctypes.cast(key, u64p), ctypes.cast(out, u64p))
    return [int(v) for v in out]


def permutation(model_seed: int, s: int) -> np.ndarray:
    """pi_r as an index table: t_p = T_{perm[p]}.  Fisher-Yates from the top:
    for j = s-1 down to 1 swap perm[j] with perm[w_j mod (j+1)], where w_j is
    word j of the PERM stream."""
    perm = list(range(s))
    for j in range(s - 1, 0, -1):
        w = _philox(model_seed, TAG_PERM, j >> 2)[j & 3]
        k = w % (j + 1)
        perm[j], perm[k] = perm[k], perm[j]
    return np.array(perm, dtype=np.int64)


def h3_matrix(model_seed: int, tuple_bits: int, addr_bits: int) -> np.ndarray:
    """Row i of the H3 matrix: the low addr_bits bits of word i of the H3
    stream."""
    rows = []
    for i in range(tuple_bits):
        w = _philox(model_seed, TAG_H3, i >> 2)[i & 3]
        rows.append(w & ((1 << addr_bits) - 1))
    return np.array(rows, dtype=np.int64)


def quantize(values: np.ndarray, T: int) -> np.ndarray:
    """Linear quantisation f_r(x) = floor(x / r) with r = 256 / (T+1), which
    maps a byte to a level in 0..T; computed as (v * (T+1)) >> 8."""
    return (values.astype(np.int64) * (T + 1)) >> 8


def thermometer_levels(level: np.ndarray, T: int) -> np.ndarray:
    """T_T of each level: bit i is 1 iff i < level (Section 2.3.2)."""
    level = np.asarray(level, dtype=np.int64)
    return (np.arange(T) < level[..., None]).astype(np.uint8)


def thermometer(values: np.ndarray, T: int) -> np.ndarray:
    """Quantise, then thermometer-encode; bits of value f sit at f*T + i."""
    bits = thermometer_levels(quantize(values, T), T)
    return bits.reshape(values.shape[0], -1)


def h3_hash(tuples: np.ndarray, Hm: np.ndarray) -> np.ndarray:
    """H3 hash of each row of `tuples` (n, tuple_bits) of 0/1 bits:
    h(x) = XOR of the matrix rows Hm[i] whose bit x_i is 1."""
    n = tuples.shape[0]
    h = np.zeros(n, dtype=np.int64)
    for i in range(tuples.shape[1]):
        h ^= np.where(tuples[:, i] == 1, int(Hm[i]), 0)
    return h


def encode(P, values: np.ndarray, perm=None, h3=None) -> np.ndarray:
    """Data bits the client encrypts, shape (n, n_data).  Plain workloads
    send the thermometer bits in their original order (the server applies
    pi_r); hashed workloads apply pi_r, cut a tuple of tuple_bits per RAM
    and send its addr_bits hash, h(x) = XOR of H3 rows i with x_i = 1, hash
    bit i as the RAM's address bit i.  perm / h3 replace the seeded pi_r /
    H3 matrix (worked examples)."""
    cfg = P.cfg
    tb = thermometer(values, cfg.therm_bits)
    if not cfg.hash_h3:
        return tb
    if perm is None:
        perm = permutation(cfg.model_seed, P.s)
    t = tb[:, perm]
    Hm = h3_matrix(cfg.model_seed, cfg.tuple_bits, P.a) if h3 is None else np.asarray(h3, dtype=np.int64)
    n = values.shape[0]
    out = np.zeros((n, P.k0 * P.a), dtype=np.uint8)
    for j in range(P.k0):
        lo = j * cfg.tuple_bits
        h = h3_hash(t[:, lo:lo + cfg.tuple_bits], Hm)
        for i in range(P.a):
            out[:, j * P.a + i] = (h >> i) & 1
    return out


def ram_bits(P, perm=None) -> np.ndarray:
    """For RAM j and address bit i, the index of the data bit it reads, or -1
    for the constant-0 bits that pad a short last tuple.  The tuple of RAM j
    is t_{ja} .. t_{ja+a-1} of the permuted input t_p = T_{perm[p]}
    (Definition 1, f_comp); perm defaults to the seeded pi_r."""
    cfg = P.cfg
    tab = np.full((P.k0, P.a), -1, dtype=np.int64)
    if cfg.hash_h3:
        for j in range(P.k0):
            tab[j] = j * P.a + np.arange(P.a)
        return tab
    if perm is None:
        perm = permutation(cfg.model_seed, P.s)
    for j in range(P.k0):
        for i in range(P.a):
            idx = j * P.a + i
            if idx < P.s:
                tab[j, i] = perm[idx]
    return tab


def addresses(P, data_bits: np.ndarray, perm=None) -> np.ndarray:
    """f_comp for every RAM: address = sum_i bit_i 2^i, shape (n, k0)."""
    tab = ram_bits(P, perm)
    n = data_bits.shape[0]
    addr = np.zeros((n, P.k0), dtype=np.int64)
    for i in range(P.a):
        col = tab[:, i]
        valid = col >= 0
        bits = np.zeros((n, P.k0), dtype=np.int64)
        bits[:, valid] = data_bits[:, col[valid]]
        addr |= bits << i
    return addr


def integer_wisard_train(P, data_bits, labels, perm=None) -> np.ndarray:
    """Algorithm 4: W[L_i][j][f_comp(t, j)] += 1; W has shape (l, k0, 2^a)."""
    W = np.zeros((P.cfg.n_classes, P.k0, 1 << P.a), dtype=np.int64)
    addr = addresses(P, data_bits, perm)
    for i in range(data_bits.shape[0]):
        W[labels[i], np.arange(P.k0), addr[i]] += 1
    return W


def lookups(P, W, data_bits) -> np.ndarray:
    """u[i][c][j] = W[c][j][f_comp(t_i, j)], shape (n, l, k0)."""
    addr = addresses(P, data_bits)
    n = data_bits.shape[0]
    out = np.zeros((n, P.cfg.n_classes, P.k0), dtype=np.int64)
    for i in range(n):
        out[i] = W[:, np.arange(P.k0), addr[i]]
    return out


def bitlen(x):
    """Number of binary digits of x >= 0 (0 for x = 0)."""
    x = np.asarray(x, dtype=np.int64)
    out = np.zeros_like(x)
    v = x.copy()
    while np.any(v > 0):
        out += (v > 0)
        v >>= 1
    return out


def log_act(x):
    """floor(log2(x + 1)) for counters x >= 0: the integer reading of the log
    activation f(x) = log2(x + 1) (Section 3.2), floored as the paper's
    logarithmic quantiser floor(log_b(x + 1)) is (Section 2.3.1)."""
    return bitlen(np.asarray(x, dtype=np.int64) + 1) - 1


def activate(cfg, u):
    u = np.asarray(u, dtype=np.int64)
    if cfg.act == "log":
        return log_act(u)
    if cfg.act == "blog":
        return np.minimum(log_act(u), cfg.act_arg)
    if cfg.act == "bin":
        return (u > cfg.act_arg).astype(np.int64)
    raise ValueError(cfg.act)


def pdact(cfg, u):
    """PD-act on decrypted responses u (n, l, k0): scores and labels."""
    scores = activate(cfg, u).sum(axis=2)
    labels = np.argmax(scores, axis=1).astype(np.int64)  # first maximum wins
    return scores, labels


def balanced_pdact(cfg, u, class_counts):
    """PD-act with the dataset-balancing rescale of Section 3.6.1.  The
    paper leaves the rule open; reading: a per-class learning rate
    n_ref / n_c (n_ref = the largest class count), applied to the decrypted
    counters before the activation with floor division,
    u'[i][c][j] = floor(u[i][c][j] * n_ref / n_c) (u' = u where n_c = 0,
    whose counters are all 0).  It equals training on a set where every
    class is repeated up to n_ref samples."""
    u = np.asarray(u, dtype=np.int64)
    n = np.asarray(class_counts, dtype=np.int64)
    n_ref = int(n.max()) if n.size else 0
    scaled = u.copy()
    for c in range(u.shape[1]):
        if n[c] > 0:
            scaled[:, c, :] = (u[:, c, :] * n_ref) // n[c]
    return pdact(cfg, scaled)


def evaluate(P, W, data_bits):
    """Algorithm 2 with the activation applied to the looked-up counters."""
    return pdact(P.cfg, lookups(P, W, data_bits))
