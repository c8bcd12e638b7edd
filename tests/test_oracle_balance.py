"""Dataset balancing (Section 3.6.1) in the oracle.

Pins: the class-count ciphertext decrypts to the class histogram (a closed
form); balanced PD-act reduces to PD-act when the classes are balanced and is
unchanged when every count is scaled by the same factor; and it equals plain
Integer WiSARD trained on the set where each minority class is repeated up to
the majority's count (the learning-rate reading of the rescale)."""
import numpy as np

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset

TINY = dict(log_n=6, n_primes=2, prime_bits=50, log_beta=0, log_p=16, n_classes=3,
            n_values=7, therm_bits=2, addr_bits=6, tuple_bits=6, data_kind="uniform",
            act="log", act_arg=0)


def _decrypt_counts(o, s, C):
    vals = o.decrypt_rlwe(s, C)
    return np.asarray(vals, dtype=np.int64).reshape(-1)


def test_count_ciphertext_decrypts_to_the_histogram():
    cfg = get_config("cfg1", **TINY)
    o = Oracle(cfg)
    s = o.keygen(3)
    labels = np.array([0, 2, 2, 1, 2, 0, 2], dtype=np.int64)
    C = o.count_classes(np.zeros(o.rlwe_words, dtype=np.uint64), s, 17, labels)
    dec = _decrypt_counts(o, s, C)
    assert list(dec[:3]) == list(np.bincount(labels, minlength=3))
    assert not dec[3:].any()


def test_balanced_pdact_special_cases():
    cfg = get_config("cfg1", **TINY)
    rng = np.random.default_rng(4)
    u = rng.integers(0, 40, size=(5, 3, 9))
    s0, l0 = wisard.pdact(cfg, u)
    s1, l1 = wisard.balanced_pdact(cfg, u, [6, 6, 6])
    assert np.array_equal(s0, s1) and np.array_equal(l0, l1)
    a = wisard.balanced_pdact(cfg, u, [3, 5, 2])
    b = wisard.balanced_pdact(cfg, u, [21, 35, 14])
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_balanced_pdact_equals_training_on_the_repeated_set():
    cfg = get_config("cfg1", **TINY)
    P = Oracle(cfg).P
    vals, _ = make_dataset(cfg, "train", n=8)
    labels = np.array([0, 0, 0, 0, 1, 1, 2, 2], dtype=np.int64)  # counts 4, 2, 2
    bits = wisard.encode(P, vals)
    tvals, _ = make_dataset(cfg, "test", n=6)
    tbits = wisard.encode(P, tvals)
    W = wisard.integer_wisard_train(P, bits, labels)
    bal = wisard.balanced_pdact(cfg, wisard.lookups(P, W, tbits), np.bincount(labels, minlength=3))
    # repeat the minority samples until every class has 4
    rep_bits = np.concatenate([bits, bits[4:], ])
    rep_labels = np.concatenate([labels, labels[4:]])
    W2 = wisard.integer_wisard_train(P, rep_bits, rep_labels)
    plain = wisard.evaluate(P, W2, tbits)
    assert np.array_equal(bal[0], plain[0]) and np.array_equal(bal[1], plain[1])
