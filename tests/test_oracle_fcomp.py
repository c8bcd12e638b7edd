"""Pins of the oracle's tuple map and H3 hash, against hand-worked cases.

* Definition 1 (Section 2.2): f_comp(x, d) = sum over i < min(a, s - a d) of
  x_{i + a d} 2^i on the permuted input t_p = T_{pi(p)}, k = ceil(s / a)
  RAMs; a short last tuple reads its real bits and constant 0s.  The case
  s = 5, a = 2 tells bit weight 2^i from 2^(a-1-i), the disjoint tuples of
  Definition 1 from the overlapping windows of Algorithms 6 and 7, and the
  permutation from its inverse.
* Figure 1 (Section 2.2): the figure's permutation arrows, routed through
  wisard.addresses, give the highlighted RAM rows and the score.
* H3 (the hashed addressing of the at-scale digit workload): a fixed 4 x 3
  matrix and hand-computed XORs, which tell row i from row a-1-i; the
  encoder's hashed branch puts hash bit i at address bit i.
* The seeded H3 matrix and the permutation's stream are words of numpy's
  Philox4x64-10 (an implementation independent of the oracle's C code).
"""
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import wisard

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


def _plain_P(s, a, n_classes=2, model_seed=0):
    cfg = SimpleNamespace(hash_h3=0, model_seed=model_seed, n_classes=n_classes)
    return SimpleNamespace(cfg=cfg, s=s, a=a, k0=-(-s // a))


def test_definition1_tuple_table():
    ex = GOLDEN["def1_fcomp_short_tuple"]
    P = _plain_P(ex["s"], ex["a"])
    assert P.k0 == 3
    tab = wisard.ram_bits(P, perm=np.array(ex["permutation"]))
    assert tab.tolist() == ex["ram_bits"]


def test_definition1_addresses():
    ex = GOLDEN["def1_fcomp_short_tuple"]
    P = _plain_P(ex["s"], ex["a"])
    x = np.array([ex["input"]], dtype=np.uint8)
    perm = np.array(ex["permutation"])
    assert x[0, perm].tolist() == ex["permuted"]
    addr = wisard.addresses(P, x, perm=perm)
    assert addr[0].tolist() == ex["addresses"]
    # every misreading the case was built against gives other addresses
    for name, wrong in ex["misreadings"].items():
        assert wrong != ex["addresses"], name


def test_definition1_misreadings_are_detected():
    """The hand values of the misreadings follow from their own formulas, so
    an oracle that implemented one of them would fail the test above."""
    ex = GOLDEN["def1_fcomp_short_tuple"]
    s, a = ex["s"], ex["a"]
    T = ex["input"]
    perm = ex["permutation"]
    t = [T[perm[p]] for p in range(s)]
    k = -(-s // a)

    def bit(v, i):
        return v[i] if i < s else 0
    rev = [sum(bit(t, d * a + i) << (a - 1 - i) for i in range(a)) for d in range(k)]
    over = [sum(bit(t, d + i) << i for i in range(a)) for d in range(k)]
    inv = [0] * s
    for p in range(s):
        inv[perm[p]] = p
    ti = [T[inv[p]] for p in range(s)]
    inverse = [sum(bit(ti, d * a + i) << i for i in range(a)) for d in range(k)]
    ident = [sum(bit(T, d * a + i) << i for i in range(a)) for d in range(k)]
    m = ex["misreadings"]
    assert rev == m["weights_2^(a-1-i)"]
    assert over == m["overlapping_windows_t_j..t_j+a-1"]
    assert inverse == m["inverse_permutation"]
    assert ident == m["no_permutation"]


def test_definition1_training_counts():
    """Algorithm 4 on two hand-worked samples: W[L_i][j][f_comp(t, j)] = 1."""
    ex = GOLDEN["def1_fcomp_short_tuple"]
    P = _plain_P(ex["s"], ex["a"])
    tr = ex["train"]
    x = np.array(tr["inputs"], dtype=np.uint8)
    W = wisard.integer_wisard_train(P, x, np.array(tr["labels"]), perm=np.array(ex["permutation"]))
    assert W.tolist() == tr["counts"]


def test_figure1_through_addresses():
    """Figure 1: input 1010, the drawn permutation, RAM rows 01 and 10
    highlighted, score 1 with the binary activation."""
    ex = GOLDEN["fig1_wisard_evaluation"]
    a = 2
    P = _plain_P(len(ex["input"]), a, n_classes=1)
    perm = np.array(ex["permutation"])
    x = np.array([ex["input"]], dtype=np.uint8)
    assert x[0, perm].tolist() == ex["permuted_address"]
    addr = wisard.addresses(P, x, perm=perm)[0]
    assert addr.tolist() == ex["addresses"]
    W = np.zeros((1, len(ex["rams"]), 1 << a), dtype=np.int64)
    for j, ram in enumerate(ex["rams"]):
        for lab, val in zip(ex["labels"], ram):
            W[0, j, sum(int(ch) << i for i, ch in enumerate(lab))] = val
    u = W[0, np.arange(len(ex["rams"])), addr]
    act = SimpleNamespace(act=ex["activation"]["act"], act_arg=ex["activation"]["thr"])
    assert int(wisard.activate(act, u).sum()) == ex["score"]


def test_h3_hand_hashes():
    ex = GOLDEN["h3_hand"]
    h = wisard.h3_hash(np.array(ex["tuples"]), np.array(ex["matrix"]))
    assert h.tolist() == ex["hashes"]
    assert ex["misreadings"]["rows_reversed"] != ex["hashes"]
    hr = wisard.h3_hash(np.array(ex["tuples"]), np.array(ex["matrix"][::-1]))
    assert hr.tolist() == ex["misreadings"]["rows_reversed"]


def test_h3_encode_bit_layout():
    ex = GOLDEN["h3_hand"]
    e = ex["encode"]
    vals = np.array([e["values"]], dtype=np.uint8)
    s = len(e["values"]) * e["therm_bits"]
    a = ex["addr_bits"]
    cfg = SimpleNamespace(hash_h3=1, model_seed=0, therm_bits=e["therm_bits"], tuple_bits=e["tuple_bits"])
    P = SimpleNamespace(cfg=cfg, s=s, a=a, k0=-(-s // e["tuple_bits"]))
    out = wisard.encode(P, vals, perm=np.array(e["permutation"]), h3=np.array(ex["matrix"]))
    assert out[0].tolist() == e["bits"]


def _numpy_philox_words(seed, tag, c0):
    """Words of counter (c0, 0, 0, 0), key (seed, tag) from numpy's Philox
    (which increments its 256-bit counter before each block)."""
    m = (1 << 64) - 1
    ctr = [c0 - 1, 0, 0, 0] if c0 > 0 else [m, m, m, m]
    return [int(v) for v in np.random.Philox(counter=ctr, key=[seed, tag]).random_raw(4)]


@pytest.mark.parametrize("seed", [0, 7, 2**40 + 3])
def test_h3_matrix_rows_are_stream_words(seed):
    rows = wisard.h3_matrix(seed, 16, 12)
    for i in range(16):
        w = _numpy_philox_words(seed, wisard.TAG_H3, i >> 2)[i & 3]
        assert int(rows[i]) == w & 0xFFF


def test_permutation_follows_fisher_yates_on_stream_words():
    seed, s = 11, 37
    perm = list(range(s))
    for j in range(s - 1, 0, -1):
        w = _numpy_philox_words(seed, wisard.TAG_PERM, j >> 2)[j & 3]
        k = w % (j + 1)
        perm[j], perm[k] = perm[k], perm[j]
    assert wisard.permutation(seed, s).tolist() == perm
