"""Pins of the oracle's WiSARD layer:

* the paper's worked examples (Figures 1 and 2, the T_4 examples);
* linear quantisation against floor(x / r) with exact rationals;
* the homomorphic training invariant: decrypted counters equal the Integer
  WiSARD counts of Algorithm 4 exactly, for every tree shape the workloads
  use (z = 0, z <= L, z > L, hashed tuples, a short last tuple);
* inference: decrypted responses equal the plaintext lookups, per-class sums
  equal the Algorithm 2 scores, PD-act labels equal the plaintext labels;
* brute force over every input of a tiny configuration;
* the federated merge (Section 3.6.2): shards added equal central training,
  bit for bit;
* noise-free exactness of the whole pipeline (trivial encryptions).
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")))


class _Act:
    def __init__(self, act, thr):
        self.act, self.act_arg = act, thr


@pytest.mark.parametrize("name", ["fig1_wisard_evaluation", "fig2a_binary_discriminator",
                                  "fig2b_bleaching_discriminator"])
def test_worked_example_scores(name):
    ex = GOLDEN[name]
    a = 2
    # rows are printed under bit-string labels x_0 x_1; f_comp index = x_0 + 2 x_1
    W = np.zeros((1, len(ex["rams"]), 1 << a), dtype=np.int64)
    for j, ram in enumerate(ex["rams"]):
        for lab, val in zip(ex["labels"], ram):
            W[0, j, sum(int(ch) << i for i, ch in enumerate(lab))] = val
    t = ex["permuted_address"]
    u = [W[0, j, sum(t[j * a + i] << i for i in range(a))] for j in range(len(ex["rams"]))]
    act = _Act(ex["activation"]["act"], ex["activation"]["thr"])
    assert int(wisard.activate(act, np.array(u)).sum()) == ex["score"]


def test_worked_example_thermometer():
    for case in GOLDEN["thermometer"]["cases"]:
        assert list(wisard.thermometer_levels(np.array(case["x"]), case["N"])) == case["bits"]


@pytest.mark.parametrize("T", [1, 2, 3, 4, 8])
def test_quantisation_is_linear_floor(T):
    v = np.arange(256, dtype=np.uint8)
    r = Fraction(256, T + 1)
    expect = [int(Fraction(int(x)) // r) for x in v]
    assert list(wisard.quantize(v[None, :], T)[0]) == expect


def test_permutation_is_a_permutation():
    perm = wisard.permutation(7, 1568)
    assert sorted(perm.tolist()) == list(range(1568))
    assert not np.array_equal(perm, np.arange(1568))


def test_log_activation_is_floor_log2_x_plus_1():
    x = np.arange(0, 5000)
    expect = [int(np.floor(np.log2(v + 1))) for v in x]
    assert wisard.log_act(x).tolist() == expect
    assert wisard.bitlen(x).tolist() == [int(v).bit_length() for v in x]


# tiny configurations covering every tree shape of the workloads
TINY = {
    # z = 0 (cfg1-like): label bit is a rotation bit; base-32 gadget
    "z0": dict(log_n=5, n_primes=1, prime_bits=30, log_beta=5, log_p=8, n_classes=2,
               n_values=5, therm_bits=2, addr_bits=3, tuple_bits=3),
    # z = L (cfg2-like): the tree holds exactly the label bits; short last tuple
    "zL": dict(log_n=3, n_primes=2, prime_bits=50, log_beta=0, log_p=16, n_classes=3,
               n_values=5, therm_bits=2, addr_bits=3, tuple_bits=3),
    # z < L (cfg3-like): a label bit is a rotation bit; hashed tuples
    "zltL_h3": dict(log_n=3, n_primes=3, prime_bits=55, log_beta=0, log_p=20, n_classes=5,
                    n_values=4, therm_bits=3, addr_bits=2, tuple_bits=4, hash_h3=1),
    # z > L (cfg4-like): an address bit enters the tree; pruned gates
    "zgtL": dict(log_n=3, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3,
                 n_values=4, therm_bits=2, addr_bits=4, tuple_bits=4),
}


def tiny(name, **kw):
    d = dict(TINY[name])
    d.update(kw)
    return Oracle(get_config("cfg1", data_kind="uniform", act="log", act_arg=0, **d))


@pytest.mark.parametrize("name", list(TINY))
def test_structure_of_tiny_configs(name):
    o = tiny(name)
    P = o.P
    if name == "z0":
        assert P.z == 0
    elif name == "zL":
        assert P.z == P.L and P.s % P.a != 0
    elif name == "zltL_h3":
        assert 0 < P.z < P.L
    else:
        assert P.z > P.L and P.k1 < (1 << P.z)


@pytest.mark.parametrize("name", list(TINY))
def test_training_invariant_and_inference(name):
    o = tiny(name)
    P = o.P
    vals, labels = make_dataset(o.cfg, "train", n=9)
    bits = wisard.encode(P, vals)
    s = o.keygen(21)
    H = o.train(o.new_model(), s, 31, bits, labels)
    W = wisard.integer_wisard_train(P, bits, labels)
    assert np.array_equal(o.decrypt_model(s, H), W)
    tv, _ = make_dataset(o.cfg, "test", n=4)
    tb = wisard.encode(P, tv)
    resp, sums = o.infer(H, s, 41, tb)
    u = np.array([[[o.decrypt_lwe(s, resp[i, c, j]) for j in range(P.k0)]
                   for c in range(o.cfg.n_classes)] for i in range(4)])
    look = wisard.lookups(P, W, tb)
    assert np.array_equal(u, look)
    S = np.array([[o.decrypt_lwe(s, sums[i, c]) for c in range(o.cfg.n_classes)] for i in range(4)])
    assert np.array_equal(S, look.sum(axis=2))
    _, lab_enc = wisard.pdact(o.cfg, u)
    _, lab_plain = wisard.evaluate(P, W, tb)
    assert np.array_equal(lab_enc, lab_plain)


def test_brute_force_every_input():
    """Every input of a 2-value, 2-level configuration (9 inputs) is
    classified by encrypted inference exactly as by the plaintext model."""
    o = tiny("zL", n_values=2, addr_bits=2, tuple_bits=2, n_classes=3)
    P = o.P
    vals, labels = make_dataset(o.cfg, "train", n=12)
    bits = wisard.encode(P, vals)
    s = o.keygen(3)
    H = o.train(o.new_model(), s, 5, bits, labels)
    W = wisard.integer_wisard_train(P, bits, labels)
    grid = np.array([[a, b] for a in (0, 100, 200) for b in (0, 100, 200)], dtype=np.uint8)
    tb = wisard.encode(P, grid)
    assert len({tuple(r) for r in tb}) == 9
    resp, _ = o.infer(H, s, 7, tb)
    u = np.array([[[o.decrypt_lwe(s, resp[i, c, j]) for j in range(P.k0)]
                   for c in range(3)] for i in range(9)])
    assert np.array_equal(wisard.pdact(o.cfg, u)[1], wisard.evaluate(P, W, tb)[1])


def test_federated_merge_is_bit_identical():
    o = tiny("zgtL")
    vals, labels = make_dataset(o.cfg, "train", n=6)
    bits = wisard.encode(o.P, vals)
    s = o.keygen(2)
    central = o.train(o.new_model(), s, 9, bits, labels)
    a = o.train(o.new_model(), s, 9, bits[:4], labels[:4])
    b = o.train(o.new_model(), s, 9, bits[4:], labels[4:], sample_offset=4)
    from oracle._lib import lib, u64p
    for j in range(o.P.k0):
        for t in range(o.P.k1):
            lib().or_rlwe_add(o.ctx, a[j, t].ctypes.data_as(u64p), b[j, t].ctypes.data_as(u64p))
    assert np.array_equal(a, central)


@pytest.mark.parametrize("name", ["z0", "zgtL"])
def test_noise_free_pipeline_is_exact(name):
    """With trivial encryptions every model ciphertext is (0, Delta * counts)."""
    o = tiny(name)
    P = o.P
    vals, labels = make_dataset(o.cfg, "train", n=5)
    bits = wisard.encode(P, vals)
    s = o.keygen(1)
    H = o.train(o.new_model(), s, 1, bits, labels, trivial=True)
    W = wisard.integer_wisard_train(P, bits, labels)
    Hr = H.reshape(P.k0, P.k1, 2, P.r, P.n)
    assert not Hr[:, :, 0].any()
    for j in range(P.k0):
        for v in P.V:
            for x in range(P.n):
                m = v + (x << P.z)
                c, addr = m % (1 << P.L), m >> P.L
                cnt = int(W[c, j, addr]) if c < o.cfg.n_classes and addr < (1 << P.a) else 0
                for pj in range(P.r):
                    assert int(Hr[j, P.slot[v], 1, pj, x]) == (P.delta * cnt) % P.q[pj]


def test_full_config_parameters():
    """Derived sizes of the four workloads (k0, k1, z, gates)."""
    expect = {"cfg1": (30, 1, 0, 0), "cfg2": (131, 10, 4, 9), "cfg3": (147, 8, 3, 7),
              "cfg4": (504, 14, 4, 13)}
    for name, (k0, k1, z, gates) in expect.items():
        P = Oracle(get_config(name)).P
        assert (P.k0, P.k1, P.z, int(P.gate.sum())) == (k0, k1, z, gates)
