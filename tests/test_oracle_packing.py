"""Horizontal packing (Section 6) in the oracle.

Pins: ExtractLWE at coefficient 0 equals the C core's independent
ExtractLWE(., 0); the LWE extracted at any coefficient k decrypts to
coefficient k of the RLWE's own decryption; and packed inference decrypts to
the plaintext lookups of Algorithm 2 on every tree shape packing applies to
(none is left when a tree level is an encrypted address bit)."""
import numpy as np
import pytest

from oracle import Oracle, wisard
from oracle._lib import lib
from synthdata import get_config, make_dataset
from test_oracle_tfhe import enc_msg, p64, rand_ct

SHAPES = {
    "z0": dict(log_n=6, n_primes=1, prime_bits=30, log_beta=5, log_p=8, n_classes=2,
               n_values=5, therm_bits=2, addr_bits=3, tuple_bits=3),
    "zL": dict(log_n=6, n_primes=2, prime_bits=50, log_beta=0, log_p=16, n_classes=3,
               n_values=7, therm_bits=2, addr_bits=6, tuple_bits=6),
    "zltL": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=20, n_classes=5,
                 n_values=4, therm_bits=3, addr_bits=5, tuple_bits=8, hash_h3=1),
    "zgtL": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3,
                 n_values=4, therm_bits=2, addr_bits=7, tuple_bits=7),
}


def _cfg(name):
    return get_config("cfg1", data_kind="uniform", act="log", act_arg=0, **SHAPES[name])


def test_extract_at_zero_matches_the_c_core():
    o = Oracle(_cfg("zL"))
    ct = rand_ct(o, 3)
    ref = np.zeros(o.P.r * (o.P.n + 1), dtype=np.uint64)
    lib().or_extract_lwe0(o.ctx, p64(ct), p64(ref))
    assert np.array_equal(o.extract_lwe(ct, 0), ref)


def test_extract_at_k_decrypts_to_coefficient_k():
    o = Oracle(_cfg("zltL"))
    P = o.P
    s = o.keygen(5)
    rng = np.random.default_rng(8)
    msg = rng.integers(0, 1 << o.cfg.log_p, size=P.n)
    ct = enc_msg(o, s, msg, seed=9, stream=1)
    dec = o.decrypt_rlwe(s, ct)
    assert list(dec) == [int(m) for m in msg]
    for k in (0, 1, P.n // 2, P.n - 1):
        assert o.decrypt_lwe(s, o.extract_lwe(ct, k)) == int(msg[k])


@pytest.mark.parametrize("name", list(SHAPES))
def test_packed_inference_decrypts_to_the_lookups(name):
    cfg = _cfg(name)
    o = Oracle(cfg)
    P = o.P
    vals, labels = make_dataset(cfg, "train", n=6)
    tvals, _ = make_dataset(cfg, "test", n=3)
    bits, tbits = wisard.encode(P, vals), wisard.encode(P, tvals)
    s = o.keygen(2)
    H = o.train(o.new_model(), s, 5, bits, labels)
    resp, sums = o.infer_packed(H, s, 6, tbits)
    W = wisard.integer_wisard_train(P, bits, labels)
    look = wisard.lookups(P, W, tbits)
    dec = np.array([[[o.decrypt_lwe(s, resp[i, c, j]) for j in range(P.k0)]
                     for c in range(cfg.n_classes)] for i in range(3)])
    assert np.array_equal(dec, look)
    groups = o.packing_groups()
    if name == "zgtL":
        assert groups == {}
    else:
        assert sorted(c for g in groups.values() for c in g) == list(range(cfg.n_classes))
        assert len(groups) == min(cfg.n_classes, 1 << P.z)
