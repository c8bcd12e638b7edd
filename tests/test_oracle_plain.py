"""Unencrypted-model inference (Section 3.6.2) in the oracle.

Pins: the RLWE-by-plaintext product multiplies the phase by the plaintext
exactly (against the schoolbook negacyclic product of the phases); with
noise-free RGSWs every response is exactly the trivial LWE (0, Delta W[c][j]
[addr]) -- which fixes the rotation direction, the table layout and the
CMUX tree of an encrypted address bit; with noisy ones the responses decrypt
to the plaintext lookups of Algorithm 2 and the sums to its scores, on every
tree shape (z = 0, z = L, z < L with H3, and z > L where one address bit
drives the tree)."""
import ctypes

import numpy as np
import pytest

from oracle import Oracle, wisard
from oracle._lib import lib
from synthdata import get_config, make_dataset
from test_oracle_packing import SHAPES
from test_oracle_tfhe import p64, rand_ct

ll_p = ctypes.POINTER(ctypes.c_longlong)


def _cfg(name):
    return get_config("cfg1", data_kind="uniform", act="log", act_arg=0, **SHAPES[name])


def _random_model(P, l, seed, hi):
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(l, P.k0, 1 << P.a)).astype(np.int64)


def test_plaintext_product_multiplies_the_phase():
    o = Oracle(_cfg("zltL"))
    P = o.P
    s = o.keygen(4)
    ct = rand_ct(o, 11)
    rng = np.random.default_rng(3)
    t = rng.integers(-40, 40, size=P.n).astype(np.int64)
    out = np.zeros(o.rlwe_words, dtype=np.uint64)
    lib().or_rlwe_mul_plain(o.ctx, p64(ct), t.ctypes.data_as(ll_p), p64(out))
    ph, ph_out = o.rlwe_phase(s, ct), o.rlwe_phase(s, out)
    for j in range(P.r):
        q = int(P.q[j])
        tq = np.array([int(x) % q for x in t], dtype=np.uint64)
        ref = np.zeros(P.n, dtype=np.uint64)
        lib().or_poly_mul_schoolbook(p64(np.ascontiguousarray(ph[j])), p64(tq), p64(ref), P.n, q)
        assert np.array_equal(ph_out[j], ref)


def test_tables_cover_every_address_once():
    for name in SHAPES:
        o = Oracle(_cfg(name))
        P = o.P
        zt = o.plain_split()
        assert P.a - zt <= P.log_n
        W = _random_model(P, o.cfg.n_classes, 1, 1000)
        tabs = o.plain_tables(W, P.k0 - 1, 1)
        assert len(tabs) == 1 << zt
        for addr in range(1 << P.a):
            assert tabs[addr % (1 << zt)][addr >> zt] == W[1, P.k0 - 1, addr]


@pytest.mark.parametrize("name", list(SHAPES))
def test_noise_free_responses_are_exact(name):
    cfg = _cfg(name)
    o = Oracle(cfg)
    P = o.P
    tvals, _ = make_dataset(cfg, "test", n=2)
    tbits = wisard.encode(P, tvals)
    W = _random_model(P, cfg.n_classes, 7, 50)
    s = o.keygen(2)
    resp, _ = o.infer_plain(W, s, 6, tbits, trivial=True)
    look = wisard.lookups(P, W, tbits)
    for i in range(2):
        for c in range(cfg.n_classes):
            for j in range(P.k0):
                lwe = resp[i, c, j].reshape(P.r, P.n + 1)
                for jp in range(P.r):
                    q = int(P.q[jp])
                    assert not lwe[jp, :P.n].any()
                    assert int(lwe[jp, P.n]) == (P.delta * int(look[i, c, j])) % q


@pytest.mark.parametrize("name", list(SHAPES))
def test_clear_model_inference_decrypts_to_the_lookups(name):
    cfg = _cfg(name)
    o = Oracle(cfg)
    P = o.P
    vals, labels = make_dataset(cfg, "train", n=8)
    tvals, _ = make_dataset(cfg, "test", n=3)
    bits, tbits = wisard.encode(P, vals), wisard.encode(P, tvals)
    W = wisard.integer_wisard_train(P, bits, labels)
    # spread counters over every address as well, so that a wrong table
    # index reads a different value
    W = W + _random_model(P, cfg.n_classes, 9, 3)
    s = o.keygen(2)
    resp, sums = o.infer_plain(W, s, 5, tbits)
    look = wisard.lookups(P, W, tbits)
    dec = np.array([[[o.decrypt_lwe(s, resp[i, c, j]) for j in range(P.k0)]
                     for c in range(cfg.n_classes)] for i in range(3)])
    assert np.array_equal(dec, look)
    if name != "z0":  # the 30-bit ring's sums are not decoded (budget of p)
        sc = np.array([[o.decrypt_lwe(s, sums[i, c]) for c in range(cfg.n_classes)]
                       for i in range(3)])
        assert np.array_equal(sc, look.sum(axis=2) % P.p)


def test_encrypted_and_clear_model_responses_decrypt_alike():
    cfg = _cfg("zL")
    o = Oracle(cfg)
    P = o.P
    vals, labels = make_dataset(cfg, "train", n=6)
    tvals, _ = make_dataset(cfg, "test", n=2)
    bits, tbits = wisard.encode(P, vals), wisard.encode(P, tvals)
    s = o.keygen(3)
    H = o.train(o.new_model(), s, 5, bits, labels)
    W = o.decrypt_model(s, H)
    r_enc, _ = o.infer(H, s, 6, tbits)
    r_pl, _ = o.infer_plain(W, s, 6, tbits)
    for i in range(2):
        for c in range(cfg.n_classes):
            for j in range(P.k0):
                assert o.decrypt_lwe(s, r_enc[i, c, j]) == o.decrypt_lwe(s, r_pl[i, c, j])
