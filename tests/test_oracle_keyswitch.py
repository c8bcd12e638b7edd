"""PackingKeySwitching (Section 2.4) in the oracle.

Pins: with a noise-free, mask-free key the packed RLWE is exactly
(0, sum_i phase(LWE_i) X^i) -- the definition with every term visible; with
a real key, coefficient i of the packed RLWE decrypts to the message of LWE
i for i < k and to 0 above; and key rows decrypt to s_x * g_rho."""
import numpy as np
import pytest

from oracle import Oracle
from oracle._lib import lib
from synthdata import get_config
from test_oracle_tfhe import enc_msg, p64

SHAPES = {
    "beta32": dict(log_n=6, n_primes=1, prime_bits=30, log_beta=5, log_p=8, n_classes=2,
                   n_values=5, therm_bits=2, addr_bits=3, tuple_bits=3),
    "rns3": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=20, n_classes=5,
                 n_values=4, therm_bits=3, addr_bits=5, tuple_bits=8, hash_h3=1),
}


def _cfg(name):
    return get_config("cfg1", data_kind="uniform", act="log", act_arg=0, **SHAPES[name])


def _lwes(o, s, msgs, seed):
    """LWEs of the given messages: extracted coefficients of encrypted RLWEs."""
    P = o.P
    out = []
    for t, m in enumerate(msgs):
        poly = np.zeros(P.n, dtype=np.int64)
        poly[t % P.n] = m
        ct = enc_msg(o, s, poly, seed=seed, stream=t)
        out.append(o.extract_lwe(ct, t % P.n))
    return np.stack(out)


def _phase(o, s, lwe):
    P = o.P
    ph = np.zeros(P.r, dtype=np.uint64)
    from oracle._lib import i8p
    lib().or_lwe_phase(o.ctx, s.ctypes.data_as(i8p), p64(np.ascontiguousarray(lwe)), p64(ph))
    return ph


@pytest.mark.parametrize("name", list(SHAPES))
def test_noise_free_key_gives_the_phases_exactly(name):
    o = Oracle(_cfg(name))
    P = o.P
    s = o.keygen(3)
    msgs = [5, 0, 1, 7, 3]
    lw = _lwes(o, s, msgs, seed=11)
    C = o.pack(o.ksk_gen(s, 4, trivial=True), lw)
    a = C[: P.r * P.n].reshape(P.r, P.n)
    b = C[P.r * P.n:].reshape(P.r, P.n)
    assert not a.any()
    for i in range(len(msgs)):
        assert np.array_equal(b[:, i], _phase(o, s, lw[i]))
    assert not b[:, len(msgs):].any()


@pytest.mark.parametrize("name", list(SHAPES))
def test_packed_rlwe_decrypts_to_the_messages(name):
    cfg = _cfg(name)
    o = Oracle(cfg)
    P = o.P
    s = o.keygen(8)
    rng = np.random.default_rng(2)
    k = P.n - 5
    msgs = [int(v) for v in rng.integers(0, 1 << cfg.log_p, size=k)]
    C = o.pack(o.ksk_gen(s, 9), _lwes(o, s, msgs, seed=12))
    dec = o.decrypt_rlwe(s, C)
    assert list(dec[:k]) == msgs and not dec[k:].any()


def test_key_rows_decrypt_to_key_times_gadget():
    o = Oracle(_cfg("rns3"))
    P = o.P
    s = o.keygen(1)
    ksk = o.ksk_gen(s, 2).reshape(P.n, P.dnum, -1)
    for x in (0, 1, P.n - 1):
        for rho in range(P.dnum):
            ph = o.rlwe_phase(s, ksk[x, rho])  # (r, N) residues of the phase
            # phase = s_x * g_rho + e: at prime rho (beta = q_i) g is 1, else 0
            for j in range(P.r):
                v = int(ph[j, 0])
                q = int(P.q[j])
                centred = v - q if v > q // 2 else v
                expect = int(s[x]) if j == rho else 0
                assert abs(centred - expect) <= 19  # the Gaussian's support bounds e
