"""Pins of the oracle's TFHE layer (Section 2.4) and LUT blocks (Sections
2.4.2 and 3.3) against facts fixed by the mathematics:

* gadget recomposition sum_rho d_rho g_rho = x (mod Q), checked with Python
  integers and the CRT;
* the structure of trivial (noise-free) RGSW rows and the noise bound of
  real ones (phase minus message part within the Gaussian's support);
* noise-free exactness: a trivial RGSW of m multiplies any RLWE by m exactly;
* decryption invariants of CMUX, blind rotation, extraction, CDEMUX, IVP, VP.
"""
import ctypes

import numpy as np
import pytest

from oracle import Oracle
from oracle._lib import lib, u64p, i8p
from synthdata import get_config

CASES = {
    "r1_beta32": dict(log_n=5, n_primes=1, prime_bits=30, log_beta=5, log_p=8),
    "r2_rns": dict(log_n=5, n_primes=2, prime_bits=50, log_beta=0, log_p=16),
    "r3_rns": dict(log_n=4, n_primes=3, prime_bits=55, log_beta=0, log_p=22),
    "r2_beta1024": dict(log_n=4, n_primes=2, prime_bits=30, log_beta=10, log_p=12),
}


def make(case, **kw):
    d = dict(CASES[case])
    d.update(kw)
    return Oracle(get_config("cfg1", data_kind="uniform", n_values=4, therm_bits=2,
                             addr_bits=3, tuple_bits=3, n_classes=2, **d))


def p64(a):
    return a.ctypes.data_as(u64p)


def centred(v, q):
    v = int(v) % q
    return v - q if v > q // 2 else v


def rand_ct(o, seed):
    P = o.P
    rng = np.random.default_rng(seed)
    ct = np.zeros(o.rlwe_words, dtype=np.uint64)
    for comp in range(2):
        for j in range(P.r):
            off = (comp * P.r + j) * P.n
            ct[off:off + P.n] = rng.integers(0, P.q[j], size=P.n, dtype=np.uint64)
    return ct


def enc_msg(o, s, msg, seed=3, stream=0, trivial=False):
    """RLWE encryption of the message polynomial msg (values in [0, p))."""
    P = o.P
    m_scaled = np.zeros(P.r * P.n, dtype=np.uint64)
    for j in range(P.r):
        for k in range(P.n):
            m_scaled[j * P.n + k] = (P.delta * int(msg[k])) % P.q[j]
    out = np.zeros(o.rlwe_words, dtype=np.uint64)
    lib().or_encrypt_rlwe(o.ctx, s.ctypes.data_as(i8p), seed, stream, p64(m_scaled), int(trivial),
                          p64(out))
    return out


def negashift(msg, e, n, p):
    """msg * X^e in Z_p[X]/(X^N+1) by moving coefficients (sign on wrap)."""
    out = [0] * n
    e %= 2 * n
    for i, v in enumerate(msg):
        t, neg = i + e, False
        while t >= n:
            t -= n
            neg = not neg
        out[t] = (-v if neg else v) % p
    return out


@pytest.mark.parametrize("case", list(CASES))
def test_gadget_recomposition(case):
    o = make(case)
    P = o.P
    beta = 1 << o.cfg.log_beta if o.cfg.log_beta else None
    rng = np.random.default_rng(7)
    x = np.zeros(P.r * P.n, dtype=np.uint64)
    for j in range(P.r):
        x[j * P.n:(j + 1) * P.n] = rng.integers(0, P.q[j], size=P.n, dtype=np.uint64)
    x[0] = 0
    x[1] = P.q[0] - 1
    x[2] = (P.q[0] - 1) // 2
    X = [o.crt([x[j * P.n + k] for j in range(P.r)]) for k in range(P.n)]
    total = [0] * P.n
    dig = np.zeros(P.r * P.n, dtype=np.uint64)
    for rho in range(P.dnum):
        i, kk = divmod(rho, P.dpp)
        Mi = P.Q // P.q[i]
        g = (Mi * pow(Mi % P.q[i], -1, P.q[i]) * (beta ** kk if beta else 1)) % P.Q
        lib().or_decompose(o.ctx, p64(x), rho, p64(dig))
        for k in range(P.n):
            d = centred(dig[i * P.n + k], P.q[i])
            # the same signed digit lifted to every prime
            assert all(int(dig[j * P.n + k]) == d % P.q[j] for j in range(P.r))
            if beta and kk < P.dpp - 1:
                assert -beta // 2 <= d < beta // 2
            else:
                assert abs(d) <= P.q[i] // 2 + 1
            total[k] += d * g
    for k in range(P.n):
        assert total[k] % P.Q == X[k]


def _philox_words(seed, tag, c0, c1, c2):
    """Block (c0, c1, c2, 0) of Philox4x64-10 keyed (seed, tag), from numpy's
    implementation (it increments its 256-bit counter before each block)."""
    v = (c0 + (c1 << 64) + (c2 << 128) - 1) % (1 << 256)
    ctr = [(v >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
    return [int(w) for w in np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                                              key=np.array([seed, tag], dtype=np.uint64)).random_raw(4)]


def _smallest_primitive_root(q, n):
    """min over the primitive 2N-th roots of unity mod q: the odd powers of
    any one of them."""
    x = 2
    while True:
        c = pow(x, (q - 1) // (2 * n), q)
        if pow(c, n, q) == q - 1:
            return min(pow(c, 2 * i + 1, q) for i in range(n))
        x += 1


def _brv(k, bits):
    return int(format(k, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("bit", [0, 1])
def test_rgsw_mask_values_at_the_roots(case, bit):
    """Each row's mask a takes the uniform draw of sampling index k at
    zeta_k = psi_min^(2 brv(k) + 1) (psi_min the smallest primitive 2N-th root
    of unity): a evaluated there by Horner's rule (not a transform) equals
    (hi 2^64 + lo) mod q of words 2(k&1), 2(k&1)+1 of the RGSW_A block
    (k >> 1, row r + j, stream).  Rows dnum.. carry m g on a's constant
    term, which adds m g at every point."""
    o = make(case)
    P = o.P
    beta = 1 << o.cfg.log_beta if o.cfg.log_beta else None
    s = o.keygen(5)
    seed, stream = 9, 3
    rows = o.export_rgsw(o.encrypt_bit(s, seed, stream, bit)).reshape(2 * P.dnum, 2, P.r, P.n)
    for j in range(P.r):
        q = P.q[j]
        pmin = _smallest_primitive_root(q, P.n)
        zeta = [pow(pmin, 2 * _brv(k, P.log_n) + 1, q) for k in range(P.n)]
        for row in range(2 * P.dnum):
            rho = row % P.dnum
            i, kk = divmod(rho, P.dpp)
            g = (beta ** kk if beta else 1) % q if j == i else 0
            shift = bit * g if row >= P.dnum else 0
            a = [int(v) for v in rows[row, 0, j]]
            for k in range(P.n):
                val = 0
                for coef in reversed(a):
                    val = (val * zeta[k] + coef) % q
                w = _philox_words(seed, 2, k >> 1, row * P.r + j, stream)
                u = ((w[2 * (k & 1)] << 64) | w[2 * (k & 1) + 1]) % q
                assert val == (u + shift) % q, (row, j, k)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("bit", [0, 1])
def test_rgsw_rows(case, bit):
    """Rows 0..dnum-1 have phase e + m g (gadget on b), rows dnum.. have
    phase e - m g s (gadget on a); trivial rows are exactly (0, m g) and
    (m g, 0).  e is one integer polynomial shared by all primes."""
    o = make(case)
    P = o.P
    beta = 1 << o.cfg.log_beta if o.cfg.log_beta else None
    s = o.keygen(5)
    for trivial in (1, 0):
        rg = o.export_rgsw(o.encrypt_bit(s, 9, 3, bit, trivial=bool(trivial)))
        rows = rg.reshape(2 * P.dnum, 2, P.r, P.n)
        for row in range(2 * P.dnum):
            rho = row % P.dnum
            i, kk = divmod(rho, P.dpp)
            g = [(beta ** kk if beta else 1) % P.q[j] if j == i else 0 for j in range(P.r)]
            if trivial:
                for j in range(P.r):
                    exp_a = np.zeros(P.n, dtype=np.uint64)
                    exp_b = np.zeros(P.n, dtype=np.uint64)
                    if row < P.dnum:
                        exp_b[0] = bit * g[j]
                    else:
                        exp_a[0] = bit * g[j]
                    assert np.array_equal(rows[row, 0, j], exp_a)
                    assert np.array_equal(rows[row, 1, j], exp_b)
                continue
            ph = o.rlwe_phase(s, np.ascontiguousarray(rows[row].reshape(-1)))
            for k in range(P.n):
                errs = set()
                for j in range(P.r):
                    q = P.q[j]
                    if row < P.dnum:
                        expect = bit * g[j] if k == 0 else 0
                    else:  # -m g s: coefficient k of the constant g times s
                        expect = (-bit * g[j] * int(s[k])) % q
                    errs.add(centred(int(ph[j, k]) - expect, q))
                assert len(errs) == 1 and abs(errs.pop()) <= 19


@pytest.mark.parametrize("case", list(CASES))
def test_rlwe_roundtrip_and_trivial_exactness(case):
    o = make(case)
    P = o.P
    s = o.keygen(2)
    rng = np.random.default_rng(1)
    msg = [int(v) for v in rng.integers(0, P.p, size=P.n)]
    msg[0], msg[1] = 0, P.p - 1
    ct = enc_msg(o, s, msg)
    assert list(o.decrypt_rlwe(s, ct)) == msg
    ct0 = enc_msg(o, s, msg, trivial=True)
    for j in range(P.r):
        assert not ct0[j * P.n:(j + 1) * P.n].any()
        b = ct0[(P.r + j) * P.n:(P.r + j + 1) * P.n]
        assert [int(v) for v in b] == [(P.delta * m) % P.q[j] for m in msg]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("bit", [0, 1])
def test_external_product_noise_free_exact(case, bit):
    o = make(case)
    s = o.keygen(4)
    rg = o.encrypt_bit(s, 1, 0, bit, trivial=True)
    for seed in range(3):
        ct = rand_ct(o, seed)
        out = np.zeros_like(ct)
        lib().or_ext_product(o.ctx, p64(rg), p64(ct), p64(out))
        assert np.array_equal(out, ct if bit else np.zeros_like(ct))


@pytest.mark.parametrize("case", list(CASES))
def test_external_product_and_cmux_decrypt(case):
    o = make(case)
    P = o.P
    s = o.keygen(8)
    rng = np.random.default_rng(2)
    m1 = [int(v) for v in rng.integers(0, P.p, size=P.n)]
    m0 = [int(v) for v in rng.integers(0, P.p, size=P.n)]
    c1 = enc_msg(o, s, m1, stream=1)
    c0 = enc_msg(o, s, m0, stream=2)
    for bit in (0, 1):
        rg = o.encrypt_bit(s, 6, 10 + bit, bit)
        out = np.zeros_like(c1)
        lib().or_ext_product(o.ctx, p64(rg), p64(c1), p64(out))
        assert list(o.decrypt_rlwe(s, out)) == (m1 if bit else [0] * P.n)
        lib().or_cmux(o.ctx, p64(rg), p64(c1), p64(c0), p64(out))
        assert list(o.decrypt_rlwe(s, out)) == (m1 if bit else m0)


def test_rotation_moves_coefficients_negacyclically():
    o = make("r2_rns")
    P = o.P
    s = o.keygen(1)
    msg = list(range(P.n))
    ct = enc_msg(o, s, msg)
    for e in (0, 1, 5, P.n - 1, P.n, P.n + 3, 2 * P.n - 1, -3):
        out = np.zeros_like(ct)
        lib().or_rlwe_rotate(o.ctx, p64(ct), e, p64(out))
        assert list(o.decrypt_rlwe(s, out)) == negashift(msg, e, P.n, P.p)


@pytest.mark.parametrize("sign", [1, -1])
def test_blind_rotate(sign):
    o = make("r1_beta32")
    P = o.P
    s = o.keygen(3)
    msg = [(3 * k + 1) % P.p for k in range(P.n)]
    ct = enc_msg(o, s, msg)
    bits = [1, 0, 1, 1]
    rgs = [o.encrypt_bit(s, 2, 20 + t, b) for t, b in enumerate(bits)]
    ptrs = (u64p * 5)(*[p64(r) for r in rgs], ctypes.cast(None, u64p))
    clear = (ctypes.c_int * 5)(0, 0, 0, 0, 1)  # last bit given in clear, value 1
    acc = ct.copy()
    lib().or_blind_rotate(o.ctx, p64(acc), ptrs, clear, 5, sign)
    total = sum(b << t for t, b in enumerate(bits + [1]))
    assert list(o.decrypt_rlwe(s, acc)) == negashift(msg, -sign * total, P.n, P.p)


@pytest.mark.parametrize("case", ["r1_beta32", "r3_rns"])
def test_extract_phase_is_coefficient_zero(case):
    o = make(case)
    P = o.P
    s = o.keygen(6)
    ct = rand_ct(o, 9)
    lwe = np.zeros(P.r * (P.n + 1), dtype=np.uint64)
    lib().or_extract_lwe0(o.ctx, p64(ct), p64(lwe))
    ph = o.rlwe_phase(s, ct)
    lph = np.zeros(P.r, dtype=np.uint64)
    lib().or_lwe_phase(o.ctx, s.ctypes.data_as(i8p), p64(lwe), p64(lph))
    assert [int(v) for v in lph] == [int(ph[j, 0]) for j in range(P.r)]


@pytest.mark.parametrize("bit", [0, 1])
def test_cdemux_outputs_sum_to_input(bit):
    o = make("r2_rns")
    P = o.P
    s = o.keygen(2)
    msg = [(7 * k) % P.p for k in range(P.n)]
    d = enc_msg(o, s, msg)
    rg = o.encrypt_bit(s, 4, 1, bit)
    lo, hi = d.copy(), np.zeros_like(d)
    lib().or_cdemux(o.ctx, p64(rg), p64(lo), p64(hi))
    tot = lo.copy()
    lib().or_rlwe_add(o.ctx, p64(tot), p64(hi))
    assert np.array_equal(tot, d)  # bit-exact: (d - C.d) + C.d = d
    assert list(o.decrypt_rlwe(s, hi)) == (msg if bit else [0] * P.n)
    assert list(o.decrypt_rlwe(s, lo)) == ([0] * P.n if bit else msg)


def _ivp_case(o, s, m, k, z):
    P = o.P
    rgs = [o.encrypt_bit(s, 12, 100 + t, (m >> t) & 1) for t in range(k)]
    ptrs = (u64p * k)(*[p64(r) for r in rgs])
    clear = (ctypes.c_int * k)()
    gate = np.ones(max(1, z) * max(1, 1 << max(0, z - 1)), dtype=np.uint8)
    L = np.zeros((1 << z) * o.rlwe_words, dtype=np.uint64)
    lhat = o.trivial_one()
    lib().or_ivp(o.ctx, p64(lhat), ptrs, clear, k, z, gate.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                 p64(L))
    return L.reshape(1 << z, -1), rgs


@pytest.mark.parametrize("m", [0, 5, 11, 31, 44, 63])
def test_ivp_is_one_hot_and_vp_reads_it_back(m):
    """IVP(b, (0,1)) with z = 2 tree bits and 4 rotation bits on N = 16
    decrypts to a one-hot LUT at m (ciphertext m mod 4, coefficient m >> 2);
    VP over the same bits reads 1 back, and reads LUT[m] of a random LUT."""
    o = make("r2_rns", log_n=4)
    P = o.P
    s = o.keygen(13)
    k, z = 6, 2
    L, rgs = _ivp_case(o, s, m, k, z)
    for v in range(1 << z):
        dec = o.decrypt_rlwe(s, L[v])
        expect = [0] * P.n
        if v == m % (1 << z):
            expect[m >> z] = 1
        assert list(dec) == expect
    ptrs = (u64p * k)(*[p64(r) for r in rgs])
    clear = (ctypes.c_int * k)()
    Lin = (u64p * (1 << z))(*[p64(np.ascontiguousarray(L[v])) for v in range(1 << z)])
    lwe = np.zeros(P.r * (P.n + 1), dtype=np.uint64)
    lib().or_vp(o.ctx, Lin, ptrs, clear, k, z, p64(lwe))
    assert o.decrypt_lwe(s, lwe) == 1
    # an arbitrary LUT: ciphertext v holds entries v + 4 * coefficient
    lut = np.random.default_rng(m).integers(0, P.p, size=1 << k)
    cts = [enc_msg(o, s, [int(lut[v + (x << z)]) for x in range(P.n)], stream=200 + v)
           for v in range(1 << z)]
    Lin = (u64p * (1 << z))(*[p64(c) for c in cts])
    lib().or_vp(o.ctx, Lin, ptrs, clear, k, z, p64(lwe))
    assert o.decrypt_lwe(s, lwe) == int(lut[m])
