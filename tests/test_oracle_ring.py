"""Pins of the oracle's ring layer against definitions it does not share:
sympy primality, direct evaluation at the odd powers of psi, the schoolbook
negacyclic product (X^N = -1, Section 2.1), numpy's Philox4x64-10 and the
moments of the discrete Gaussian."""
import ctypes

import numpy as np
import pytest
import sympy

from oracle import _lib
from oracle._lib import lib, u64p
from oracle.cdt import cdt_table, probabilities

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def arr(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.uint64))


def p64(a):
    return a.ctypes.data_as(u64p)


@pytest.mark.parametrize("log_n,bits,r", [(10, 30, 1), (12, 50, 2), (13, 55, 3), (4, 20, 3)])
def test_primes_are_the_largest_ntt_friendly(log_n, bits, r):
    out = (ctypes.c_uint64 * r)()
    assert lib().or_find_primes(log_n, bits, r, ctypes.cast(out, u64p)) == 0
    qs = [int(v) for v in out]
    two_n = 2 << log_n
    for q in qs:
        assert sympy.isprime(q) and q % two_n == 1 and q < (1 << bits)
    assert qs == sorted(qs, reverse=True)
    # every candidate = 1 mod 2N above the smallest one found is either found or composite
    cand = ((1 << bits) - 2) // two_n * two_n + 1
    while cand >= qs[-1]:
        assert (cand in qs) == bool(sympy.isprime(cand))
        cand -= two_n


@pytest.mark.parametrize("log_n,bits", [(10, 30), (12, 50), (13, 55)])
def test_psi_is_primitive_2n_th_root(log_n, bits):
    out = (ctypes.c_uint64 * 1)()
    lib().or_find_primes(log_n, bits, 1, ctypes.cast(out, u64p))
    q = int(out[0])
    psi = int(lib().or_find_psi(q, log_n))
    n = 1 << log_n
    assert pow(psi, n, q) == q - 1
    assert pow(psi, 2 * n, q) == 1


def negacyclic_bigint(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [v % q for v in out]


SMALL = [(3, 97), (4, 97), (4, 7681), (6, 7681), (5, 12289), (6, 12289)]


@pytest.mark.parametrize("log_n,q", SMALL)
def test_transform_is_evaluation_at_odd_powers(log_n, q):
    n = 1 << log_n
    psi = int(lib().or_find_psi(q, log_n))
    rng = np.random.default_rng(log_n * q)
    a = [int(v) for v in rng.integers(0, q, size=n)]
    x = arr(a)
    lib().or_ntt_fwd(p64(x), log_n, q, psi)
    for k in range(n):
        ev = sum(a[i] * pow(psi, (2 * k + 1) * i, q) for i in range(n)) % q
        assert int(x[k]) == ev
    lib().or_ntt_inv(p64(x), log_n, q, psi)
    assert [int(v) for v in x] == a


@pytest.mark.parametrize("log_n,bits", [(3, 30), (5, 30), (6, 50), (6, 55)])
def test_ntt_product_matches_schoolbook_real_primes(log_n, bits):
    out = (ctypes.c_uint64 * 1)()
    lib().or_find_primes(log_n, bits, 1, ctypes.cast(out, u64p))
    q = int(out[0])
    psi = int(lib().or_find_psi(q, log_n))
    n = 1 << log_n
    rng = np.random.default_rng(bits)
    for trial in range(3):
        a = [int(v) for v in rng.integers(0, q, size=n, dtype=np.uint64)]
        b = [int(v) for v in rng.integers(0, q, size=n, dtype=np.uint64)]
        if trial == 1:  # edge values
            a = [q - 1] * n
            b = [(q - 1) // 2] * n
        ref = negacyclic_bigint(a, b, q)
        o1 = arr([0] * n)
        o2 = arr([0] * n)
        lib().or_poly_mul(p64(arr(a)), p64(arr(b)), p64(o1), log_n, q, psi)
        lib().or_poly_mul_schoolbook(p64(arr(a)), p64(arr(b)), p64(o2), n, q)
        assert [int(v) for v in o1] == ref
        assert [int(v) for v in o2] == ref


@pytest.mark.parametrize("log_n,q", SMALL)
def test_ntt_product_matches_schoolbook_small_primes(log_n, q):
    n = 1 << log_n
    psi = int(lib().or_find_psi(q, log_n))
    rng = np.random.default_rng(q + log_n)
    a = [int(v) for v in rng.integers(0, q, size=n)]
    b = [int(v) for v in rng.integers(0, q, size=n)]
    o = arr([0] * n)
    lib().or_poly_mul(p64(arr(a)), p64(arr(b)), p64(o), log_n, q, psi)
    assert [int(v) for v in o] == negacyclic_bigint(a, b, q)


def test_philox_matches_numpy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        ctr = [int(v) for v in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        ctr[0] |= 1  # numpy increments before generating: pass ctr - 1 without borrow
        c = (ctypes.c_uint64 * 4)(*ctr)
        k = (ctypes.c_uint64 * 2)(*key)
        o = (ctypes.c_uint64 * 4)()
        lib().or_philox(ctypes.cast(c, u64p), ctypes.cast(k, u64p), ctypes.cast(o, u64p))
        g = np.random.Philox(counter=[ctr[0] - 1] + ctr[1:], key=key)
        assert [int(v) for v in o] == [int(v) for v in g.random_raw(4)]


def test_cdt_table_shape_and_symmetry():
    t = cdt_table()
    assert len(t) == 38
    assert all(0 < x < 2**63 for x in t)
    assert list(t) == sorted(t)
    # P(X <= -1 - k) == P(X >= 1 + k): threshold i and 37 - i sum to 2^63 (up to flooring)
    for i in range(19):
        assert abs(t[i] + t[37 - i] - 2**63) <= 2


def test_gaussian_moments_and_frequencies():
    """Sampling 400k words through the oracle's inversion reproduces the
    distribution's moments (variance about sigma^2 = 10.24) and frequencies."""
    cfg_q = (ctypes.c_uint64 * 1)(97)
    cdt = (ctypes.c_uint64 * 38)(*cdt_table())
    ctx = lib().or_ctx_new(3, 1, ctypes.cast(cfg_q, u64p), ctypes.cast(cfg_q, u64p), 0, 1,
                           ctypes.cast(cdt, u64p))
    try:
        words = np.random.default_rng(1).integers(0, 2**64, size=400_000, dtype=np.uint64)
        xs = np.array([lib().or_gaussian(ctx, int(w)) for w in words], dtype=np.int64)
    finally:
        lib().or_ctx_free(ctx)
    probs = np.array(probabilities())
    exp_var = float(np.sum(probs * np.arange(-19, 20) ** 2))
    assert abs(exp_var - 10.24) < 0.01
    assert abs(xs.mean()) < 0.02
    assert abs(xs.var() - exp_var) < 0.1
    counts = np.bincount(xs + 19, minlength=39)
    # chi-square over the cells with expected count >= 20
    e = probs * xs.size
    m = e >= 20
    chi2 = float(np.sum((counts[m] - e[m]) ** 2 / e[m]))
    assert chi2 < 60.0  # about 25 degrees of freedom; p ~ 1e-4 bound
    assert xs.min() >= -19 and xs.max() <= 19


def test_library_builds():
    assert _lib.build()
