"""Derived parameters of a workload, computed by the oracle on its own.

TEST INFRASTRUCTURE ONLY.

Ring and modulus (Section 2.4, Setup): the paper works over a 64-bit torus
and leaves q unspecified; this project's reading is an RNS modulus
Q = q_0 ... q_{r-1} of the r largest primes below 2^prime_bits with
q = 1 (mod 2N), and Delta = floor(Q / p).

Model shape (Definition 2): k0 = ceil(s / a) RAMs.  The LUT index of a RAM
is m = label + 2^L * address with L = ceil(log2 l) label bits in the low
positions (Algorithm 6 puts the label bits first).  The low z = max(0,
L + a - log2 N) bits select the ciphertext (the CDEMUX/CMUX tree) and the
rest select the coefficient (the blind rotation), as Algorithms 3 and 5 do.
Only ciphertext indices reachable by a label below l are stored (the set V);
a tree gate is evaluated only if some index of V lies below its upper output.
"""
from dataclasses import dataclass
import math

import numpy as np

from ._lib import lib, u64p
import ctypes


@dataclass
class Params:
    cfg: object
    log_n: int
    n: int
    r: int
    q: list
    psi: list
    Q: int
    p: int
    delta: int
    L: int
    s: int
    a: int
    k0: int
    z: int
    V: list
    slot: dict
    k1: int
    gate: np.ndarray          # uint8 [max(z,1) * max(2^(z-1),1)]
    dpp: int
    dnum: int
    n_data: int
    n_slots: int


def label_bits(l: int) -> int:
    return max(0, math.ceil(math.log2(l))) if l > 1 else 0


def primes(log_n: int, bits: int, r: int):
    out = (ctypes.c_uint64 * r)()
    rc = lib().or_find_primes(log_n, bits, r, ctypes.cast(out, u64p))
    if rc != 0:
        raise ValueError("not enough NTT-friendly primes")
    return [int(v) for v in out]


def derive(cfg) -> Params:
    L = label_bits(cfg.n_classes)
    n = 1 << cfg.log_n
    q = primes(cfg.log_n, cfg.prime_bits, cfg.n_primes)
    psi = [int(lib().or_find_psi(qi, cfg.log_n)) for qi in q]
    Q = 1
    for qi in q:
        Q *= qi
    p = 1 << cfg.log_p
    s = cfg.n_values * cfg.therm_bits
    a = cfg.addr_bits
    if cfg.hash_h3:
        k0 = -(-s // cfg.tuple_bits)
        n_data = k0 * a
    else:
        k0 = -(-s // a)
        n_data = s
    z = max(0, L + a - cfg.log_n)
    vs = set()
    for c in range(cfg.n_classes):
        for x in range(1 << max(0, z - L)):
            vs.add((c + (x << L)) % (1 << z))
    V = sorted(vs)
    slot = {v: i for i, v in enumerate(V)}
    half = max(1, 1 << max(0, z - 1))
    gate = np.zeros(max(1, z) * half, dtype=np.uint8)
    for i in range(z):
        for j in range(1 << i):
            if any(v % (1 << (i + 1)) == j + (1 << i) for v in V):
                gate[i * half + j] = 1
    dpp = -(-cfg.prime_bits // cfg.log_beta) if cfg.log_beta else 1
    return Params(cfg=cfg, log_n=cfg.log_n, n=n, r=cfg.n_primes, q=q, psi=psi, Q=Q, p=p,
                  delta=Q // p, L=L, s=s, a=a, k0=k0, z=z, V=V, slot=slot, k1=len(V),
                  gate=gate, dpp=dpp, dnum=cfg.n_primes * dpp, n_data=n_data,
                  n_slots=L + n_data)
