"""Homomorphic training and inference of the oracle.  TEST INFRASTRUCTURE ONLY.

Thin Python orchestration over the C routines of oracle.c, following
Algorithm 6 (training) and Algorithm 7 (inference, PD-act) item by item.
Decryption rounds with Python integers: the phase residues are combined by
the Chinese remainder theorem into phi in [0, Q) and the message is
round(p * phi / Q) mod p = floor((p * phi + floor(Q/2)) / Q) mod p
(DecRLWE/DecLWE, Section 2.4; Q is odd and p a power of two, so no ties).

Encrypted-bit streams: bit slot b of sample i (slot l < L is label bit l,
slot L + d is data bit d) is encrypted under stream index i * n_slots + b.
"""
import ctypes

import numpy as np

from . import wisard
from ._lib import lib, u64p, i8p, u8p
from .cdt import cdt_table
from .params import derive


def _p64(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(u64p)


class Oracle:
    def __init__(self, cfg):
        self.cfg = cfg
        self.P = P = derive(cfg)
        q = (ctypes.c_uint64 * P.r)(*P.q)
        psi = (ctypes.c_uint64 * P.r)(*P.psi)
        cdt = (ctypes.c_uint64 * 38)(*cdt_table())
        self.ctx = lib().or_ctx_new(P.log_n, P.r, ctypes.cast(q, u64p), ctypes.cast(psi, u64p),
                                    cfg.log_beta, P.dpp, ctypes.cast(cdt, u64p))
        self.rlwe_words = int(lib().or_rlwe_words(self.ctx))
        self.rgsw_words = int(lib().or_rgsw_words(self.ctx))
        self.ram_bits = wisard.ram_bits(P)

    def __del__(self):
        try:
            lib().or_ctx_free(self.ctx)
        except Exception:
            pass

    # ---------------------------------------------------------------- keys
    def keygen(self, seed: int) -> np.ndarray:
        s = np.zeros(self.P.n, dtype=np.int8)
        lib().or_keygen(self.ctx, seed, s.ctypes.data_as(i8p))
        return s

    # ---------------------------------------------------------- encryption
    def encrypt_bit(self, s, seed, stream_idx, value, trivial=False) -> np.ndarray:
        out = np.zeros(self.rgsw_words, dtype=np.uint64)
        lib().or_encrypt_rgsw(self.ctx, s.ctypes.data_as(i8p), seed, stream_idx, int(value),
                              int(trivial), _p64(out))
        return out

    def export_rgsw(self, rgsw) -> np.ndarray:
        out = np.zeros(self.rgsw_words, dtype=np.uint64)
        lib().or_rgsw_export(self.ctx, _p64(rgsw), _p64(out))
        return out

    def encrypt_slots(self, s, seed, sample_idx, data_bits_row, label, slots, trivial=False):
        """RGSW of the requested bit slots of one sample, keyed by slot."""
        P = self.P
        out = {}
        for b in slots:
            if b < P.L:
                val = (int(label) >> b) & 1
            else:
                val = int(data_bits_row[b - P.L])
            out[b] = self.encrypt_bit(s, seed, sample_idx * P.n_slots + b, val, trivial)
        return out

    def slots_for_rams(self, rams, with_labels=True):
        P = self.P
        sl = set(range(P.L)) if with_labels else set()
        for j in rams:
            for d in self.ram_bits[j]:
                if d >= 0:
                    sl.add(P.L + int(d))
        return sorted(sl)

    def trivial_one(self) -> np.ndarray:
        """(0, Delta * 1): the trivial RLWE of the constant 1."""
        P = self.P
        ct = np.zeros(self.rlwe_words, dtype=np.uint64)
        for j in range(P.r):
            ct[(P.r + j) * P.n] = P.delta % P.q[j]
        return ct

    # ------------------------------------------------------------ training
    def ivp_item(self, rgsw_by_slot, j) -> np.ndarray:
        """IVP(b, (0,1)) for RAM j with b = [label bits, tuple bits of RAM j]
        (Algorithm 6); returns the 2^z RLWE outputs."""
        P = self.P
        k = P.L + P.a
        ptrs = (u64p * k)()
        clear = (ctypes.c_int * k)()
        keep = []
        for t in range(P.L):
            ptrs[t] = _p64(rgsw_by_slot[t])
        for i in range(P.a):
            d = int(self.ram_bits[j][i])
            if d >= 0:
                ptrs[P.L + i] = _p64(rgsw_by_slot[P.L + d])
            else:
                ptrs[P.L + i] = ctypes.cast(None, u64p)
                clear[P.L + i] = 0
        lhat = self.trivial_one()
        L = np.zeros((1 << P.z) * self.rlwe_words, dtype=np.uint64)
        keep.append(lhat)
        lib().or_ivp(self.ctx, _p64(lhat), ptrs, clear, k, P.z, P.gate.ctypes.data_as(u8p), _p64(L))
        return L.reshape(1 << P.z, self.rlwe_words)

    def new_model(self) -> np.ndarray:
        P = self.P
        return np.zeros((P.k0, P.k1, self.rlwe_words), dtype=np.uint64)

    def train(self, H, s, seed, data_bits, labels, rams=None, sample_offset=0, trivial=False):
        """Algorithm 6 over the given samples; only the listed RAMs are
        updated (rows of H are independent).  H is modified in place."""
        P = self.P
        rams = list(range(P.k0)) if rams is None else list(rams)
        slots = self.slots_for_rams(rams)
        for i in range(data_bits.shape[0]):
            rg = self.encrypt_slots(s, seed, sample_offset + i, data_bits[i], labels[i], slots,
                                    trivial)
            for j in rams:
                L = self.ivp_item(rg, j)
                for v in P.V:
                    lib().or_rlwe_add(self.ctx, _p64(H[j, P.slot[v]]), _p64(np.ascontiguousarray(L[v])))
        return H

    # ---------------------------------------------- dataset balancing (3.6.1)
    def count_item(self, rgsw_by_slot) -> np.ndarray:
        """Section 3.6.1: a small IVP over the label bits of one sample --
        BlindRotate from the trivial (0, Delta) with weights -2^t (X^{+2^t})
        over the L label slots -- leaves Delta at coefficient = label."""
        P = self.P
        acc = self.trivial_one()
        ptrs = (u64p * P.L)()
        clear = (ctypes.c_int * P.L)()
        for t in range(P.L):
            ptrs[t] = _p64(rgsw_by_slot[t])
        lib().or_blind_rotate(self.ctx, _p64(acc), ptrs, clear, P.L, -1)
        return acc

    def count_classes(self, counts, s, seed, labels, sample_offset=0):
        """Adds every sample's class-count RLWE into `counts` (rlwe_words),
        from the same encrypted label bits training uses; coefficient c of the
        sum decrypts to the number of samples of class c."""
        P = self.P
        for i, lab in enumerate(labels):
            rg = self.encrypt_slots(s, seed, sample_offset + i, None, lab, range(P.L))
            lib().or_rlwe_add(self.ctx, _p64(counts), _p64(self.count_item(rg)))
        return counts

    # ----------------------------------------------------------- inference
    def vp_item(self, H, rgsw_by_slot, j, c) -> np.ndarray:
        """VP(b, H[j]) with clear label bits of class c (Algorithm 7)."""
        P = self.P
        k = P.L + P.a
        ptrs = (u64p * k)()
        clear = (ctypes.c_int * k)()
        for t in range(P.L):
            ptrs[t] = ctypes.cast(None, u64p)
            clear[t] = (c >> t) & 1
        for i in range(P.a):
            d = int(self.ram_bits[j][i])
            if d >= 0:
                ptrs[P.L + i] = _p64(rgsw_by_slot[P.L + d])
            else:
                ptrs[P.L + i] = ctypes.cast(None, u64p)
                clear[P.L + i] = 0
        nl = 1 << P.z
        Lin = (u64p * nl)()
        rows = []
        for v in range(nl):
            if v in P.slot:
                row = np.ascontiguousarray(H[j, P.slot[v]])
                rows.append(row)
                Lin[v] = _p64(row)
            else:
                Lin[v] = ctypes.cast(None, u64p)
        lwe = np.zeros(P.r * (P.n + 1), dtype=np.uint64)
        lib().or_vp(self.ctx, Lin, ptrs, clear, k, P.z, _p64(lwe))
        return lwe

    # --------------------------------------------- PackingKeySwitching
    def ksk_gen(self, s, seed, trivial=False) -> np.ndarray:
        """PackingKeySwitching key (Section 2.4): N * dnum RLWE rows
        (x, rho) encrypting s_x * g_rho, coefficient form."""
        P = self.P
        out = np.zeros(P.n * P.dnum * self.rlwe_words, dtype=np.uint64)
        lib().or_ksk_gen(self.ctx, s.ctypes.data_as(i8p), seed, int(trivial), _p64(out))
        return out

    def pack(self, ksk, lwes) -> np.ndarray:
        """PackingKeySwitching of k <= N LWEs (k, r*(N+1)) into one RLWE
        encrypting sum_i m_i X^i."""
        lwes = np.ascontiguousarray(lwes, dtype=np.uint64).reshape(-1)
        k = lwes.size // (self.P.r * (self.P.n + 1))
        assert k <= self.P.n
        out = np.zeros(self.rlwe_words, dtype=np.uint64)
        lib().or_pack_keyswitch(self.ctx, _p64(ksk), _p64(lwes), k, _p64(out))
        return out

    # ------------------------------------------------ horizontal packing
    def packing_groups(self):
        """Classes that share a stored ciphertext and differ only in clear
        rotation bits (label bits z..L-1), keyed by c mod 2^z; empty when a
        tree level is an encrypted address bit (z > L): no packing then."""
        P = self.P
        if P.z > P.L:
            return {}
        g = {}
        for c in range(self.cfg.n_classes):
            g.setdefault(c % (1 << P.z), []).append(c)
        return g

    def extract_lwe(self, ct, k) -> np.ndarray:
        """ExtractLWE(ct, k): the LWE of coefficient k of the phase,
        a'_x = a_{k-x} for x <= k, -a_{N+k-x} otherwise, b' = b_k."""
        P = self.P
        n, r = P.n, P.r
        a = ct[: r * n].reshape(r, n)
        b = ct[r * n:].reshape(r, n)
        out = np.zeros((r, n + 1), dtype=np.uint64)
        for j in range(r):
            q = int(P.q[j])
            for x in range(n):
                out[j, x] = a[j, k - x] if x <= k else (q - int(a[j, n + k - x])) % q
            out[j, n] = b[j, k]
        return out.reshape(-1)

    def vp_item_packed(self, H, rgsw_by_slot, j, rho) -> dict:
        """Horizontal packing (Section 6): one VP of H[j] for every class
        c = rho (mod 2^z) at once -- the clear label bits above z are not
        rotated, so the lookup of class c sits at coefficient c >> z of the
        accumulator; returns {c: LWE}."""
        P = self.P
        k = P.L + P.a
        ptrs = (u64p * k)()
        clear = (ctypes.c_int * k)()
        for t in range(P.L):
            ptrs[t] = ctypes.cast(None, u64p)
            clear[t] = ((rho >> t) & 1) if t < P.z else 0
        for i in range(P.a):
            d = int(self.ram_bits[j][i])
            if d >= 0:
                ptrs[P.L + i] = _p64(rgsw_by_slot[P.L + d])
            else:
                ptrs[P.L + i] = ctypes.cast(None, u64p)
                clear[P.L + i] = 0
        nl = 1 << P.z
        Lin = (u64p * nl)()
        rows = []
        for v in range(nl):
            if v in P.slot:
                row = np.ascontiguousarray(H[j, P.slot[v]])
                rows.append(row)
                Lin[v] = _p64(row)
            else:
                Lin[v] = ctypes.cast(None, u64p)
        acc = np.zeros(self.rlwe_words, dtype=np.uint64)
        lib().or_vp_rlwe(self.ctx, Lin, ptrs, clear, k, P.z, _p64(acc))
        return {c: self.extract_lwe(acc, c >> P.z) for c in self.packing_groups()[rho]}

    def infer_packed(self, H, s, seed, data_bits, rams=None, sample_offset=0):
        """Inference with horizontal packing: responses u[i][c][j] (LWE) and
        per-class sums, as infer() lays them out."""
        P = self.P
        l = self.cfg.n_classes
        groups = self.packing_groups()
        if not groups:
            return self.infer(H, s, seed, data_bits, rams, sample_offset)
        rams = list(range(P.k0)) if rams is None else list(rams)
        slots = self.slots_for_rams(rams, with_labels=False)
        n = data_bits.shape[0]
        lw = P.r * (P.n + 1)
        resp = np.zeros((n, l, len(rams), lw), dtype=np.uint64)
        sums = np.zeros((n, l, lw), dtype=np.uint64)
        for i in range(n):
            rg = self.encrypt_slots(s, seed, sample_offset + i, data_bits[i], 0, slots)
            for jj, j in enumerate(rams):
                for rho in groups:
                    for c, lwe in self.vp_item_packed(H, rg, j, rho).items():
                        resp[i, c, jj] = lwe
            for c in range(l):
                for jj in range(len(rams)):
                    lib().or_lwe_add(self.ctx, _p64(sums[i, c]), _p64(np.ascontiguousarray(resp[i, c, jj])))
        return resp, sums

    # ------------------------------------- unencrypted-model inference
    def plain_split(self):
        """Address bits of a clear-model lookup: the low zt = max(0, z - L)
        bits drive a CMUX tree (the table of one class does not fit one
        polynomial), the other a - zt <= log2 N bits the blind rotation."""
        P = self.P
        return max(0, P.z - P.L)

    def plain_tables(self, W, j, c):
        """The clear LUT of RAM j, class c as 2^zt plaintext polynomials:
        coefficient k of table v is the counter of address v + 2^zt k."""
        P = self.P
        zt = self.plain_split()
        row = np.asarray(W[c, j], dtype=np.int64)
        out = []
        for v in range(1 << zt):
            t = np.zeros(P.n, dtype=np.int64)
            part = row[v::1 << zt]
            t[: part.size] = part
            out.append(t)
        return out

    def vp_plain_item(self, W, rgsw_by_slot, j) -> dict:
        """VP of RAM j against a model in clear (Section 3.6.2 notes that
        inference is faster when the model is not encrypted).  The lookup
        tables are plaintexts, so the blind rotation depends only on the
        sample: R = BlindRotate((0, Delta), address bits zt..a-1) with weights
        +2^0, +2^1, ... (X^-2^t) runs once, and class c's response is
        ExtractLWE of the CMUX tree (address bits 0..zt-1, Algorithm 3's
        tree) over the products R * T_v -- coefficient 0 of
        Delta X^-addr T_v(X) is Delta T_v[addr].  Returns {c: LWE}."""
        P = self.P
        zt = self.plain_split()
        nb = P.a - zt
        ptrs = (u64p * max(nb, 1))()
        clear = (ctypes.c_int * max(nb, 1))()
        for i in range(nb):
            d = int(self.ram_bits[j][zt + i])
            ptrs[i] = _p64(rgsw_by_slot[P.L + d]) if d >= 0 else ctypes.cast(None, u64p)
        acc = self.trivial_one()
        lib().or_blind_rotate(self.ctx, _p64(acc), ptrs, clear, nb, +1)
        tptrs = (u64p * max(zt, 1))()
        tclear = (ctypes.c_int * max(zt, 1))()
        for i in range(zt):
            d = int(self.ram_bits[j][i])
            tptrs[i] = _p64(rgsw_by_slot[P.L + d]) if d >= 0 else ctypes.cast(None, u64p)
        out = {}
        for c in range(self.cfg.n_classes):
            prods = []
            Lin = (u64p * (1 << zt))()
            for v, t in enumerate(self.plain_tables(W, j, c)):
                pr = np.zeros(self.rlwe_words, dtype=np.uint64)
                lib().or_rlwe_mul_plain(self.ctx, _p64(acc),
                                        t.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _p64(pr))
                prods.append(pr)
                Lin[v] = _p64(pr)
            lwe = np.zeros(P.r * (P.n + 1), dtype=np.uint64)
            lib().or_vp(self.ctx, Lin, tptrs, tclear, zt, zt, _p64(lwe))
            out[c] = lwe
        return out

    def infer_plain(self, W, s, seed, data_bits, rams=None, sample_offset=0, trivial=False):
        """Inference against the clear counters W[c][j][addr] (Algorithm 4's
        model): responses u[i][c][j] and per-class sums, laid out as infer()."""
        P = self.P
        l = self.cfg.n_classes
        rams = list(range(P.k0)) if rams is None else list(rams)
        slots = self.slots_for_rams(rams, with_labels=False)
        n = data_bits.shape[0]
        lw = P.r * (P.n + 1)
        resp = np.zeros((n, l, len(rams), lw), dtype=np.uint64)
        sums = np.zeros((n, l, lw), dtype=np.uint64)
        for i in range(n):
            rg = self.encrypt_slots(s, seed, sample_offset + i, data_bits[i], 0, slots, trivial)
            for jj, j in enumerate(rams):
                for c, lwe in self.vp_plain_item(W, rg, j).items():
                    resp[i, c, jj] = lwe
            for c in range(l):
                for jj in range(len(rams)):
                    lib().or_lwe_add(self.ctx, _p64(sums[i, c]), _p64(np.ascontiguousarray(resp[i, c, jj])))
        return resp, sums

    def infer(self, H, s, seed, data_bits, rams=None, sample_offset=0, trivial=False):
        """Algorithm 7 (PD-act): responses u[i][c][j] as LWE ciphertexts and
        the per-class sums over the listed RAMs."""
        P = self.P
        l = self.cfg.n_classes
        rams = list(range(P.k0)) if rams is None else list(rams)
        slots = self.slots_for_rams(rams, with_labels=False)
        n = data_bits.shape[0]
        lw = P.r * (P.n + 1)
        resp = np.zeros((n, l, len(rams), lw), dtype=np.uint64)
        sums = np.zeros((n, l, lw), dtype=np.uint64)
        for i in range(n):
            rg = self.encrypt_slots(s, seed, sample_offset + i, data_bits[i], 0, slots, trivial)
            for jj, j in enumerate(rams):
                for c in range(l):
                    resp[i, c, jj] = self.vp_item(H, rg, j, c)
                    lib().or_lwe_add(self.ctx, _p64(sums[i, c]), _p64(resp[i, c, jj]))
        return resp, sums

    # ---------------------------------------------------------- decryption
    def crt(self, residues):
        P = self.P
        phi = 0
        for j in range(P.r):
            Mj = P.Q // P.q[j]
            phi += int(residues[j]) * Mj * pow(Mj % P.q[j], -1, P.q[j])
        return phi % P.Q

    def decode(self, residues) -> int:
        P = self.P
        phi = self.crt(residues)
        return ((P.p * phi + P.Q // 2) // P.Q) % P.p

    def rlwe_phase(self, s, ct) -> np.ndarray:
        P = self.P
        ph = np.zeros(P.r * P.n, dtype=np.uint64)
        lib().or_rlwe_phase(self.ctx, s.ctypes.data_as(i8p), _p64(np.ascontiguousarray(ct)), _p64(ph))
        return ph.reshape(P.r, P.n)

    def decrypt_rlwe(self, s, ct) -> np.ndarray:
        ph = self.rlwe_phase(s, ct)
        return np.array([self.decode(ph[:, k]) for k in range(self.P.n)], dtype=np.int64)

    def decrypt_lwe(self, s, lwe) -> int:
        P = self.P
        ph = np.zeros(P.r, dtype=np.uint64)
        lib().or_lwe_phase(self.ctx, s.ctypes.data_as(i8p), _p64(np.ascontiguousarray(lwe)), _p64(ph))
        return self.decode(ph)

    def decrypt_model(self, s, H, rams=None) -> np.ndarray:
        """Counters W[c][j][addr] from H, for the listed RAMs (others 0)."""
        P = self.P
        rams = list(range(P.k0)) if rams is None else list(rams)
        W = np.zeros((self.cfg.n_classes, P.k0, 1 << P.a), dtype=np.int64)
        for j in rams:
            dec = {v: self.decrypt_rlwe(s, H[j, P.slot[v]]) for v in P.V}
            for c in range(self.cfg.n_classes):
                for addr in range(1 << P.a):
                    m = c + (addr << P.L)
                    W[c, j, addr] = dec[m % (1 << P.z)][m >> P.z]
        return W
