"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

Small cases cover every tree shape of the workloads on tiny rings; the four
workload parameter sets are checked on the oracle's sampled outputs (chosen
RAMs, a few samples), and at batch size with properties that hold at any
size: decrypted counters equal the Integer WiSARD counts (Algorithm 4) and
PD-act labels equal the plaintext labels.  Integer work: tolerance 0.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset

pytestmark = pytest.mark.gpu


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2403_20190_gb300 import binding, build
    build.build()
    binding.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def session(cfg, geometry=None):
    from paper_2403_20190_gb300.session import Session
    return Session(cfg, 0, geometry=geometry)


# every tree shape of the workloads on N = 64 rings (the smallest ring the
# CUDA path supports)
TINY = {
    # z = 0: label bit among the rotation bits; base-32 gadget; short last tuple
    "z0": dict(log_n=6, n_primes=1, prime_bits=30, log_beta=5, log_p=8, n_classes=2,
               n_values=5, therm_bits=2, addr_bits=3, tuple_bits=3),
    # z = L: the tree holds exactly the label bits; short last tuple
    "zL": dict(log_n=6, n_primes=2, prime_bits=50, log_beta=0, log_p=16, n_classes=3,
               n_values=7, therm_bits=2, addr_bits=6, tuple_bits=6),
    # z < L: a label bit among the rotation bits; hashed tuples
    "zltL_h3": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=20, n_classes=5,
                    n_values=4, therm_bits=3, addr_bits=5, tuple_bits=8, hash_h3=1),
    # z > L: an address bit in the tree; the last RAM has only that bit
    "zgtL": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3,
                 n_values=4, therm_bits=2, addr_bits=7, tuple_bits=7),
    # several digits per prime over two primes
    "r2_beta1024": dict(log_n=6, n_primes=2, prime_bits=30, log_beta=10, log_p=12, n_classes=4,
                        n_values=6, therm_bits=2, addr_bits=3, tuple_bits=3),
}


def tiny_cfg(name):
    return get_config("cfg1", data_kind="uniform", act="log", act_arg=0, **TINY[name])


def run_pipeline(cfg, n_train, n_test, seed_tr=31, seed_te=41, key_seed=21, geometry=None):
    sess = session(cfg, geometry)
    dev = sess.device
    vals, labels = make_dataset(cfg, "train", n=n_train)
    tvals, _ = make_dataset(cfg, "test", n=n_test)
    key = sess.keygen(key_seed)
    bits = sess.encode(torch.from_numpy(vals).to(dev))
    rg = sess.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=seed_tr)
    model = sess.new_model()
    sess.train(model, rg, n_train)
    tbits = sess.encode(torch.from_numpy(tvals).to(dev))
    trg = sess.encrypt(key, tbits, None, seed=seed_te)
    resp, sums = sess.infer(model, trg, n_test)
    torch.cuda.synchronize()
    return dict(sess=sess, key=key, vals=vals, labels=labels, tvals=tvals, bits=bits, tbits=tbits,
                rg=rg, trg=trg, model=model, resp=resp, sums=sums)


@pytest.mark.parametrize("name", list(TINY))
def test_tiny_rings_full_parity(name):
    tiny_full_parity(name, None)


def tiny_full_parity(name, geometry):
    cfg = tiny_cfg(name)
    o = Oracle(cfg)
    P = o.P
    R = run_pipeline(cfg, 7, 3, geometry=geometry)
    sess = R["sess"]
    s = o.keygen(21)
    # key
    key = u64(R["key"]).reshape(2, P.r, P.n)
    for j in range(P.r):
        assert [int(v) for v in key[0, j]] == [int(x) % P.q[j] for x in s]
    # client encoding
    obits = wisard.encode(P, R["vals"])
    assert np.array_equal(R["bits"].cpu().numpy(), obits)
    # encryption (every slot of sample 1, canonical form)
    exp = u64(sess.export_rgsw(R["rg"], 7 * P.n_slots)).reshape(7, P.n_slots, -1)
    for b in range(P.n_slots):
        val = (int(R["labels"][1]) >> b) & 1 if b < P.L else int(obits[1, b - P.L])
        ref = o.export_rgsw(o.encrypt_bit(s, 31, 1 * P.n_slots + b, val))
        assert np.array_equal(exp[1, b], ref), f"RGSW slot {b}"
    # training: whole model
    H = o.train(o.new_model(), s, 31, obits, R["labels"])
    assert np.array_equal(u64(R["model"]).reshape(H.shape), H)
    # inference: responses and class sums
    otb = wisard.encode(P, R["tvals"])
    oresp, osums = o.infer(H, s, 41, otb)
    assert np.array_equal(u64(R["resp"]).reshape(oresp.shape), oresp)
    assert np.array_equal(u64(R["sums"]).reshape(osums.shape), osums)
    # decryption and PD-act
    W = wisard.integer_wisard_train(P, obits, R["labels"])
    dec = sess.decrypt_model_counts(R["key"], R["model"]).cpu().numpy()
    assert np.array_equal(dec, o.decrypt_model(s, H))  # HW_DEC_MODEL, element by element
    assert np.array_equal(dec, W)
    counts = sess.responses_counts(R["key"], R["resp"], 3)
    assert np.array_equal(counts.cpu().numpy(), wisard.lookups(P, W, otb))
    sums_dec = sess.decrypt_lwe(R["key"], R["sums"], 3 * cfg.n_classes).view(3, cfg.n_classes)
    assert np.array_equal(sums_dec.cpu().numpy(), wisard.lookups(P, W, otb).sum(axis=2))
    _, lab = sess.pdact(counts.contiguous(), 3)
    assert np.array_equal(lab.cpu().numpy(), wisard.evaluate(P, W, otb)[1])


def test_ntt_roundtrip_and_edge_values():
    cfg = get_config("cfg3")
    sess = session(cfg)
    sz = sess.sz
    n, r = sz["n"], sz["r"]
    count = 3 * r + 1  # ragged: polynomial t uses prime t mod r
    rng = np.random.default_rng(0)
    x = np.zeros((count, n), dtype=np.uint64)
    for t in range(count):
        q = sz["q"][t % r]
        x[t] = rng.integers(0, q, size=n, dtype=np.uint64)
    x[0, :4] = [0, sz["q"][0] - 1, (sz["q"][0] - 1) // 2, 1]
    dev = torch.from_numpy(x.view(np.int64)).to(sess.device)
    from paper_2403_20190_gb300 import binding as B
    B.hw_ntt_forward(sess.ctx, dev, count)
    fwd = u64(dev).reshape(count, n).copy()
    assert not np.array_equal(fwd, x)
    for t in range(count):
        assert (fwd[t] < sz["q"][t % r]).all()
    B.hw_ntt_inverse(sess.ctx, dev, count)
    assert np.array_equal(u64(dev).reshape(count, n), x)


@pytest.mark.parametrize("name,ntt_loge", [("cfg1", 4), ("cfg1", 3), ("z0", 4), ("z0", 3)])
def test_ntt_bulk_pipeline_equals_one_block_per_polynomial(name, ntt_loge):
    """The bulk-copy pipeline of the 32-bit transform (16-byte aligned
    buffers: persistent blocks, several polynomials each through two
    alternating stages) against the one-block-per-polynomial form (the same
    data 8 bytes off that alignment), both directions, radix 16 and 8, on
    cfg1's ring and on a 64-point ring (blocks smaller than a warp); the
    count leaves a ragged last round of the grid."""
    from paper_2403_20190_gb300 import binding as B
    cfg = tiny_cfg(name) if name in TINY else get_config(name)
    sess = session(cfg, dict(ntt_loge=ntt_loge, ntt_limbs=1))
    assert (sess.geometry["ntt_loge"], sess.geometry["ntt_limbs"]) == (ntt_loge, 1)
    sz = sess.sz
    n, r = sz["n"], sz["r"]
    count = 3 * 152 * 32 + 5  # more than the persistent grid holds at once
    rng = np.random.default_rng(7)
    x = np.zeros((count, n), dtype=np.uint64)
    for t in range(count):
        x[t] = rng.integers(0, sz["q"][t % r], size=n, dtype=np.uint64)
    flat = torch.from_numpy(x.reshape(-1).view(np.int64)).to(sess.device)
    buf = torch.zeros(count * n + 2, dtype=torch.int64, device=sess.device)
    aligned = buf[:count * n]
    shifted = buf.new_zeros(count * n + 2)[1:1 + count * n]
    assert aligned.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 8
    aligned.copy_(flat)
    shifted.copy_(flat)
    B.hw_ntt_forward(sess.ctx, aligned, count)
    B.hw_ntt_forward(sess.ctx, shifted, count)
    torch.cuda.synchronize()
    assert torch.equal(aligned, shifted)
    assert not torch.equal(aligned, flat)
    B.hw_ntt_inverse(sess.ctx, aligned, count)
    B.hw_ntt_inverse(sess.ctx, shifted, count)
    torch.cuda.synchronize()
    assert torch.equal(aligned, flat) and torch.equal(shifted, flat)
    B.hw_check_context(sess.ctx)  # no bulk-copy wait ran out


def _library_root(q, log_n):
    """The library's documented root choice: psi = x^((q-1)/2N) for the
    first odd x >= 3 with psi^N = -1."""
    n = 1 << log_n
    x = 3
    while True:
        psi = pow(x, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi
        x += 2


@pytest.mark.parametrize("name,ntt_loge,ntt_limbs", [
    ("cfg1", 4, 1), ("cfg1", 3, 1), ("cfg1", 4, 2), ("cfg1", 3, 2),
    ("cfg2", 4, 2), ("cfg2", 3, 2), ("cfg4", 4, 2), ("cfg4", 3, 2)])
def test_ntt_is_evaluation_at_odd_powers(name, ntt_loge, ntt_limbs):
    """Every batched-transform variant (radix 8 or 16; 32-bit arithmetic for
    cfg1's 30-bit prime, 64-bit everywhere) puts a(psi^(2 brv(pos) + 1)) at
    position pos, and its inverse undoes it."""
    from paper_2403_20190_gb300 import binding as B
    cfg = get_config(name)
    sess = session(cfg, dict(ntt_loge=ntt_loge, ntt_limbs=ntt_limbs))
    assert (sess.geometry["ntt_loge"], sess.geometry["ntt_limbs"]) == (ntt_loge, ntt_limbs)
    sz = sess.sz
    n, r, log_n = sz["n"], sz["r"], cfg.log_n
    rng = np.random.default_rng(1)
    x = np.zeros((r, n), dtype=np.uint64)
    for j in range(r):
        x[j] = rng.integers(0, sz["q"][j], size=n, dtype=np.uint64)
    dev = torch.from_numpy(x.view(np.int64).copy()).to(sess.device)
    B.hw_ntt_forward(sess.ctx, dev, r)
    out = u64(dev).reshape(r, n)
    for j in range(r):
        q = sz["q"][j]
        psi = _library_root(q, log_n)
        a = [int(v) for v in x[j]]
        for pos in (0, 1, n // 2 + 3, n - 1):
            b = int(format(pos, f"0{log_n}b")[::-1], 2)
            w = pow(psi, 2 * b + 1, q)
            acc, p = 0, 1
            for c in a:
                acc = (acc + c * p) % q
                p = p * w % q
            assert int(out[j, pos]) == acc
    B.hw_ntt_inverse(sess.ctx, dev, r)
    assert np.array_equal(u64(dev).reshape(r, n), x)


@pytest.mark.parametrize("name,n_train,n_test,rams", [
    ("cfg1", 6, 3, [0, 13, 29]),
    ("cfg2", 3, 2, [0, 77, 130]),
    ("cfg3", 2, 2, [5, 146]),
    ("cfg4", 2, 2, [0, 503]),
])
def test_workload_parameters_sampled_parity(name, n_train, n_test, rams):
    """Real ring sizes and primes: RGSW rows, trained model rows and
    inference responses on chosen RAMs (the last RAM included) bit-exact."""
    workload_sampled_parity(name, n_train, n_test, rams, None)


def workload_sampled_parity(name, n_train, n_test, rams, geometry):
    cfg = get_config(name)
    o = Oracle(cfg)
    P = o.P
    R = run_pipeline(cfg, n_train, n_test, geometry=geometry)
    sess = R["sess"]
    s = o.keygen(21)
    obits = wisard.encode(P, R["vals"])
    assert np.array_equal(R["bits"].cpu().numpy(), obits)
    # one label slot and one data slot of the last sample, canonical form
    i = n_train - 1
    for b in (0, P.n_slots - 1):
        exp = u64(sess.export_rgsw(R["rg"][(i * P.n_slots + b) * sess.sz["rgsw_words"]:
                                         (i * P.n_slots + b + 1) * sess.sz["rgsw_words"]], 1))
        val = (int(R["labels"][i]) >> b) & 1 if b < P.L else int(obits[i, b - P.L])
        ref = o.export_rgsw(o.encrypt_bit(s, 31, i * P.n_slots + b, val))
        assert np.array_equal(exp, ref), f"RGSW slot {b}"
    H = o.train(o.new_model(), s, 31, obits, R["labels"], rams=rams)
    gH = u64(R["model"]).reshape(H.shape)
    assert np.array_equal(gH[rams], H[rams])
    otb = wisard.encode(P, R["tvals"])
    oresp, _ = o.infer(H, s, 41, otb, rams=rams)
    gresp = u64(R["resp"]).reshape(n_test, cfg.n_classes, P.k0, -1)
    assert np.array_equal(gresp[:, :, rams], oresp)


@pytest.mark.parametrize("name,n_train,n_test", [("cfg1", 200, 100), ("cfg2", 64, 32), ("cfg3", 16, 16),
                                                  ("cfg4", 4, 4)])
def test_batch_invariants(name, n_train, n_test):
    """At batch size (cfg3 and cfg4: the bench's batches): decrypted
    counters == Algorithm 4 counts for every RAM, decrypted responses ==
    plaintext lookups, class sums == Algorithm 2 scores (cfg2-4; cfg1's
    30-bit modulus leaves class sums undecodable by design), PD-act labels
    == plaintext labels."""
    cfg = get_config(name)
    o = Oracle(cfg)
    P = o.P
    R = run_pipeline(cfg, n_train, n_test)
    sess = R["sess"]
    obits = wisard.encode(P, R["vals"])
    W = wisard.integer_wisard_train(P, obits, R["labels"])
    assert np.array_equal(sess.decrypt_model_counts(R["key"], R["model"]).cpu().numpy(), W)
    otb = wisard.encode(P, R["tvals"])
    counts = sess.responses_counts(R["key"], R["resp"], n_test)
    assert np.array_equal(counts.cpu().numpy(), wisard.lookups(P, W, otb))
    if name != "cfg1":
        sd = sess.decrypt_lwe(R["key"], R["sums"], n_test * cfg.n_classes).view(n_test, -1)
        assert np.array_equal(sd.cpu().numpy(), wisard.lookups(P, W, otb).sum(axis=2))
    _, lab = sess.pdact(counts.contiguous(), n_test)
    assert np.array_equal(lab.cpu().numpy(), wisard.evaluate(P, W, otb)[1])


def test_empty_batches_and_scratch_checks():
    from paper_2403_20190_gb300 import binding as B
    cfg = tiny_cfg("zL")
    sess = session(cfg)
    model = sess.new_model()
    empty = sess.words(1)
    B.hw_train_accumulate(sess.ctx, model, empty, 0, empty)
    assert not model.any()
    key = sess.keygen(1)
    bits = torch.zeros((2, sess.sz["n_data"]), dtype=torch.uint8, device=sess.device)
    rg = sess.encrypt(key, bits, torch.zeros(2, dtype=torch.int32, device=sess.device), seed=1)
    small = sess.words(B.hw_train_scratch_words(sess.ctx, 2) - 1)
    with pytest.raises(B.HwError):
        B.hw_train_accumulate(sess.ctx, model, rg, 2, small)


def test_split_batches_equal_one_batch():
    """Training in two calls equals training in one (addition mod q is
    associative): the batched path is bit-identical to sequential calls."""
    cfg = tiny_cfg("zgtL")
    sess = session(cfg)
    dev = sess.device
    vals, labels = make_dataset(cfg, "train", n=6)
    key = sess.keygen(3)
    bits = sess.encode(torch.from_numpy(vals).to(dev))
    lab = torch.from_numpy(labels.astype(np.int32)).to(dev)
    rg = sess.encrypt(key, bits, lab, seed=5)
    one = sess.train(sess.new_model(), rg, 6)
    two = sess.new_model()
    sw = sess.sz["sample_words"]
    sess.train(two, rg[:4 * sw], 4)
    sess.train(two, rg[4 * sw:], 2)
    torch.cuda.synchronize()
    assert torch.equal(one, two)
