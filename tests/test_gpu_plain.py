"""Unencrypted-model inference (Section 3.6.2) on the GPU against the oracle:
responses and class sums bit for bit on every tree shape (the address bit
of z > L in a CMUX), in several kernel geometries, decrypting to the
plaintext lookups; sampled RAMs at the workloads' ring sizes; and at batch
size, a model trained and decrypted on the GPU answers through its clear
tables with the plaintext lookups, scores and labels.  Integer results:
tolerance 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset
from test_gpu_parity import TINY, run_pipeline, session, tiny_cfg, u64

pytestmark = pytest.mark.gpu


def _random_counts(P, l, seed, hi):
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(l, P.k0, 1 << P.a)).astype(np.int64)


def _plain_case(cfg, geometry, n_test, hi, rams=None):
    o = Oracle(cfg)
    P = o.P
    sess = session(cfg, geometry)
    dev = sess.device
    key = sess.keygen(21)
    tvals, _ = make_dataset(cfg, "test", n=n_test)
    trg = sess.encrypt(key, sess.encode(torch.from_numpy(tvals).to(dev)), None, seed=41)
    W = _random_counts(P, cfg.n_classes, 5, hi)
    plain = sess.plain_model(torch.from_numpy(W).to(dev))
    resp, sums = sess.infer_plain(plain, trg, n_test)
    torch.cuda.synchronize()
    otb = wisard.encode(P, tvals)
    oresp, osums = o.infer_plain(W, o.keygen(21), 41, otb, rams=rams)
    gresp = u64(resp).reshape(n_test, cfg.n_classes, P.k0, -1)
    if rams is None:
        assert np.array_equal(gresp, oresp)
        assert np.array_equal(u64(sums).reshape(osums.shape), osums)
    else:
        assert np.array_equal(gresp[:, :, rams], oresp)
    dec = sess.responses_counts(key, resp, n_test).cpu().numpy()
    assert np.array_equal(dec, wisard.lookups(P, W, otb))
    return sess


@pytest.mark.parametrize("geometry", [None, dict(ext_loge=4, ext_np=1), dict(ext_loge=3, ext_np=2, ext_smem=1),
                                      dict(ext_loge=2, ext_np=2), dict(ext_loge=4, ext_np=1, ext_smem=2)])
@pytest.mark.parametrize("name", list(TINY))
def test_tiny_plain_responses(name, geometry):
    _plain_case(tiny_cfg(name), geometry, 3, 4)


@pytest.mark.parametrize("name,rams,geometry", [
    ("cfg1", [0, 13, 29], None),
    ("cfg2", [0, 77, 130], dict(ext_loge=3, ext_np=2, ext_smem=1)),
    ("cfg2", [5, 130], dict(ext_loge=2, ext_np=1)),
    ("cfg4", [0, 503], None),
])
def test_workload_plain_sampled(name, rams, geometry):
    """Real rings: cfg1 (base-32 gadget, so the rotated accumulator is
    transformed again), cfg2 (one digit per prime) and cfg4 (z > L: the
    CMUX of address bit 0 over the two half tables)."""
    _plain_case(get_config(name), geometry, 1, 3, rams)


def test_trained_model_in_clear_at_batch_size():
    """A model trained on the GPU and decrypted by its owner, answered in
    clear: counters, lookups, Algorithm 2 scores and PD-act labels all equal
    the plaintext Integer WiSARD's."""
    cfg = get_config("cfg2")
    P = Oracle(cfg).P
    R = run_pipeline(cfg, 64, 32)
    sess = R["sess"]
    W = sess.decrypt_model_counts(R["key"], R["model"])
    obits = wisard.encode(P, R["vals"])
    Wref = wisard.integer_wisard_train(P, obits, R["labels"])
    assert np.array_equal(W.cpu().numpy(), Wref)
    plain = sess.plain_model(W)
    resp, sums = sess.infer_plain(plain, R["trg"], 32)
    otb = wisard.encode(P, R["tvals"])
    counts = sess.responses_counts(R["key"], resp, 32)
    assert np.array_equal(counts.cpu().numpy(), wisard.lookups(P, Wref, otb))
    sd = sess.decrypt_lwe(R["key"], sums, 32 * cfg.n_classes).view(32, -1)
    assert np.array_equal(sd.cpu().numpy(), wisard.lookups(P, Wref, otb).sum(axis=2))
    _, lab = sess.pdact(counts.contiguous(), 32)
    assert np.array_equal(lab.cpu().numpy(), wisard.evaluate(P, Wref, otb)[1])


def test_plain_argument_checks():
    from paper_2403_20190_gb300 import binding as B
    cfg = tiny_cfg("zL")
    sess = session(cfg)
    P = Oracle(cfg).P
    W = torch.zeros((cfg.n_classes, P.k0, 1 << P.a), dtype=torch.int64, device=sess.device)
    plain = sess.plain_model(W)
    resp, sums, scratch = sess.infer_buffers(2)
    rg = sess.words(2 * sess.sz["sample_words"])
    B.hw_infer_plain(sess.ctx, plain, rg, 0, resp, sums, scratch)  # empty batch: nothing to do
    # inference against a clear model needs the persistent blocks' buffers
    # only (hw_infer's scratch for one sample)
    with pytest.raises(B.HwError):
        B.hw_infer_plain(sess.ctx, plain, rg, 2, resp, sums, scratch[:B.hw_infer_scratch_words(sess.ctx, 1) - 1])
    assert B.hw_plain_model_words(sess.ctx) == cfg.n_classes * P.k0 * P.r * P.n
