"""Dataset balancing (Section 3.6.1) on the GPU against the oracle: the
class-count ciphertext bit for bit, its decryption equal to the class
histogram, and balanced PD-act labels equal to the oracle's.  Integer
results: tolerance 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset
from test_gpu_parity import tiny_cfg, u64

pytestmark = pytest.mark.gpu


def _session(cfg, geometry=None):
    from paper_2403_20190_gb300.session import Session
    return Session(cfg, 0, geometry=geometry)


@pytest.mark.parametrize("name,geometry", [("zL", None), ("zgtL", None), ("zltL_h3", dict(ext_smem=1)),
                                           ("r2_beta1024", dict(ext_loge=4, ext_np=1, ext_smem=2))])
def test_count_ciphertext_and_balanced_labels_tiny(name, geometry):
    cfg = tiny_cfg(name)
    o = Oracle(cfg)
    P = o.P
    n_tr, n_te = 7, 4
    vals, labels = make_dataset(cfg, "train", n=n_tr)
    tvals, _ = make_dataset(cfg, "test", n=n_te)
    s = _session(cfg, geometry)
    dev = s.device
    key = s.keygen(21)
    bits = s.encode(torch.from_numpy(vals).to(dev))
    rg = s.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=31)
    counts = s.count_classes(s.new_counts(), rg, 4)
    s.count_classes(counts, rg[4 * s.sz["sample_words"]:], n_tr - 4)  # two batches add up
    model = s.train(s.new_model(), rg, n_tr)
    tb = s.encode(torch.from_numpy(tvals).to(dev))
    resp, _ = s.infer(model, s.encrypt(key, tb, None, seed=41), n_te)
    cc = s.class_counts(key, counts)
    u = s.responses_counts(key, resp, n_te)
    _, lab = s.pdact_balanced(u.contiguous(), cc, n_te)
    torch.cuda.synchronize()
    sk = o.keygen(21)
    ref = o.count_classes(np.zeros(o.rlwe_words, dtype=np.uint64), sk, 31, labels)
    assert np.array_equal(u64(counts), ref)
    hist = np.bincount(labels, minlength=cfg.n_classes)
    assert np.array_equal(cc.cpu().numpy(), hist)
    obits = wisard.encode(P, vals)
    W = wisard.integer_wisard_train(P, obits, labels)
    _, olab = wisard.balanced_pdact(cfg, wisard.lookups(P, W, wisard.encode(P, tvals)), hist)
    assert np.array_equal(lab.cpu().numpy(), olab)


def test_skewed_workload_counts():
    """cfg4's skewed priors: counts of a 24-sample batch decrypt to its histogram."""
    cfg = get_config("cfg4")
    s = _session(cfg)
    n = 3
    vals, labels = make_dataset(cfg, "train", n=n)
    key = s.keygen(5)
    bits = s.encode(torch.from_numpy(vals).to(s.device))
    rg = s.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(s.device), seed=77)
    counts = s.new_counts()
    for _ in range(8):  # the same encrypted batch counted 8 times: 24 samples
        s.count_classes(counts, rg, n)
    cc = s.class_counts(key, counts)
    torch.cuda.synchronize()
    assert np.array_equal(cc.cpu().numpy(), 8 * np.bincount(labels, minlength=cfg.n_classes))
