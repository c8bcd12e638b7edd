"""hw_infer_static_scratch: inference for callers that cannot allocate device
memory (for example a plug-in that only receives a request's input and
output buffers, or a request loop that may not call cudaMalloc).  Its
per-block accumulators live in the library's static device array instead of
a caller-provided scratch buffer.

Checked through the C ABI against hw_infer on the same inputs, twice in a
row (the array keeps the previous call's contents), bit for bit: the path is
integer arithmetic, so the tolerance is zero.  This file is collected last so
that a run stopping at the first failure has already run every other test;
it also passes alone in a fresh process (the first call on the device looks
up the array's address).
"""
import numpy as np
import pytest
import torch

from synthdata import get_config, make_dataset

pytestmark = pytest.mark.gpu

CASES = {
    "tiny_tree": dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3,
                      n_values=4, therm_bits=2, addr_bits=7, tuple_bits=7, data_kind="uniform",
                      act="log", act_arg=0),
    "cfg2": {},
}


def _setup(name, n_train, n_test):
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.session import Session
    build.build()
    cfg = get_config("cfg2" if name == "cfg2" else "cfg1", **CASES[name])
    sess = Session(cfg, 0)
    dev = sess.device
    vals, labels = make_dataset(cfg, "train", n=n_train)
    tvals, _ = make_dataset(cfg, "test", n=n_test)
    key = sess.keygen(5)
    bits = sess.encode(torch.from_numpy(vals).to(dev))
    rg = sess.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=9)
    model = sess.train(sess.new_model(), rg, n_train)
    tbits = sess.encode(torch.from_numpy(tvals).to(dev))
    trg = sess.encrypt(key, tbits, None, seed=11)
    return sess, model, trg


@pytest.mark.parametrize("name,n_train,n_test", [("tiny_tree", 5, 3), ("cfg2", 2, 2)])
def test_static_scratch_inference_matches_hw_infer(name, n_train, n_test):
    from paper_2403_20190_gb300 import binding as B
    sess, model, trg = _setup(name, n_train, n_test)
    ref_resp, ref_sums = sess.infer(model, trg, n_test)
    for _ in range(2):
        resp = torch.full_like(ref_resp, -1)
        sums = torch.full_like(ref_sums, -1)
        B.hw_infer_static_scratch(sess.ctx, model, trg, n_test, resp, sums)
        torch.cuda.synchronize()
        assert torch.equal(resp, ref_resp)
        assert torch.equal(sums, ref_sums)


def test_static_scratch_empty_batch_is_a_no_op():
    from paper_2403_20190_gb300 import binding as B
    sess, model, trg = _setup("tiny_tree", 2, 1)
    resp = torch.full((sess.sz["resp_words"],), -1, dtype=torch.int64, device=sess.device)
    sums = torch.full((sess.sz["sums_words"],), -1, dtype=torch.int64, device=sess.device)
    B.hw_infer_static_scratch(sess.ctx, model, trg, 0, resp, sums)
    torch.cuda.synchronize()
    assert (resp == -1).all() and (sums == -1).all()
