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
    "cfg3": {},
}
BASE = {"tiny_tree": "cfg1", "cfg2": "cfg2", "cfg3": "cfg3"}
# per-block stride of the static array: 3 RLWEs (evaluation form in global
# memory, ext_smem 0) or 2 (ext_smem 1)
GEOMETRIES = {"smem0": dict(ext_loge=3, ext_np=2, ext_smem=0),
              "smem1": dict(ext_loge=3, ext_np=2, ext_smem=1)}


def _setup(name, n_train, n_test, geometry=None):
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.session import Session
    build.build()
    cfg = get_config(BASE[name], **CASES[name])
    sess = Session(cfg, 0, geometry=GEOMETRIES.get(geometry))
    dev = sess.device
    vals, labels = make_dataset(cfg, "train", n=n_train)
    tvals, _ = make_dataset(cfg, "test", n=n_test)
    key = sess.keygen(5)
    bits = sess.encode(torch.from_numpy(vals).to(dev))
    rg = sess.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=9)
    model = sess.train(sess.new_model(), rg, n_train)
    del rg
    tbits = sess.encode(torch.from_numpy(tvals).to(dev))
    trg = sess.encrypt(key, tbits, None, seed=11)
    return sess, model, trg


def _check_twice(sess, model, trg, n_test):
    from paper_2403_20190_gb300 import binding as B
    ref_resp, ref_sums = sess.infer(model, trg, n_test)
    for _ in range(2):
        resp = torch.full_like(ref_resp, -1)
        sums = torch.full_like(ref_sums, -1)
        B.hw_infer_static_scratch(sess.ctx, model, trg, n_test, resp, sums)
        torch.cuda.synchronize()
        assert torch.equal(resp, ref_resp)
        assert torch.equal(sums, ref_sums)


@pytest.mark.parametrize("geometry", sorted(GEOMETRIES))
def test_static_scratch_tiny_ring_both_strides(geometry):
    sess, model, trg = _setup("tiny_tree", 5, 3, geometry)
    assert sess.geometry["ext_smem"] == GEOMETRIES[geometry]["ext_smem"]
    _check_twice(sess, model, trg, 3)


def test_static_scratch_cfg2():
    sess, model, trg = _setup("cfg2", 2, 2)
    _check_twice(sess, model, trg, 2)


def test_static_scratch_capped_grid_cfg3():
    """N = 8192 with three 55-bit primes: one block takes 1.18 MB of the
    48 MiB array, so fewer blocks run than the persistent grid has."""
    sess, model, trg = _setup("cfg3", 1, 1)
    sz = sess.sz
    per_block = (3 if sess.geometry["ext_smem"] == 0 else 2) * sz["rlwe_words"] * 8
    assert (48 << 20) // per_block < torch.cuda.get_device_properties(0).multi_processor_count
    _check_twice(sess, model, trg, 1)


def test_static_scratch_empty_batch_is_a_no_op():
    from paper_2403_20190_gb300 import binding as B
    sess, model, trg = _setup("tiny_tree", 2, 1)
    resp = torch.full((sess.sz["resp_words"],), -1, dtype=torch.int64, device=sess.device)
    sums = torch.full((sess.sz["sums_words"],), -1, dtype=torch.int64, device=sess.device)
    B.hw_infer_static_scratch(sess.ctx, model, trg, 0, resp, sums)
    torch.cuda.synchronize()
    assert (resp == -1).all() and (sums == -1).all()
