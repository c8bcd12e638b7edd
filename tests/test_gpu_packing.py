"""Horizontal packing (Section 6) on the GPU against the oracle: packed
responses and class sums bit for bit, decrypting to the plaintext lookups;
a tree level on an encrypted address bit (z > L) falls back to plain VP.
Integer results: tolerance 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config
from test_gpu_parity import TINY, run_pipeline, tiny_cfg, u64

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", list(TINY))
def test_tiny_packed_responses(name):
    cfg = tiny_cfg(name)
    o = Oracle(cfg)
    P = o.P
    R = run_pipeline(cfg, 7, 3)
    s = R["sess"]
    # packed inference on the same model and encrypted test batch
    resp, sums = s.infer(R["model"], R["trg"], 3, packed=True)
    torch.cuda.synchronize()
    sk = o.keygen(21)
    obits = wisard.encode(P, R["vals"])
    H = o.train(o.new_model(), sk, 31, obits, R["labels"])
    otb = wisard.encode(P, R["tvals"])
    oresp, osums = o.infer_packed(H, sk, 41, otb)
    assert np.array_equal(u64(resp).reshape(oresp.shape), oresp)
    assert np.array_equal(u64(sums).reshape(osums.shape), osums)
    W = wisard.integer_wisard_train(P, obits, R["labels"])
    dec = s.responses_counts(R["key"], resp, 3).cpu().numpy()
    assert np.array_equal(dec, wisard.lookups(P, W, otb))
    if not o.packing_groups():  # z > L: plain VP
        assert torch.equal(resp, R["resp"])


@pytest.mark.parametrize("name,rams,n_test", [("cfg1", [0, 17, 29], 1), ("cfg3", [5, 146], 2)])
def test_workload_packed_sampled(name, rams, n_test):
    """Two cfg3 test samples: the batch path that transforms the first
    CMUX's digits once for both."""
    cfg = get_config(name)
    o = Oracle(cfg)
    P = o.P
    R = run_pipeline(cfg, 2, n_test)
    s = R["sess"]
    resp, _ = s.infer(R["model"], R["trg"], n_test, packed=True)
    torch.cuda.synchronize()
    sk = o.keygen(21)
    obits = wisard.encode(P, R["vals"])
    H = o.train(o.new_model(), sk, 31, obits, R["labels"], rams=rams)
    oresp, _ = o.infer_packed(H, sk, 41, wisard.encode(P, R["tvals"]), rams=rams)
    gresp = u64(resp).reshape(n_test, cfg.n_classes, P.k0, -1)
    assert np.array_equal(gresp[:, :, rams], oresp)
