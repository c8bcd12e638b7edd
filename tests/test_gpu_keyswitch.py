"""PackingKeySwitching (Section 2.4) on the GPU: the packed RLWE of every
test sample bit for bit against the oracle (tiny rings, a cfg1 sample), and
at cfg2's size its decryption equal to the decrypted LWE responses it packs.
Integer results: tolerance 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config
from test_gpu_parity import TINY, run_pipeline, tiny_cfg, u64

pytestmark = pytest.mark.gpu


def _check_against_oracle(cfg, R, n_test):
    o = Oracle(cfg)
    P = o.P
    s = R["sess"]
    ksk = s.ksk_gen(R["key"], 77)
    packed = s.pack_responses(ksk, R["resp"], n_test)
    torch.cuda.synchronize()
    sk = o.keygen(21)
    oksk = o.ksk_gen(sk, 77)
    resp = u64(R["resp"]).reshape(n_test, -1, P.r * (P.n + 1))
    gp = u64(packed).reshape(n_test, -1)
    for i in range(n_test):
        assert np.array_equal(gp[i], o.pack(oksk, resp[i])), f"sample {i}"
    # the packed coefficients decrypt to the lookups
    obits = wisard.encode(P, R["vals"])
    W = wisard.integer_wisard_train(P, obits, R["labels"])
    look = wisard.lookups(P, W, wisard.encode(P, R["tvals"]))
    assert np.array_equal(s.packed_counts(R["key"], packed, n_test).cpu().numpy(), look)


@pytest.mark.parametrize("name", list(TINY))
def test_tiny_packed_rlwe(name):
    cfg = tiny_cfg(name)
    _check_against_oracle(cfg, run_pipeline(cfg, 7, 3), 3)


def test_cfg1_packed_rlwe():
    cfg = get_config("cfg1")
    _check_against_oracle(cfg, run_pipeline(cfg, 6, 1), 1)


def test_cfg2_packed_rlwe_decrypts_to_the_responses():
    cfg = get_config("cfg2")
    R = run_pipeline(cfg, 2, 2)
    s = R["sess"]
    packed = s.pack_responses(s.ksk_gen(R["key"], 5), R["resp"], 2)
    a = s.packed_counts(R["key"], packed, 2)
    b = s.responses_counts(R["key"], R["resp"], 2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # everything above the l * k0 packed slots decrypts to 0
    full = s.decrypt_rlwe(R["key"], packed, 2).view(2, -1)
    assert not full[:, cfg.n_classes * s.sz["k0"]:].any()


@pytest.mark.parametrize("name", ["zL", "zgtL"])
def test_grouped_passes_equal_one_pass(name):
    """A scratch for one sample packs sample by sample, one for all samples in
    one pass, one for two samples in passes of two and a ragged last pass:
    the packed RLWEs are the same bits."""
    from paper_2403_20190_gb300 import binding as B
    cfg = tiny_cfg(name)
    R = run_pipeline(cfg, 7, 5)
    s = R["sess"]
    ksk = s.ksk_gen(R["key"], 11)
    outs = []
    for group in (1, 2, 5):
        scr = s.words(B.hw_pack_scratch_words(s.ctx, group), zero=False)
        outs.append(s.pack_responses(ksk, R["resp"], 5, scratch=scr))
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    with pytest.raises(B.HwError):
        s.pack_responses(ksk, R["resp"], 5, scratch=s.words(B.hw_pack_scratch_words(s.ctx, 1) - 1))
