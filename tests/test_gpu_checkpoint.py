"""Checkpoint and resume on the GPU: training stopped after a batch, saved,
loaded into a fresh context and continued gives the model of an
uninterrupted run, bit for bit (the model is a running sum mod q_i,
Section 3.6.2)."""
import numpy as np
import pytest
import torch

from synthdata import get_config, make_dataset
from test_gpu_parity import session, tiny_cfg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg", [tiny_cfg("zgtL"), get_config("cfg1")], ids=["zgtL", "cfg1"])
def test_resume_equals_uninterrupted_training(cfg, tmp_path):
    sess = session(cfg)
    dev = sess.device
    vals, labels = make_dataset(cfg, "train", n=6)
    key = sess.keygen(3)
    bits = sess.encode(torch.from_numpy(vals).to(dev))
    rg = sess.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=5)
    whole = sess.train(sess.new_model(), rg, 6)
    sw = sess.sz["sample_words"]
    part = sess.train(sess.new_model(), rg[:4 * sw], 4)
    path = str(tmp_path / "model.ckpt")
    sess.save_model(path, part, 4)
    fresh = session(cfg)  # another context of the same parameters and geometry
    model, samples = fresh.load_model(path)
    assert samples == 4
    fresh.train(model, rg[4 * sw:], 2)
    torch.cuda.synchronize()
    assert torch.equal(model, whole)
    with pytest.raises(ValueError):
        session(get_config("cfg1", log_p=9)).load_model(path)
