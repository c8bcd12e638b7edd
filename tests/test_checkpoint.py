"""Model checkpoints (host logic, no GPU): words and the trained-sample
count round-trip exactly; files of another parameter set, another format,
or cut short are refused."""
import numpy as np
import pytest
import torch

from paper_2403_20190_gb300 import checkpoint
from synthdata import get_config


def _model(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 1 << 55, size=n, dtype=np.uint64)
    w[:3] = [0, (1 << 55) - 1, 1]
    return torch.from_numpy(w.view(np.int64).copy())


def test_round_trip(tmp_path):
    cfg = get_config("cfg2")
    m = _model(4099, 1)
    path = str(tmp_path / "m.ckpt")
    checkpoint.save(path, cfg, m, samples=1234)
    back, samples = checkpoint.load(path, cfg)
    assert samples == 1234 and torch.equal(back, m)


def test_refusals(tmp_path):
    cfg = get_config("cfg2")
    path = str(tmp_path / "m.ckpt")
    checkpoint.save(path, cfg, _model(64, 2), samples=3)
    with pytest.raises(ValueError, match="another parameter set"):
        checkpoint.load(path, get_config("cfg2", log_p=12))
    blob = open(path, "rb").read()
    cut = str(tmp_path / "cut.ckpt")
    open(cut, "wb").write(blob[:-8])
    with pytest.raises(ValueError, match="bytes of model words"):
        checkpoint.load(cut, cfg)
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(b"NOTACKPT" + blob[8:])
    with pytest.raises(ValueError, match="not a model checkpoint"):
        checkpoint.load(bad, cfg)


def test_digest_covers_every_parameter():
    base = checkpoint.params_digest(get_config("cfg1"))
    assert base == checkpoint.params_digest(get_config("cfg1"))
    for change in (dict(log_n=11), dict(n_primes=2), dict(log_beta=6), dict(model_seed=99)):
        assert checkpoint.params_digest(get_config("cfg1", **change)) != base
