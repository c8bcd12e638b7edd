"""Model checkpoints (host logic, no GPU): the exported-model format's header
checks in the library (hw_model_header_check, hw_params_digest) and the
file round trip.  Words and the trained-sample count round-trip exactly;
files of another parameter set, another format, or cut short are refused."""
import numpy as np
import pytest

from paper_2403_20190_gb300 import binding as B
from paper_2403_20190_gb300 import checkpoint
from synthdata import get_config


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2403_20190_gb300 import build
    build.build()
    return B.load()


def _export(cfg, n, seed, samples):
    """Words laid out as hw_model_export documents them (header, then n
    model words)."""
    rng = np.random.default_rng(seed)
    body = rng.integers(0, 1 << 55, size=n, dtype=np.uint64)
    head = np.array([B.HW_MODEL_MAGIC, B.HW_MODEL_VERSION, B.hw_params_digest(cfg), samples,
                     131, 10, 2, 4096, n], dtype=np.uint64)
    assert head.size == B.HW_MODEL_HEADER_WORDS
    return np.concatenate([head, body])


def test_round_trip(tmp_path):
    cfg = get_config("cfg2")
    w = _export(cfg, 4099, 1, samples=1234)
    path = str(tmp_path / "m.ckpt")
    checkpoint.write_words(path, w)
    back = checkpoint.read_words(path)
    assert back.dtype == np.uint64 and np.array_equal(back, w)
    assert checkpoint.check(path, cfg) == 1234


def test_refusals(tmp_path):
    cfg = get_config("cfg2")
    path = str(tmp_path / "m.ckpt")
    w = _export(cfg, 64, 2, samples=3)
    checkpoint.write_words(path, w)
    with pytest.raises(ValueError, match="another parameter set"):
        checkpoint.check(path, get_config("cfg2", log_p=12))
    cut = str(tmp_path / "cut.ckpt")
    checkpoint.write_words(cut, w[:-1])
    with pytest.raises(ValueError, match="not a usable"):
        checkpoint.check(cut, cfg)
    bad = w.copy()
    bad[0] ^= 1
    checkpoint.write_words(str(tmp_path / "bad.ckpt"), bad)
    with pytest.raises(ValueError, match="not a usable"):
        checkpoint.check(str(tmp_path / "bad.ckpt"), cfg)
    other = w.copy()
    other[1] = B.HW_MODEL_VERSION + 1
    checkpoint.write_words(str(tmp_path / "v.ckpt"), other)
    with pytest.raises(ValueError, match="not a usable"):
        checkpoint.check(str(tmp_path / "v.ckpt"), cfg)
    with open(str(tmp_path / "odd.ckpt"), "wb") as f:
        f.write(b"\0" * 13)
    with pytest.raises(ValueError, match="whole number of words"):
        checkpoint.check(str(tmp_path / "odd.ckpt"), cfg)


def test_header_check_codes():
    cfg = get_config("cfg1")
    w = _export(cfg, 10, 3, samples=7)
    assert B.hw_model_header_check(cfg, w) == 7
    with pytest.raises(B.HwError) as e:
        B.hw_model_header_check(get_config("cfg1", model_seed=5), w)
    assert e.value.code == B.HW_EMISMATCH
    with pytest.raises(B.HwError) as e:
        B.hw_model_header_check(cfg, w[:5])
    assert e.value.code == B.HW_EINVAL


def test_digest_covers_every_parameter():
    base = B.hw_params_digest(get_config("cfg1"))
    assert base == B.hw_params_digest(get_config("cfg1"))
    seen = {base}
    for change in (dict(log_n=11), dict(n_primes=2), dict(prime_bits=29), dict(log_beta=6), dict(log_p=9),
                   dict(n_classes=3), dict(n_values=31), dict(therm_bits=7), dict(tuple_bits=9),
                   dict(addr_bits=9), dict(hash_h3=1), dict(act="bin"), dict(act_arg=2),
                   dict(model_seed=99)):
        d = B.hw_params_digest(get_config("cfg1", **change))
        assert d not in seen, change
        seen.add(d)
