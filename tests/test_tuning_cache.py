"""The autotuner's on-disk cache (host logic, no GPU): a choice is reused for
the same GPU, parameters and probe size, and measured again when the loaded
library builds other candidate geometries or when asked to refresh."""
from paper_2403_20190_gb300 import binding as B
from paper_2403_20190_gb300 import tuning
from synthdata import get_config

GEO_A = [dict(ext_loge=3, ext_np=2, ext_smem=0), dict(ext_loge=3, ext_np=2, ext_smem=1)]
GEO_B = GEO_A + [dict(ext_loge=3, ext_np=2, ext_smem=2)]


def test_cache_is_keyed_by_the_built_geometries(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "CACHE", str(tmp_path / "tuning.json"))
    monkeypatch.setattr(tuning.torch.cuda, "get_device_name", lambda d=0: "GB300 (test)")
    calls = []

    def fake_autotune(cfg, device, n_probe, reps):
        calls.append(n_probe)
        return dict(ext_loge=3, ext_np=2, ext_smem=len(calls) % 2), [{"ms_infer": 1.0}]

    monkeypatch.setattr(B, "hw_autotune", fake_autotune)
    built = {"list": GEO_A}
    monkeypatch.setattr(B, "hw_list_geometries", lambda cfg: built["list"])
    cfg = get_config("cfg2")

    g1, entries, cached = tuning.tuned_geometry(cfg, 0)
    assert not cached and entries and len(calls) == 1
    g2, entries, cached = tuning.tuned_geometry(cfg, 0)
    assert cached and entries is None and g2 == g1 and len(calls) == 1
    # another probe size and other parameters are other keys
    tuning.tuned_geometry(cfg, 0, n_probe=8)
    tuning.tuned_geometry(get_config("cfg3"), 0)
    assert len(calls) == 3
    # a library with other candidates measures again
    built["list"] = GEO_B
    _, _, cached = tuning.tuned_geometry(cfg, 0)
    assert not cached and len(calls) == 4
    # an explicit refresh measures again
    _, _, cached = tuning.tuned_geometry(cfg, 0, refresh=True)
    assert not cached and len(calls) == 5
