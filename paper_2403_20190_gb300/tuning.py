"""Kernel-geometry selection with an on-disk cache.

hw_autotune (in the library) times every built geometry of a parameter set
on a probe step; this module remembers the winner per (GPU name, parameters,
probe size) in a JSON file beside the built library, so a workload pays for
the measurement once per machine.  Every geometry computes the same results:
the choice only changes speed.
"""
import json
import os

import torch

from . import binding as B
from . import build as _build

CACHE = os.path.join(_build.OUT, "tuning.json")


def _key(cfg, device, n_probe):
    """GPU name, parameters, probe size and the geometries the loaded library
    builds for them: a library with other candidates measures again."""
    p = B.params_from_config(cfg)
    fields = [f for f, _ in B.HwParams._fields_ if f != "reserved"]
    prm = ",".join(f"{f}={getattr(p, f)}" for f in fields)
    built = ";".join(f"{g['ext_loge']}.{g['ext_np']}.{g['ext_smem']}" for g in B.hw_list_geometries(cfg))
    return f"{torch.cuda.get_device_name(device)}|{prm}|n_probe={n_probe}|built={built}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_geometry(cfg, device: int = 0, n_probe: int = 4, reps: int = 2, refresh: bool = False):
    """Returns (geometry dict, measured candidates or None if cached, cached?)."""
    key = _key(cfg, device, n_probe)
    cache = _load()
    if not refresh and key in cache:
        return cache[key]["geometry"], None, True
    best, entries = B.hw_autotune(cfg, device, n_probe, reps)
    cache = _load()
    cache[key] = {"geometry": best, "entries": entries}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    return best, entries, False
