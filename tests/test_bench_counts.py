"""The bench's algorithmic work (the roofline's numerator), on the CPU: the
external products per training and test sample of each workload match the
counts derived from the parameter sets (ring, gadget, RAM bit layout,
pruned tree) -- 270 / 2747 / 2940 / 13104 per training sample and 480 /
15680 / 17640 / 49392 per test sample -- and one cfg2 external product is
360 448 modular products."""
import pytest

import bench
from oracle import Oracle, wisard
from synthdata import get_config

EXPECT = {"cfg1": (270, 480), "cfg2": (2747, 15680), "cfg3": (2940, 17640), "cfg4": (13104, 49392)}


def _work(name):
    cfg = get_config(name)
    o = Oracle(cfg)
    P = o.P
    sz = dict(n=P.n, r=P.r, dnum=P.dnum, L=P.L, z=P.z, a=P.a, k0=P.k0, rgsw_words=o.rgsw_words)
    slots = [int(d) for j in range(P.k0) for d in wisard.ram_bits(P)[j]]
    return bench.algorithmic_work(sz, slots, cfg.n_classes)


@pytest.mark.parametrize("name", list(EXPECT))
def test_external_products_per_sample(name):
    w = _work(name)
    assert (w["ext_train_per_sample"], w["ext_infer_per_sample"]) == EXPECT[name]
    # a model in clear shares each (sample, RAM)'s rotation between the classes
    assert w["ext_clear_per_sample"] < w["ext_infer_per_sample"]


def test_modular_products_per_external_product():
    assert _work("cfg2")["per_ext_modmul"] == 360448
