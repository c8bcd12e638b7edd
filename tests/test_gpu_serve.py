"""Serving: every request's result is the same alone and in the mix.

A seeded stream of train and infer requests over three resident models is
served with continuous batching (all requests arriving at once, so they are
batched and overlapped as much as possible).  Each request is then served
again alone by a fresh server holding the same models.  Infer requests must
return bit-identical encrypted responses and labels; the training deltas of
the requests served alone must add up (mod q) to the delta of the mixed run;
closing the window adds the delta into the model.  Integer results:
tolerance 0.
"""
import numpy as np
import pytest
import torch

from synthdata import get_config, make_dataset

pytestmark = pytest.mark.gpu

CFGS = {
    "tiny_rns": dict(base="cfg1", log_n=6, n_primes=2, prime_bits=50, log_beta=0, log_p=16,
                     n_classes=3, n_values=7, therm_bits=2, addr_bits=6, tuple_bits=6,
                     data_kind="uniform", act="log", act_arg=0),
    "tiny_tree": dict(base="cfg1", log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=22,
                      n_classes=3, n_values=4, therm_bits=2, addr_bits=7, tuple_bits=7,
                      data_kind="uniform", act="log", act_arg=0),
    "cfg1": dict(base="cfg1"),
}


def _configs():
    out = {}
    for nm, d in CFGS.items():
        d = dict(d)
        base = d.pop("base")
        out[nm] = get_config(base, name=nm, **d)
    return out


def _models(cfgs, pretrain=True, n_pre=8):
    from paper_2403_20190_gb300.serve import ResidentModel
    models = {}
    for k, (nm, cfg) in enumerate(sorted(cfgs.items())):
        rm = ResidentModel(cfg, 0, key_seed=40 + k)
        if pretrain:
            s = rm.sess
            v, lab = make_dataset(cfg, "train", n=n_pre, seed=11)
            bits = s.encode(torch.from_numpy(v).to(s.device))
            rg = s.encrypt(rm.key, bits, torch.from_numpy(lab.astype(np.int32)).to(s.device), seed=5)
            s.train(rm.model, rg, n_pre)
            del rg
        models[nm] = rm
    torch.cuda.synchronize()
    return models


@pytest.mark.parametrize("packed", [False, True])
def test_alone_equals_in_the_mix(packed):
    alone_equals_in_the_mix(_configs(), {"tiny_rns": 8, "tiny_tree": 8, "cfg1": 16}, n_requests=18,
                            budget=8 << 30, n_pre=8, packed=packed)


def test_alone_equals_in_the_mix_workload_rings():
    """The digit workload (N = 4096, two primes) and the skewed colour
    workload (N = 8192, three primes, an encrypted tree level) in one
    stream with cfg1: 1-2 samples per request for cfg2, 1 for cfg4."""
    cfgs = {nm: get_config(nm) for nm in ("cfg1", "cfg2", "cfg4")}
    alone_equals_in_the_mix(cfgs, {"cfg1": 16, "cfg2": 2, "cfg4": 1}, n_requests=10,
                            budget=64 << 30, n_pre=2, packed=False, seed=4)


def alone_equals_in_the_mix(cfgs, max_samples, n_requests, budget, n_pre, packed, seed=9):
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.merge import add_models
    from paper_2403_20190_gb300.serve import Server, poisson_stream
    build.build()
    mixed_models = _models(cfgs, n_pre=n_pre)
    base = {nm: rm.model.clone() for nm, rm in mixed_models.items()}
    reqs = poisson_stream(cfgs, n_requests=n_requests, rate=200.0, seed=seed, max_samples=max_samples)
    srv = Server(mixed_models, hbm_budget_bytes=budget, n_streams=4, max_batch_samples=64,
                 keep_responses=True, packed_infer=packed)
    done = srv.run(reqs, realtime=False)
    assert all(r.t_done is not None for r in done)
    batched = sum(1 for r in done if r.kind == "infer")
    assert batched > 0 and any(r.kind == "train" for r in done)

    from paper_2403_20190_gb300.arena import DeviceArena
    del srv
    arena = DeviceArena(budget, torch.device("cuda", 0))
    alone_models = _models(cfgs, pretrain=False)
    for nm in cfgs:
        alone_models[nm].model.copy_(base[nm])
    delta_sum = {nm: torch.zeros_like(rm.delta) for nm, rm in alone_models.items()}
    for r in done:
        rm = alone_models[r.cfg_name]
        rm.delta.zero_()
        srv1 = Server(alone_models, n_streams=1, keep_responses=True, arena=arena, packed_infer=packed)
        import copy
        r1 = copy.copy(r)
        r1.t_done = r1.labels_out = r1.resp = None
        srv1.run([r1], realtime=False)
        if r.kind == "infer":
            assert np.array_equal(r1.labels_out, r.labels_out), f"request {r.rid} labels"
            assert torch.equal(r1.resp, r.resp), f"request {r.rid} responses"
        else:
            q, n = rm.sess.sz["q"], rm.sess.sz["n"]
            delta_sum[r.cfg_name] = add_models(delta_sum[r.cfg_name], rm.delta, q, n)
    torch.cuda.synchronize()
    for nm, rm in mixed_models.items():
        assert torch.equal(rm.delta, delta_sum[nm]), f"{nm}: training deltas differ"
        q, n = rm.sess.sz["q"], rm.sess.sz["n"]
        expect = add_models(base[nm], rm.delta, q, n)
        rm.close_window()
        assert torch.equal(rm.model, expect)
        assert not rm.delta.any()


def test_admission_respects_the_budget():
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.serve import Request, Server
    build.build()
    cfgs = {"cfg1": _configs()["cfg1"]}
    models = _models(cfgs, pretrain=False)
    rm = models["cfg1"]
    v, lab = make_dataset(cfgs["cfg1"], "train", n=4)
    one = rm.footprint("train", 4)
    srv = Server(models, hbm_budget_bytes=one, n_streams=4)
    reqs = [Request(rid=i, t_arrive=0.0, cfg_name="cfg1", kind="train", values=v, labels=lab, seed=i + 1)
            for i in range(3)]
    srv.run(reqs, realtime=False)
    assert all(r.t_done is not None for r in reqs)
    assert srv.free == srv.budget and not srv.arena.fl.used
    with pytest.raises(ValueError):
        Server(models, hbm_budget_bytes=one - 1).run(
            [Request(rid=9, t_arrive=0.0, cfg_name="cfg1", kind="train", values=v, labels=lab, seed=1)],
            realtime=False)


def test_training_batches_of_one_model_never_overlap():
    """Many small training requests for one model, several free streams and
    a small batch limit: the server must not run two training batches of the
    model at once (both would add into its delta).  The mixed delta equals
    the sum of the deltas of the requests trained alone."""
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.merge import add_models
    from paper_2403_20190_gb300.serve import Request, Server
    build.build()
    cfgs = {"tiny_rns": _configs()["tiny_rns"]}
    models = _models(cfgs, pretrain=False)
    rm = models["tiny_rns"]
    v, lab = make_dataset(cfgs["tiny_rns"], "train", n=24, seed=5)
    reqs = [Request(rid=i, t_arrive=0.0, cfg_name="tiny_rns", kind="train",
                    values=np.ascontiguousarray(v[2 * i:2 * i + 2]),
                    labels=np.ascontiguousarray(lab[2 * i:2 * i + 2]), seed=100 + i)
            for i in range(12)]
    srv = Server(models, hbm_budget_bytes=4 << 30, n_streams=4, max_batch_samples=2)
    srv.run(reqs, realtime=False)
    torch.cuda.synchronize()
    mixed = rm.delta.clone()
    q, n = rm.sess.sz["q"], rm.sess.sz["n"]
    total = torch.zeros_like(mixed)
    for r in reqs:
        rm.delta.zero_()
        Server(models, hbm_budget_bytes=1 << 30, n_streams=1).run([Request(
            rid=r.rid, t_arrive=0.0, cfg_name=r.cfg_name, kind="train", values=r.values,
            labels=r.labels, seed=r.seed)], realtime=False)
        total = add_models(total, rm.delta, q, n)
    torch.cuda.synchronize()
    assert torch.equal(mixed, total)
