"""Host logic of the server (no GPU): the seeded request stream, the
grouping of pending requests into candidate batches, the expected-cost
rule and the latency statistics."""
import numpy as np

from paper_2403_20190_gb300.serve import Request, Server, latency_stats, poisson_stream
from synthdata import get_config


def _req(rid, t, nm, kind, n):
    return Request(rid=rid, t_arrive=t, cfg_name=nm, kind=kind,
                   values=np.zeros((n, 4), dtype=np.uint8),
                   labels=np.zeros(n, dtype=np.int64) if kind == "train" else None)


def _server(max_batch):
    srv = Server.__new__(Server)  # the policy methods only, no models or streams
    srv.max_batch = max_batch
    srv.cost = {}
    return srv


def test_stream_is_seeded_and_clipped():
    cfgs = {nm: get_config(nm) for nm in ("cfg1", "cfg2")}
    caps = {"cfg1": 256, "cfg2": 16}
    a = poisson_stream(cfgs, 30, rate=200.0, seed=7, max_samples=caps)
    b = poisson_stream(cfgs, 30, rate=200.0, seed=7, max_samples=caps)
    assert [(r.t_arrive, r.cfg_name, r.kind, r.n, r.seed) for r in a] == \
           [(r.t_arrive, r.cfg_name, r.kind, r.n, r.seed) for r in b]
    assert all(np.array_equal(x.values, y.values) for x, y in zip(a, b))
    assert all(a[i].t_arrive < a[i + 1].t_arrive for i in range(len(a) - 1))
    for r in a:
        assert 1 <= r.n <= caps[r.cfg_name]
        assert r.n & (r.n - 1) == 0 or r.n == caps[r.cfg_name]  # a power of two, or the cap
        assert (r.labels is not None) == (r.kind == "train")
        assert r.values.shape == (r.n, cfgs[r.cfg_name].n_values)


def test_groups_by_model_and_kind_in_arrival_order_up_to_the_limit():
    srv = _server(max_batch=8)
    pending = [_req(0, 0.0, "cfg1", "train", 4), _req(1, 0.1, "cfg2", "infer", 2),
               _req(2, 0.2, "cfg1", "train", 4), _req(3, 0.3, "cfg1", "train", 1),
               _req(4, 0.4, "cfg1", "infer", 16), _req(5, 0.5, "cfg1", "infer", 1)]
    g = srv._groups(pending)
    assert sorted(g) == [("cfg1", "infer"), ("cfg1", "train"), ("cfg2", "infer")]
    # 4 + 4 fills the limit; the next train request waits for another batch
    assert [r.rid for r in g[("cfg1", "train")][0]] == [0, 2] and g[("cfg1", "train")][1] == 8
    # a request larger than the limit still forms a batch of its own
    assert [r.rid for r in g[("cfg1", "infer")][0]] == [4] and g[("cfg1", "infer")][1] == 16
    assert [r.rid for r in g[("cfg2", "infer")][0]] == [1]


def test_expected_cost_uses_calibration_then_the_prior():
    class FakeModel:
        class cfg:
            name = "cfg2"

        @staticmethod
        def prior_cost(kind):
            return 0.5 if kind == "infer" else 0.25

    srv = _server(max_batch=8)
    assert srv.expected(FakeModel, "infer", 4) == 2.0
    srv.cost[("cfg2", "infer")] = 0.1
    assert abs(srv.expected(FakeModel, "infer", 4) - 0.4) < 1e-12
    assert srv.expected(FakeModel, "train", 2) == 0.5


def test_latency_statistics():
    reqs = [_req(i, 0.1 * i, "cfg1", "infer", 2) for i in range(10)]
    for i, r in enumerate(reqs):
        r.t_done = r.t_arrive + 0.01 * (i + 1)
    st = latency_stats(reqs)
    lat = np.array([0.01 * (i + 1) for i in range(10)]) * 1000.0
    assert abs(st["p50_ms"] - np.percentile(lat, 50)) < 1e-9
    assert abs(st["p99_ms"] - np.percentile(lat, 99)) < 1e-9
    assert st["samples"] == 20 and st["requests"] == 10
    assert abs(st["span_s"] - (0.9 + 0.1)) < 1e-9
    assert abs(st["samples_per_s"] - 20 / 1.0) < 1e-9


def test_a_model_with_training_in_flight_gets_no_second_training_batch():
    srv = _server(max_batch=4)
    pending = [_req(0, 0.0, "cfg1", "train", 2), _req(1, 0.1, "cfg1", "infer", 2),
               _req(2, 0.2, "cfg2", "train", 2)]
    g = srv._groups(pending, training={"cfg1"})
    assert sorted(g) == [("cfg1", "infer"), ("cfg2", "train")]
    g = srv._groups(pending)
    assert ("cfg1", "train") in g
