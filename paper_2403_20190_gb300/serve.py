"""Continuous batching of encrypted train and infer requests over several
resident models.

Requests arrive over time, each for one workload configuration, carrying a
client's raw samples and an encryption seed.  The server keeps one encrypted
model per configuration resident in HBM and runs a loop that
  * admits pending requests while their HBM footprint (encrypted batch plus
    scratch) fits in the free budget,
  * groups admitted requests of the same (configuration, kind) into one
    batched launch on a free CUDA stream, so batches of different models
    overlap on the device,
  * retires batches whose completion events have fired and records each
    request's latency (arrival to completion).

Semantics within a serving window: inference requests answer with the model
as it stood when the window opened; training requests accumulate into a
per-model delta that is added into the model when the window closes.
Every per-sample result therefore depends only on the request itself (its
samples and seed), never on what it was batched with, and the closing model
equals sequential training of all train requests (addition mod q commutes).
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B
from .merge import add_models
from .session import Session


@dataclass
class Request:
    rid: int
    t_arrive: float
    cfg_name: str
    kind: str                     # "train" or "infer"
    values: np.ndarray            # (n, n_values) uint8
    labels: np.ndarray = None     # (n,) for train requests
    seed: int = 0
    t_done: float = None
    labels_out: np.ndarray = None  # predicted labels (infer)
    resp: torch.Tensor = None      # encrypted responses (infer), kept when asked

    @property
    def n(self):
        return int(self.values.shape[0])


class ResidentModel:
    def __init__(self, cfg, device, key_seed):
        self.cfg = cfg
        self.sess = Session(cfg, device)
        self.key = self.sess.keygen(key_seed)
        self.model = self.sess.new_model()   # frozen during a window
        self.delta = self.sess.new_model()   # this window's training

    def per_sample_bytes(self):
        return self.sess.sz["sample_words"] * 8

    def footprint(self, kind, n):
        """Device bytes one batch of n samples holds while in flight."""
        sz = self.sess.sz
        b = n * sz["sample_words"] * 8 + n * sz["n_data"]
        if kind == "train":
            b += B.hw_train_scratch_words(self.sess.ctx, n) * 8
        else:
            b += n * (sz["resp_words"] + sz["sums_words"]) * 8
            b += B.hw_infer_scratch_words(self.sess.ctx, n) * 8
            b += n * self.cfg.n_classes * (sz["k0"] + 1) * 8 + n * 4
        return b

    def close_window(self):
        q, n = self.sess.sz["q"], self.sess.sz["n"]
        self.model.copy_(add_models(self.model, self.delta, q, n))
        self.delta.zero_()


class _Batch:
    def __init__(self, rm, kind, reqs, stream, footprint):
        self.rm, self.kind, self.reqs, self.stream, self.footprint = rm, kind, reqs, stream, footprint
        self.event = torch.cuda.Event()
        self.keep = []  # buffers alive until the batch retires


class Server:
    def __init__(self, models: dict, hbm_budget_bytes: int, n_streams: int = 4,
                 max_batch_samples: int = 256, keep_responses: bool = False):
        self.models = models
        self.budget = hbm_budget_bytes
        self.free = hbm_budget_bytes
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.max_batch = max_batch_samples
        self.keep_responses = keep_responses

    # ------------------------------------------------------------------ launch
    def _launch(self, rm, kind, reqs, stream):
        s = rm.sess
        sz = s.sz
        n = sum(r.n for r in reqs)
        b = _Batch(rm, kind, reqs, stream, rm.footprint(kind, n))
        with torch.cuda.stream(stream):
            rgsw = s.words(n * sz["sample_words"], zero=False)
            b.keep.append(rgsw)
            off = 0
            for r in reqs:
                vals = torch.from_numpy(r.values).to(s.device, non_blocking=False)
                bits = torch.empty((r.n, sz["n_data"]), dtype=torch.uint8, device=s.device)
                B.hw_encode(s.ctx, vals, r.n, bits, stream)
                lab = None
                if kind == "train":
                    lab = torch.from_numpy(r.labels.astype(np.int32)).to(s.device)
                    b.keep.append(lab)
                dst = rgsw[off * sz["sample_words"]:(off + r.n) * sz["sample_words"]]
                # each request is encrypted under its own seed, sample indices
                # counted from 0, whatever it is batched with
                B.hw_encrypt_sample(s.ctx, rm.key, bits, lab, r.n, r.seed, 0, dst, stream)
                b.keep += [vals, bits]
                off += r.n
            if kind == "train":
                scratch = s.words(B.hw_train_scratch_words(s.ctx, n), zero=False)
                B.hw_train_accumulate(s.ctx, rm.delta, rgsw, n, scratch, stream)
                b.keep.append(scratch)
            else:
                resp, sums, scr = s.infer_buffers(n)
                B.hw_infer(s.ctx, rm.model, rgsw, n, resp, sums, scr, stream)
                l, k0 = rm.cfg.n_classes, sz["k0"]
                counts = torch.empty(n * l * k0, dtype=torch.int64, device=s.device)
                B.hw_decrypt(s.ctx, rm.key, B.HW_DEC_LWE, resp, n * l * k0, counts, stream)
                scores = torch.empty(n * l, dtype=torch.int64, device=s.device)
                labels = torch.empty(n, dtype=torch.int32, device=s.device)
                B.hw_pdact(s.ctx, counts, n, scores, labels, stream)
                b.keep += [resp, sums, scr, counts, scores]
                b.labels = labels
                b.resp = resp
            b.event.record(stream)
        return b

    def _retire(self, b, now):
        if b.kind == "infer":
            lab = b.labels.cpu().numpy()
            off = 0
            for r in b.reqs:
                r.labels_out = lab[off:off + r.n].copy()
                if self.keep_responses:
                    rw = b.rm.sess.sz["resp_words"]
                    r.resp = b.resp[off * rw:(off + r.n) * rw].clone()
                off += r.n
        for r in b.reqs:
            r.t_done = now
        self.free += b.footprint
        b.keep.clear()

    # -------------------------------------------------------------------- loop
    def run(self, requests, realtime=True):
        """Serve the requests (sorted by arrival); returns them completed.
        With realtime, a request is only visible once its arrival time has
        passed on the wall clock."""
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        for r in reqs:
            if self.models[r.cfg_name].footprint(r.kind, r.n) > self.budget:
                raise ValueError(f"request {r.rid} can never fit the HBM budget")
        arrivals = collections.deque(reqs)
        pending = collections.deque()
        inflight = []
        t0 = time.perf_counter()
        while arrivals or pending or inflight:
            now = time.perf_counter() - t0
            while arrivals and (not realtime or arrivals[0].t_arrive <= now):
                pending.append(arrivals.popleft())
            # retire finished batches
            for b in [b for b in inflight if b.event.query()]:
                inflight.remove(b)
                self._retire(b, time.perf_counter() - t0)
            # admit: the oldest pending request picks the (config, kind); every
            # pending request of that kind that fits joins its batch
            busy = {id(b.stream) for b in inflight}
            free_streams = [s for s in self.streams if id(s) not in busy]
            launched = False
            while pending and free_streams:
                head = pending[0]
                rm = self.models[head.cfg_name]
                group, n = [], 0
                for r in list(pending):
                    if r.cfg_name != head.cfg_name or r.kind != head.kind:
                        continue
                    if n + r.n > self.max_batch and group:
                        continue
                    if rm.footprint(r.kind, n + r.n) > self.free:
                        continue
                    group.append(r)
                    n += r.n
                if not group:
                    break  # the head waits for memory
                for r in group:
                    pending.remove(r)
                fp = rm.footprint(head.kind, n)
                self.free -= fp
                inflight.append(self._launch(rm, head.kind, group, free_streams.pop(0)))
                launched = True
            if not launched and not any(b.event.query() for b in inflight):
                if inflight:
                    time.sleep(0.0002)
                elif arrivals and realtime:
                    time.sleep(max(0.0, min(0.002, arrivals[0].t_arrive - now)))
        torch.cuda.synchronize()
        return reqs

    def run_one_at_a_time(self, requests):
        """Baseline: requests in arrival order, each alone, one stream, each
        waiting for the previous one to finish (no batching, no overlap)."""
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if r.t_arrive > now:
                time.sleep(r.t_arrive - now)
            b = self._launch(self.models[r.cfg_name], r.kind, [r], self.streams[0])
            b.event.synchronize()
            self._retire(b, time.perf_counter() - t0)
            self.free = self.budget
        return reqs


def poisson_stream(cfgs: dict, n_requests: int, rate: float, seed: int, max_samples: dict,
                   data_seed: int = 3):
    """A seeded Poisson stream: exponential inter-arrival times at `rate`
    requests/s; each request draws a configuration, a kind (train / infer)
    and a batch size from {1, 2, 4, ..., 256} clipped to max_samples[cfg]."""
    from synthdata import make_dataset
    rng = np.random.default_rng(seed)
    names = sorted(cfgs)
    pools = {}
    for nm in names:
        v, lab = make_dataset(cfgs[nm], "train", n=max(64, max_samples[nm]), seed=data_seed)
        pools[nm] = (v, lab)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate)
        nm = names[int(rng.integers(len(names)))]
        kind = "train" if rng.random() < 0.5 else "infer"
        n = min(1 << int(rng.integers(0, 9)), max_samples[nm])
        v, lab = pools[nm]
        start = int(rng.integers(0, v.shape[0] - n + 1))
        out.append(Request(rid=rid, t_arrive=t, cfg_name=nm, kind=kind,
                           values=np.ascontiguousarray(v[start:start + n]),
                           labels=np.ascontiguousarray(lab[start:start + n]) if kind == "train" else None,
                           seed=int(rng.integers(1, 2**62))))
    return out


def latency_stats(reqs):
    lat = np.array([r.t_done - r.t_arrive for r in reqs]) * 1000.0
    span = max(r.t_done for r in reqs) - min(r.t_arrive for r in reqs)
    samples = sum(r.n for r in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "samples_per_s": samples / span, "requests": len(reqs), "samples": samples,
            "span_s": span}
