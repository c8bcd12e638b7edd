"""Continuous batching of encrypted train and infer requests over several
resident models.

Requests arrive over time, each for one workload configuration, carrying a
client's raw samples and an encryption seed.  The server keeps one encrypted
model per configuration resident in HBM and runs a loop that
  * admits pending requests while their HBM footprint (encrypted batch plus
    scratch) fits in the free budget,
  * groups admitted requests of the same (configuration, kind) into one
    batched launch on a free CUDA stream, so batches of different models
    overlap on the device; a model has at most one training batch in
    flight (training adds into the model's delta in place),
  * retires batches whose completion events have fired and records each
    request's latency (arrival to completion).

Memory: every batch takes one chunk of a device arena allocated up front
(arena.py) and carves its buffers from it, so admission by footprint is
admission by placement and the loop never calls the CUDA allocator.

Order: policy "fifo" (the default) launches the group whose oldest request
arrived first: every request of the same (configuration, kind) that is
pending by then joins it, so a backlog turns into few large batches and no
request is overtaken by later ones (the tail latency stays that of arrival
order).  Policy "sjf" launches the group with the least expected GPU time,
less the age of its oldest request (shortest expected batch first with
aging, so no request waits forever).  Expected times are
per-sample costs per (configuration, kind): calibrate() times one
single-sample batch of each alone, and batches that ran with nothing else
on the GPU refine them (a batch that overlapped others is slowed by them
and says little about its own cost); before any measurement they come from
the encrypted-sample size.

Semantics within a serving window: inference requests answer with the model
as it stood when the window opened; training requests accumulate into a
per-model delta that is added into the model when the window closes.
Every per-sample result therefore depends only on the request itself (its
samples and seed), never on what it was batched with, and the closing model
equals sequential training of all train requests (addition mod q commutes).
"""
import collections
import copy
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import binding as B
from .arena import DeviceArena, align_up
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
    def __init__(self, cfg, device, key_seed, geometry=None):
        """geometry: as for Session (None, "auto" or a dict)."""
        self.cfg = cfg
        self.sess = Session(cfg, device, geometry=geometry)
        self.key = self.sess.keygen(key_seed)
        self.model = self.sess.new_model()   # frozen during a window
        self.delta = self.sess.new_model()   # this window's training

    def per_sample_bytes(self):
        return self.sess.sz["sample_words"] * 8

    def layout(self, kind, n):
        """The buffers one batch of n samples holds while in flight, in the
        order they are carved: (name, element count, dtype)."""
        sz, l = self.sess.sz, self.cfg.n_classes
        out = [("values", n * self.cfg.n_values, torch.uint8),
               ("bits", n * sz["n_data"], torch.uint8),
               ("rgsw", n * sz["sample_words"], torch.int64)]
        if kind == "train":
            out += [("labels", n, torch.int32),
                    ("scratch", B.hw_train_scratch_words(self.sess.ctx, n), torch.int64)]
        else:
            out += [("resp", n * sz["resp_words"], torch.int64),
                    ("sums", n * sz["sums_words"], torch.int64),
                    ("scratch", B.hw_infer_scratch_words(self.sess.ctx, n), torch.int64),
                    ("counts", n * l * sz["k0"], torch.int64),
                    ("scores", n * l, torch.int64),
                    ("labels_out", n, torch.int32)]
        return out

    def footprint(self, kind, n):
        """Device bytes one batch of n samples holds while in flight."""
        return sum(align_up(c * torch.empty((), dtype=d).element_size()) for _, c, d in self.layout(kind, n))

    def prior_cost(self, kind):
        """Expected GPU seconds per sample before any measurement: encrypted
        bytes over an assumed 1 GB/s of external-product throughput, times
        the class count for inference."""
        c = self.sess.sz["sample_words"] * 8 / 1e9
        return c * (self.cfg.n_classes if kind == "infer" else 1)

    def close_window(self):
        q, n = self.sess.sz["q"], self.sess.sz["n"]
        self.model.copy_(add_models(self.model, self.delta, q, n))
        self.delta.zero_()


class _Batch:
    def __init__(self, rm, kind, reqs, stream, chunk):
        self.rm, self.kind, self.reqs, self.stream, self.chunk = rm, kind, reqs, stream, chunk
        self.start = torch.cuda.Event(enable_timing=True)
        self.event = torch.cuda.Event(enable_timing=True)
        self.bufs = {}
        self.solo = True  # nothing else ran on the GPU during its lifetime


class Server:
    def __init__(self, models: dict, hbm_budget_bytes: int = None, n_streams: int = 2,
                 max_batch_samples: int = 256, keep_responses: bool = False, arena=None,
                 aging: float = 1.0, packed_infer: bool = False, policy: str = "fifo"):
        """models: name -> ResidentModel.  The arena (or a new one of
        hbm_budget_bytes on the models' device) holds every batch in flight.
        packed_infer answers inference with horizontal packing
        (hw_infer_packed: one VP per group of classes sharing a stored
        ciphertext; other ciphertexts, the same decrypted counters)."""
        self.models = models
        if arena is None:
            dev = next(iter(models.values())).sess.device
            arena = DeviceArena(hbm_budget_bytes, dev)
        self.arena = arena
        self.budget = arena.size
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.max_batch = max_batch_samples
        self.keep_responses = keep_responses
        self.aging = aging
        self.packed_infer = packed_infer
        if policy not in ("fifo", "sjf"):
            raise ValueError(f"unknown policy {policy!r}")
        self.policy = policy
        self.cost = {}  # (cfg name, kind) -> smoothed GPU seconds per sample

    @property
    def free(self):
        return self.arena.free_bytes

    # ------------------------------------------------------------------ launch
    def _launch(self, rm, kind, reqs, stream, chunk):
        s = rm.sess
        sz = s.sz
        n = sum(r.n for r in reqs)
        b = _Batch(rm, kind, reqs, stream, chunk)
        buf = b.bufs
        for name, count, dtype in rm.layout(kind, n):
            buf[name] = chunk.take(count, dtype)
        with torch.cuda.stream(stream):
            b.start.record(stream)
            vals = buf["values"].view(n, rm.cfg.n_values)
            off = 0
            for r in reqs:
                vals[off:off + r.n].copy_(torch.from_numpy(r.values))
                if kind == "train":
                    buf["labels"][off:off + r.n].copy_(torch.from_numpy(r.labels.astype(np.int32)))
                off += r.n
            B.hw_encode(s.ctx, vals, n, buf["bits"], stream)
            off = 0
            for r in reqs:
                w = sz["sample_words"]
                # each request is encrypted under its own seed, sample indices
                # counted from 0, whatever it is batched with
                lab = buf["labels"][off:off + r.n] if kind == "train" else None
                B.hw_encrypt_sample(s.ctx, rm.key, buf["bits"][off * sz["n_data"]:], lab, r.n, r.seed, 0,
                                    buf["rgsw"][off * w:(off + r.n) * w], stream)
                off += r.n
            if kind == "train":
                B.hw_train_accumulate(s.ctx, rm.delta, buf["rgsw"], n, buf["scratch"], stream)
            else:
                infer = B.hw_infer_packed if self.packed_infer else B.hw_infer
                infer(s.ctx, rm.model, buf["rgsw"], n, buf["resp"], buf["sums"], buf["scratch"], stream)
                l, k0 = rm.cfg.n_classes, sz["k0"]
                B.hw_decrypt(s.ctx, rm.key, B.HW_DEC_LWE, buf["resp"], n * l * k0, buf["counts"], stream)
                B.hw_pdact(s.ctx, buf["counts"], n, buf["scores"], buf["labels_out"], stream)
            b.event.record(stream)
        return b

    def _retire(self, b, now):
        if b.kind == "infer":
            off = 0
            for r in b.reqs:
                if self.keep_responses:
                    rw = b.rm.sess.sz["resp_words"]
                    r.resp = b.bufs["resp"][off * rw:(off + r.n) * rw].clone()
                off += r.n
            # a blocking copy on the same stream: the clones above have run
            # before the chunk goes back to the arena (the next batch may
            # overwrite it from another stream at once)
            lab = b.bufs["labels_out"].cpu().numpy()
            torch.cuda.current_stream().synchronize()
            off = 0
            for r in b.reqs:
                r.labels_out = lab[off:off + r.n].copy()
                off += r.n
        for r in b.reqs:
            r.t_done = now
        if b.solo:
            n = sum(r.n for r in b.reqs)
            key = (b.rm.cfg.name, b.kind)
            per = b.start.elapsed_time(b.event) / 1e3 / n
            self.cost[key] = per if key not in self.cost else 0.5 * self.cost[key] + 0.5 * per
        b.bufs.clear()
        self.arena.release(b.chunk)

    def expected(self, rm, kind, n):
        """Expected GPU seconds of a batch of n samples."""
        per = self.cost.get((rm.cfg.name, kind))
        return n * (per if per is not None else rm.prior_cost(kind))

    def _groups(self, pending, training=()):
        """Candidate batches: per (configuration, kind), pending requests in
        arrival order up to the batch limit.  Models named in `training`
        have a training batch in flight: their training requests wait, since
        two training batches of one model would both add into its delta."""
        groups = {}
        for r in pending:
            if r.kind == "train" and r.cfg_name in training:
                continue
            key = (r.cfg_name, r.kind)
            g = groups.setdefault(key, [[], 0])
            if g[1] + r.n > self.max_batch and g[0]:
                continue
            g[0].append(r)
            g[1] += r.n
        return groups

    # -------------------------------------------------------------------- loop
    def run(self, requests, realtime=True):
        """Serve the requests; returns them completed.  With realtime, a
        request is only visible once its arrival time has passed on the wall
        clock."""
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        for r in reqs:
            if self.models[r.cfg_name].footprint(r.kind, r.n) > self.budget:
                raise ValueError(f"request {r.rid} can never fit the HBM budget")
        arrivals = collections.deque(reqs)
        pending = []
        inflight = []
        t0 = time.perf_counter()
        while arrivals or pending or inflight:
            now = time.perf_counter() - t0
            while arrivals and (not realtime or arrivals[0].t_arrive <= now):
                pending.append(arrivals.popleft())
            for b in [b for b in inflight if b.event.query()]:
                inflight.remove(b)
                self._retire(b, time.perf_counter() - t0)
            busy = {id(b.stream) for b in inflight}
            free_streams = [s for s in self.streams if id(s) not in busy]
            launched = False
            while pending and free_streams:
                now = time.perf_counter() - t0
                ranked = []
                training = {b.rm.cfg.name for b in inflight if b.kind == "train"}
                for (nm, kind), (group, n) in self._groups(pending, training).items():
                    rm = self.models[nm]
                    oldest = min(r.t_arrive for r in group)
                    if self.policy == "fifo":
                        score = oldest
                    else:
                        score = self.expected(rm, kind, n) - self.aging * (now - oldest)
                    ranked.append((score, oldest, nm, kind, group))
                ranked.sort(key=lambda x: (x[0], x[1]))
                placed = None
                for _, _, nm, kind, group in ranked:
                    rm = self.models[nm]
                    # shrink the group (newest first) until it can be placed
                    while group:
                        chunk = self.arena.alloc(rm.footprint(kind, sum(r.n for r in group)))
                        if chunk is not None:
                            placed = (rm, kind, group, chunk)
                            break
                        group = group[:-1]
                    if placed:
                        break
                if placed is None:
                    break  # everything waits for memory
                rm, kind, group, chunk = placed
                for r in group:
                    pending.remove(r)
                for o in inflight:
                    o.solo = False
                b = self._launch(rm, kind, group, free_streams.pop(0), chunk)
                b.solo = not inflight
                inflight.append(b)
                launched = True
            if not launched and not any(b.event.query() for b in inflight):
                if inflight:
                    time.sleep(0.0002)
                elif arrivals and realtime:
                    time.sleep(max(0.0, min(0.002, arrivals[0].t_arrive - now)))
        torch.cuda.synchronize()
        return reqs

    def calibrate(self, kinds=("train", "infer")):
        """Time one single-sample batch of every (model, kind) alone and take
        it as the expected per-sample cost.  Training runs into a temporary
        delta from the arena, so the resident models do not change."""
        for nm, rm in self.models.items():
            cfg = rm.cfg
            for kind in kinds:
                req = Request(rid=-1, t_arrive=0.0, cfg_name=nm, kind=kind,
                              values=np.zeros((1, cfg.n_values), dtype=np.uint8),
                              labels=np.zeros(1, dtype=np.int64) if kind == "train" else None, seed=1)
                target, tmp = rm, None
                if kind == "train":
                    tmp = self.arena.alloc(rm.sess.sz["model_words"] * 8)
                    if tmp is None:
                        continue
                    target = copy.copy(rm)
                    target.delta = tmp.take(rm.sess.sz["model_words"], torch.int64)
                chunk = self.arena.alloc(rm.footprint(kind, 1))
                if chunk is None:
                    if tmp is not None:
                        self.arena.release(tmp)
                    continue
                b = self._launch(target, kind, [req], self.streams[0], chunk)
                b.event.synchronize()
                self._retire(b, 0.0)
                if tmp is not None:
                    self.arena.release(tmp)
        return dict(self.cost)

    def run_one_at_a_time(self, requests):
        """Baseline: requests in arrival order, each alone, one stream, each
        waiting for the previous one to finish (no batching, no overlap)."""
        reqs = sorted(requests, key=lambda r: r.t_arrive)
        t0 = time.perf_counter()
        for r in reqs:
            now = time.perf_counter() - t0
            if r.t_arrive > now:
                time.sleep(r.t_arrive - now)
            rm = self.models[r.cfg_name]
            chunk = self.arena.alloc(rm.footprint(r.kind, r.n))
            if chunk is None:
                raise ValueError(f"request {r.rid} can never fit the HBM budget")
            b = self._launch(rm, r.kind, [r], self.streams[0], chunk)
            b.event.synchronize()
            self._retire(b, time.perf_counter() - t0)
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
