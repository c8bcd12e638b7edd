#!/usr/bin/env python3
"""Benchmark of the encrypted WiSARD hot path on GB300; prints one JSON line.

A step is one pass of the whole path over one batch: B training samples are
encoded, RGSW-encrypted and trained into the resident model (IVP +
accumulate), and B test samples are encoded, encrypted, inferred (VP,
ExtractLWE, class sums), decrypted and classified with PD-act.  The headline
workload is the at-scale digit configuration (10 classes, 28x28 images,
3-level thermometer, 16-bit tuples H3-hashed to 12 address bits, N = 8192,
three ~55-bit RNS primes; B = 16).  Raw samples sit in HBM before the timed
region; encrypted batches (~125 GB per step) are far larger than L2.
`per_config` in the same line repeats a shorter measurement on the other
workloads (the 2-class feature set, the 10-class digits at N = 4096 and the
7-class colour images at N = 8192).

--impl reference times the CPU oracle on the host cores instead, on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "encrypted samples/s (train + inference, bit-exact)"
UNIT = "samples/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# Integer multiply throughput of one SM per clock (32-bit multiply-add lanes)
# and the minimum 32x32-bit multiplies of one 64-bit Shoup modular product
# (high half of x*w': 4 partial products; low halves of x*w and qhat*q: 3 each).
IMAD_PER_CLK_PER_SM = 64
MULS_PER_MODMUL = 10
# ... and of one 32-bit Shoup product (low halves of x*w and qhat*q, high
# half of x*w'), for contexts whose external products run in 32-bit words.
MULS_PER_MODMUL32 = 3

DEFAULT_CONFIG = "cfg3"
# samples per step: cfg1's whole test set; for the larger rings, what keeps one
# encrypted batch (786 MiB, 3.9 GiB, 15.5 GiB per sample) plus scratch well
# inside HBM
DEFAULT_BATCH = {"cfg1": 100, "cfg2": 64, "cfg3": 16, "cfg4": 4}
ALL_CONFIGS = ("cfg1", "cfg2", "cfg3", "cfg4")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--batch", type=int, default=0,
                    help="samples per step (0: the workload's default, sized to fit HBM)")
    ap.add_argument("--per-config-steps", type=int, default=3,
                    help="timed steps of each other workload in per_config (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ntt", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-balance", action="store_true")
    ap.add_argument("--no-packing", action="store_true")
    ap.add_argument("--no-keyswitch", action="store_true")
    ap.add_argument("--no-clear-model", action="store_true",
                    help="skip the leg that answers the test batch against the model in clear")
    ap.add_argument("--serve-requests", type=int, default=40)
    ap.add_argument("--geometry", default="auto", choices=["auto", "default"],
                    help="kernel geometry: autotuned (cached per GPU and parameters) or the library default")
    return ap.parse_args()


# DRAM bytes of the VP inference kernel per test sample, from ncu captures of
# small cases of each workload (scaled by samples: the traffic is per item);
# valid only for the kernel sources they were taken on: the VP kernel with
# the device helpers it calls (the region of hw_ext.cuh from bit_slot to the
# VP kernel's end) and the headers of the external product and the modular
# arithmetic.  Filled per (workload, geometry) when a capture of the current
# sources exists.
PROFILED_VP_TRAFFIC = [
    {"config": "cfg3", "ext_loge": 3, "ext_np": 1, "ext_smem": 3, "ext_blocks_per_sm": 1, "l2_persist": 0,
     "bytes_per_test_sample": 7.96436e10,
     "sha256": "390053d8ae31d876b16edc9f70df0a9eef4c8f8f0ca4677abe20607d138753d7"},
]
PROFILED_SOURCES = (("paper_2403_20190_gb300/csrc/hw_ext.cuh", "// Encrypted bit slot that drives",
                     "// EncRGSW."),
                    ("paper_2403_20190_gb300/csrc/hw_ext.cuh", "// ExtractLWE(ct, k) written by the block",
                     "// Dataset balancing (Section 3.6.1)"),
                    ("paper_2403_20190_gb300/csrc/hw_internal.cuh", None, None),
                    ("paper_2403_20190_gb300/csrc/modarith.cuh", None, None))


def profiled_sources_sha(root=None):
    """sha256 over the profiled source regions (whole file where no markers)."""
    import hashlib
    h = hashlib.sha256()
    for f, start, end in PROFILED_SOURCES:
        with open(os.path.join(root or ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        if start is not None:
            i = text.index(start)
            text = text[i:text.index(end, i)]
        h.update(text.encode("utf-8"))
    return h.hexdigest()


GEOMETRY_KEYS = ("ext_loge", "ext_np", "ext_smem", "ext_blocks_per_sm", "l2_persist")


def profiled_traffic(config, geometry, n_test):
    sha = None
    for t in PROFILED_VP_TRAFFIC:
        if config != t["config"] or any(geometry.get(k) != t[k] for k in GEOMETRY_KEYS):
            continue
        sha = sha or profiled_sources_sha()
        if sha == t["sha256"]:  # otherwise the kernel changed since the counters were taken
            return t["bytes_per_test_sample"] * n_test
    return None


# ----------------------------------------------------------------- helpers
def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return ws, rank, local, pg


def workload_name(cfg):
    return (f"{cfg.name}: {cfg.n_classes}-class synthetic {cfg.data_kind}, {cfg.n_values} values x "
            f"{cfg.therm_bits}-bit thermometer, {cfg.tuple_bits}-bit tuples"
            f"{' H3-hashed to ' if cfg.hash_h3 else ', '}{cfg.addr_bits}-bit RAM addresses, "
            f"N=2^{cfg.log_n}, {cfg.n_primes}x{cfg.prime_bits}-bit RNS primes")


def bench_config(cfg, bsz, ws, sample_bytes):
    """The `config` object of both arms' lines (the same workload);
    sample_bytes: one encrypted sample."""
    return {"workload": workload_name(cfg), "batch_train": bsz, "batch_test": bsz,
            "l2": "inputs larger than L2 (one step's encrypted batches ~%.0f GB)" %
                  (2 * bsz * sample_bytes / 1e9),
            "parallelism": "replicas" if ws > 1 else "single GPU"}


# -------------------------------------------------------------- the oracle
def _oracle_worker(job):
    """One worker of the CPU baseline: for its RAM j (and class c) the
    oracle encrypts one sample's bits of that RAM, runs the RAM's IVP
    (Algorithm 6) and the VP of class c (Algorithm 7) on them (the work of
    neither depends on the bit values).  Returns single-core seconds per
    encrypted bit slot, per training RAM item and per inference (RAM,
    class) item."""
    cfg_name, j, c, k = job
    sys.path.insert(0, ROOT)
    from oracle import Oracle, wisard
    from synthdata import get_config, make_dataset
    cfg = get_config(cfg_name)
    o = Oracle(cfg)
    vals, labels = make_dataset(cfg, "train", n=1, seed=101 + k)
    s = o.keygen(cfg.key_seed)
    bits = wisard.encode(o.P, vals)
    H = o.new_model()
    t0 = time.perf_counter()
    slots = o.slots_for_rams([j])
    rg = o.encrypt_slots(s, 101, 0, bits[0], labels[0], slots)
    t1 = time.perf_counter()
    o.ivp_item(rg, j)
    t2 = time.perf_counter()
    o.vp_item(H, rg, j, c)
    t3 = time.perf_counter()
    return (t1 - t0) / len(slots), t2 - t1, t3 - t2


def oracle_sample(cfg_name, workers, step=0):
    """The oracle on `workers` processes at once, each on its own (RAM,
    class) of the workload; returns the W-core rate in samples/s
    (one training and one test sample per two samples), the wall time and
    the items measured.  A sample's work is n_slots encrypted bits plus k0
    IVP items (training) or n_data encrypted bits plus k0 * l VP items
    (inference), from the per-item times of the workers."""
    import multiprocessing as mp
    from oracle import Oracle
    from synthdata import get_config
    cfg = get_config(cfg_name)
    P = Oracle(cfg).P
    l = cfg.n_classes
    jobs = []
    for w in range(workers):
        k = step * workers + w
        j = (k * 37) % P.k0
        jobs.append((cfg_name, j, (k * 7) % l, k))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    enc = statistics.mean(r[0] for r in res)
    ivp = statistics.mean(r[1] for r in res)
    vp = statistics.mean(r[2] for r in res)
    t_train = enc * P.n_slots + ivp * P.k0
    t_test = enc * P.n_data + vp * P.k0 * l
    rate = workers * 2.0 / (t_train + t_test)
    return rate, wall, {"items": workers, "enc_s_per_slot": enc, "ivp_s_per_ram": ivp,
                        "vp_s_per_ram_class": vp, "k0": P.k0, "classes": l,
                        "sample_bytes": P.n_slots * o_rgsw_bytes(P)}


def o_rgsw_bytes(P):
    return 2 * P.dnum * 2 * P.r * P.n * 8


def oracle_sample_text(info, wall):
    return (f"{info['items']} worker processes at once, each encrypting one sample's bits of one RAM "
            f"and running that RAM's IVP and one (RAM, class) VP on them; per-sample "
            f"time = per-slot encryption x slots + IVP x {info['k0']} RAMs (training) + VP x "
            f"{info['k0']} x {info['classes']} (inference), {wall:.1f} s wall")


def reference_arm(args, ws, rank):
    if ws > 1 and rank != 0:
        return
    from synthdata import get_config
    cfg = get_config(args.config)
    bsz = args.batch or DEFAULT_BATCH.get(args.config, 16)
    cores = min(os.cpu_count() or 1, 16)
    times = []
    info = None
    for it in range(args.warmup + args.steps):
        rate, wall, info = oracle_sample(args.config, cores, step=it)
        if it >= args.warmup:
            times.append((rate, wall))
    rate = statistics.mean(t[0] for t in times)
    sample = oracle_sample_text(info, statistics.mean(t[1] for t in times))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(t[1] for t in times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": bench_config(cfg, bsz, ws, info["sample_bytes"]),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ the GPU arm
def algorithmic_counts(sess, cfg):
    """algorithmic_work() for a context: its sizes and RAM bit table."""
    from paper_2403_20190_gb300 import binding as B
    return algorithmic_work(sess.sz, B.hw_get_ram_slots(sess.ctx), cfg.n_classes)


def algorithmic_work(sz, slots, l):
    """Modular multiplications of the VP kernel per test sample and of the
    IVP kernel per train sample, counted from the algorithm: every external
    product runs 2*dnum*r forward and 2*r inverse transforms of (N/2) log2 N
    butterflies each, and 2*(2*dnum)*r*N products in evaluation form.
    slots[j*a + i] is the encrypted bit slot of RAM j's address bit i (-1: a
    constant 0, which costs no external product)."""
    n, r, dnum, L, z, a, k0 = (sz["n"], sz["r"], sz["dnum"], sz["L"], sz["z"], sz["a"], sz["k0"])
    logn = n.bit_length() - 1
    bfly = (n // 2) * logn
    per_ext = 2 * dnum * r * bfly + 2 * r * bfly + 2 * 2 * dnum * r * n
    # the pruned CDEMUX tree: gate (level i, j) runs iff a stored index v has
    # v mod 2^(i+1) = j + 2^i (its control is LUT bit i)
    V = set()
    for c in range(l):
        for x in range(1 << max(0, z - L)):
            V.add((c + (x << L)) % (1 << z))
    gate_levels = [i for i in range(z) for jj in range(1 << i)
                   if any(v % (1 << (i + 1)) == jj + (1 << i) for v in V)]
    ext_train = ext_infer = ext_clear = 0
    for j in range(k0):
        enc = [slots[j * a + i] >= 0 for i in range(a)]

        def encrypted(t):  # LUT bit t: label bits are always encrypted
            return t < L or enc[t - L]
        # training: encrypted rotation bits z..L+a-1, then the gates whose
        # control is encrypted
        ext_train += sum(1 for t in range(z, L + a) if encrypted(t))
        ext_train += sum(1 for i in gate_levels if encrypted(i))
        # inference: encrypted address bits among the rotation bits, plus a tree CMUX if z > L
        rot_i = sum(1 for t in range(max(z, L), L + a) if enc[t - L])
        tree_i = 1 if (z > L and enc[z - 1 - L]) else 0
        ext_infer += l * (rot_i + tree_i)
        # inference against a model in clear: one rotation over address bits
        # zt..a-1 shared by the classes, plus the CMUX of address bit 0 per
        # class when zt = 1
        zt = max(0, z - L)
        ext_clear += sum(1 for i in range(zt, a) if enc[i]) + (l if zt and enc[0] else 0)
    return {"per_ext_modmul": per_ext, "ext_train_per_sample": ext_train,
            "ext_infer_per_sample": ext_infer, "ext_clear_per_sample": ext_clear,
            "rgsw_bytes": sz["rgsw_words"] * 8}


class Workload:
    """One workload on one GPU: a session in its tuned geometry, the train and
    test sets resident in HBM as raw bytes, a key, the resident model and the
    server side of a step captured as CUDA graphs (ServerStep)."""

    def __init__(self, name, local, bsz, geometry, rank=0):
        import numpy as np
        import torch

        from paper_2403_20190_gb300.session import ServerStep, Session
        from synthdata import get_config, make_dataset
        self.name, self.bsz = name, bsz
        self.cfg = cfg = get_config(name)
        self.sess = sess = Session(cfg, local, geometry=geometry)
        self.sz = sz = sess.sz
        dev = self.dev = sess.device
        n_pool = max(cfg.n_train, bsz)
        self.tr_vals, self.tr_lab = make_dataset(cfg, "train", n=n_pool)
        self.te_vals, _ = make_dataset(cfg, "test", n=max(cfg.n_test, bsz))
        self.tr_vals_d = torch.from_numpy(self.tr_vals).to(dev)
        self.tr_lab_d = torch.from_numpy(self.tr_lab.astype(np.int32)).to(dev)
        self.te_vals_d = torch.from_numpy(self.te_vals).to(dev)
        self.key = sess.keygen(cfg.key_seed)
        self.model = sess.new_model()
        self.st = ServerStep(sess, self.key, self.model, bsz, bsz)
        self.bits = torch.empty((bsz, sz["n_data"]), dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream()
        self.offset = rank * 7919  # replicas draw different samples
        self.vp_events = []  # (before, after) the inference graph of every timed step

    def client(self, k, host=None):
        """encode + encrypt one train and one test batch (fresh seeds)"""
        from paper_2403_20190_gb300 import binding as B
        bsz, s, st = self.bsz, self.sess, self.st
        n_tr, n_te = self.tr_vals_d.shape[0], self.te_vals_d.shape[0]
        i0 = min(((k * bsz + self.offset) % n_tr), n_tr - bsz)
        j0 = min(((k * bsz + self.offset) % n_te), n_te - bsz)
        if host is not None:
            tv, tl, tev = self.tr_vals_d[:bsz], self.tr_lab_d[:bsz], self.te_vals_d[:bsz]
            tv.copy_(host[0], non_blocking=True)
            tl.copy_(host[1], non_blocking=True)
            tev.copy_(host[2], non_blocking=True)
        else:
            tv, tl = self.tr_vals_d[i0:i0 + bsz], self.tr_lab_d[i0:i0 + bsz]
            tev = self.te_vals_d[j0:j0 + bsz]
        B.hw_encode(s.ctx, tv, bsz, self.bits, self.stream)
        B.hw_encrypt_sample(s.ctx, self.key, self.bits, tl, bsz, 1000 + k, 0, st.rgsw_train, self.stream)
        B.hw_encode(s.ctx, tev, bsz, self.bits, self.stream)
        B.hw_encrypt_sample(s.ctx, self.key, self.bits, None, bsz, 500000 + k, 0, st.rgsw_test, self.stream)

    def step(self, k, host=None, time_vp=False):
        import torch
        self.client(k, host)
        if time_vp:
            pair = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            self.vp_events.append(pair)
            self.st.replay(between=lambda i: pair[i].record(self.stream) if i < 2 else None)
        else:
            self.st.replay()
        if host is not None:
            host[3].copy_(self.st.labels, non_blocking=True)

    def warm(self, warmup):
        import torch
        for k in range(warmup):
            self.client(k)
            self.st.run()
        self.st.capture()  # the server side of a step as CUDA graphs (train, infer, post)
        torch.cuda.synchronize()

    def timed(self, k0, steps, barrier=lambda: None):
        """Device time (ms) of `steps` steps, CUDA events on the launching
        stream, a barrier and a synchronize on both sides."""
        import torch
        barrier()
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(self.stream)
        for k in range(steps):
            self.step(k0 + k, time_vp=True)
        end.record(self.stream)
        torch.cuda.synchronize()
        barrier()
        return start.elapsed_time(end)

    def phases(self, k):
        """Per-call device times (ms) of one eager step with events between
        the calls."""
        import torch

        from paper_2403_20190_gb300 import binding as B
        s, st, bsz, stream = self.sess, self.st, self.bsz, self.stream
        names = ["t0", "t1", "t2", "t3", "t4", "t5"]
        evs = {nm: torch.cuda.Event(enable_timing=True) for nm in names}
        evs["t0"].record(stream)
        B.hw_encode(s.ctx, self.tr_vals_d[:bsz], bsz, self.bits, stream)
        B.hw_encrypt_sample(s.ctx, self.key, self.bits, self.tr_lab_d[:bsz], bsz, 1000 + k, 0, st.rgsw_train,
                            stream)
        evs["t1"].record(stream)
        B.hw_train_accumulate(s.ctx, self.model, st.rgsw_train, bsz, st.scratch, stream)
        evs["t2"].record(stream)
        B.hw_encode(s.ctx, self.te_vals_d[:bsz], bsz, self.bits, stream)
        B.hw_encrypt_sample(s.ctx, self.key, self.bits, None, bsz, 500000 + k, 0, st.rgsw_test, stream)
        evs["t3"].record(stream)
        resp, sums, scr = st.ibufs
        B.hw_infer(s.ctx, self.model, st.rgsw_test, bsz, resp, sums, scr, stream)
        evs["t4"].record(stream)
        B.hw_decrypt(s.ctx, self.key, B.HW_DEC_LWE, resp, bsz * self.cfg.n_classes * self.sz["k0"], st.counts,
                     stream)
        B.hw_pdact(s.ctx, st.counts, bsz, st.scores, st.labels, stream)
        evs["t5"].record(stream)
        torch.cuda.synchronize()
        keys = ["encrypt_train", "train", "encrypt_test", "infer", "decrypt_pdact"]
        return {kn: evs[a].elapsed_time(evs[b]) for a, b, kn in zip(names[:-1], names[1:], keys)}

    def rooflines(self, ph, local, ceiling=None):
        """Roofline of the VP kernel (the dominant one: its graph's average
        duration over the timed steps) and of the IVP kernel (the training
        call of the phase breakdown), against the integer-multiply peak."""
        import torch
        pk, _ = peaks()
        alg = algorithmic_counts(self.sess, self.cfg)
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        word_bits = self.sz["word_bits"]  # the external product's word width in this context
        muls = MULS_PER_MODMUL32 if word_bits == 32 else MULS_PER_MODMUL
        peak_modmul = sm_count * IMAD_PER_CLK_PER_SM * sm_mhz * 1e6 / muls
        peak_kind = (f"derived: {sm_count} SMs x {IMAD_PER_CLK_PER_SM} int32 multiplies/clk x "
                     f"{sm_mhz:.0f} MHz / {muls} per {word_bits}-bit modular product")
        infer_modmul = alg["ext_infer_per_sample"] * self.bsz * alg["per_ext_modmul"]
        vp_ms = (statistics.mean(a.elapsed_time(b) for a, b in self.vp_events) if self.vp_events
                 else ph["infer"])
        achieved = infer_modmul / (vp_ms / 1000.0)
        vp = {"bound": "alu", "kernel": "k_vp_infer", "achieved": achieved / 1e12,
              "peak": peak_modmul / 1e12, "unit": "T modmul/s", "frac": achieved / peak_modmul,
              "traffic": profiled_traffic(self.name, self.sess.geometry, self.bsz),
              "algorithmic_rgsw_bytes": alg["rgsw_bytes"] * alg["ext_infer_per_sample"] // self.cfg.n_classes
              * self.bsz, "launch_ms": vp_ms, "peak_kind": peak_kind,
              "work": f"{alg['ext_infer_per_sample']} external products x {alg['per_ext_modmul']} modular "
                      f"products per test sample, {self.bsz} test samples per launch"}
        if ceiling:
            # the measured issue ceiling of the butterflies this context runs
            # (register-only loops, hw_butterfly_rates), beside the derived peak
            ct, gs = ("ct32", "gs32") if word_bits == 32 else ("ct64", "gs64")
            vp["butterfly_ceiling"] = {"ct_t_per_s": ceiling[ct] / 1e3, "gs_t_per_s": ceiling[gs] / 1e3,
                                       "source": "hw_butterfly_rates, measured in this run"}
        train_modmul = alg["ext_train_per_sample"] * self.bsz * alg["per_ext_modmul"]
        ivp_achieved = train_modmul / (ph["train"] / 1000.0)
        ivp = {"bound": "alu", "kernel": "k_ivp_train + k_model_reduce", "achieved": ivp_achieved / 1e12,
               "peak": peak_modmul / 1e12, "unit": "T modmul/s", "frac": ivp_achieved / peak_modmul,
               "launch_ms": ph["train"],
               "work": f"{alg['ext_train_per_sample']} external products per training sample"}
        return vp, ivp, alg

    def ntt(self, count=None):
        """Batched forward NTT of this ring (one read + one write per
        polynomial, inputs larger than L2)."""
        import torch

        from paper_2403_20190_gb300 import binding as B
        pk, pk_kind = peaks()
        nn = self.sz["n"]
        if count is None:
            count = (1 << 31) // (nn * 8)  # 2 GiB of polynomials
        polys = self.sess.words(count * nn)
        for _ in range(3):
            B.hw_ntt_forward(self.sess.ctx, polys, count, self.stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(self.stream)
        for _ in range(reps):
            B.hw_ntt_forward(self.sess.ctx, polys, count, self.stream)
        e1.record(self.stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps / 1000.0
        gbs = 2.0 * count * nn * 8 / t / 1e9
        del polys
        g = self.sess.geometry
        return {"gbs": gbs, "frac_of_hbm": gbs / pk["hbm_gbs"], "peak_gbs": pk["hbm_gbs"], "peak_kind": pk_kind,
                "polys": count, "n": nn, "prime_bits": self.cfg.prime_bits, "ms_per_launch": t * 1000.0,
                "variant": f"radix {1 << g['ntt_loge']}, {32 * g['ntt_limbs']}-bit words"}

    def keyswitch(self, infer_ms, ceiling=None):
        """PackingKeySwitching of the last test batch's responses: the key's
        generation once, then the best of two packing passes.  Each sample
        needs N * dnum * r forward transforms (one per key row and prime) and
        2 r inverse ones; against the measured 64-bit butterfly rate that
        sets a floor under the pass."""
        import torch

        from paper_2403_20190_gb300 import binding as B
        sess, st, sz, stream, bsz = self.sess, self.st, self.sz, self.stream, self.bsz
        resp = st.ibufs[0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ksk = sess.ksk_gen(self.key, self.cfg.key_seed + 1, stream=stream)
        e1.record(stream)
        pscr = sess.words(B.hw_pack_scratch_words(sess.ctx, bsz), zero=False)
        sess.pack_responses(ksk, resp, bsz, scratch=pscr, stream=stream)  # warm-up
        torch.cuda.synchronize()
        t_pack = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sess.pack_responses(ksk, resp, bsz, scratch=pscr, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            t_pack.append(a.elapsed_time(b))
        n, r, dnum = sz["n"], sz["r"], sz["dnum"]
        log_n = n.bit_length() - 1
        bfly = bsz * (n * dnum * r + 2 * r) * (n // 2) * log_n
        best = min(t_pack)
        out = {"workload": self.name, "batch": bsz, "pack_ms_per_step": best,
               "ksk_gen_ms_once": e0.elapsed_time(e1),
               "ksk_bytes": B.hw_ksk_words(sess.ctx) * 8, "pack_scratch_bytes": pscr.numel() * 8,
               "response_bytes_per_sample": {"lwe": sz["resp_words"] * 8, "packed": sz["rlwe_words"] * 8},
               "share_of_infer": best / infer_ms,
               "transforms_per_sample": n * dnum * r + 2 * r,
               "butterflies_per_s": bfly / (best * 1e-3)}
        if ceiling:
            floor_ms = bfly / (ceiling["ct64"] * 1e9) * 1e3
            out["butterfly_frac"] = out["butterflies_per_s"] / (ceiling["ct64"] * 1e9)
            out["share_of_infer_at_butterfly_ceiling"] = floor_ms / infer_ms
        del ksk, pscr
        return out

    def packed_inference(self, infer_ms):
        """Horizontal packing (Section 6) on the last test batch: the packed
        VP against the plain one's phase time, and whether every packed
        response decrypts to the plain path's counter."""
        import torch
        sess, st, sz, stream, bsz = self.sess, self.st, self.sz, self.stream, self.bsz
        groups = min(self.cfg.n_classes, 1 << sz["z"]) if sz["z"] <= sz["L"] else self.cfg.n_classes
        bufs = sess.infer_buffers(bsz)
        sess.infer(self.model, st.rgsw_test, bsz, bufs=bufs, stream=stream, packed=True)  # warm-up
        torch.cuda.synchronize()
        ts = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sess.infer(self.model, st.rgsw_test, bsz, bufs=bufs, stream=stream, packed=True)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        pc = sess.responses_counts(self.key, bufs[0], bsz, stream=stream)
        same = (pc.reshape(-1) == st.counts[: pc.numel()]).float().mean().item()
        del bufs
        return {"workload": self.name, "batch": bsz, "inferences_per_s_plain": bsz / (infer_ms / 1000.0),
                "inferences_per_s_packed": bsz / (min(ts) / 1000.0),
                "vp_per_sample": {"plain": self.cfg.n_classes * sz["k0"], "packed": groups * sz["k0"]},
                "responses_equal_to_plain_path": same}

    def summary(self, elapsed_ms, steps, ws, local, with_ntt=True, ceiling=None):
        ph = self.phases(1000 + steps)
        vp, ivp, _ = self.rooflines(ph, local, ceiling)
        out = {"workload": workload_name(self.cfg), "batch": self.bsz, "steps": steps,
               "samples_per_s": 2 * self.bsz * steps * ws / (elapsed_ms / 1000.0),
               "ms_per_step": elapsed_ms / steps,
               "train_samples_per_s": self.bsz / (ph["train"] / 1000.0),
               "inferences_per_s": self.bsz / (ph["infer"] / 1000.0),
               "phases_ms": ph, "roofline": vp, "roofline_ivp": ivp, "geometry": self.sess.geometry}
        if with_ntt:
            out["ntt"] = self.ntt()
        return out, ph


def gpu_arm(args, ws, rank, local, pg):
    import numpy as np
    import torch

    from paper_2403_20190_gb300 import binding as B
    from paper_2403_20190_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(local)
    tune = None
    geometry = None
    per_names = [nm for nm in ALL_CONFIGS if nm != args.config] if args.per_config_steps > 0 else []
    if args.geometry == "auto":
        from paper_2403_20190_gb300.tuning import tuned_geometry
        from synthdata import get_config
        t0 = time.perf_counter()
        geometry, entries, cached = tuned_geometry(get_config(args.config), local)
        tune = {"cached": cached, "seconds": round(time.perf_counter() - t0, 2), "candidates": entries}
        # every other parameter set the legs use is tuned now, before this
        # process holds any context or buffer: the tuner's probe contexts come
        # and go while nothing else is resident, and the legs find the cache
        others = set(per_names)
        if not args.no_packing:
            others.add("cfg1")
        if not args.no_serve:
            others.update(ALL_CONFIGS)
        for nm in sorted(others - {args.config}):
            tuned_geometry(get_config(nm), local)
    geo = "auto" if args.geometry == "auto" else None
    ceiling = B.hw_butterfly_rates(local)  # before any context holds the GPU
    bsz = args.batch or DEFAULT_BATCH.get(args.config, 16)
    w = Workload(args.config, local, bsz, geometry if geometry is not None else None, rank)
    cfg, sess, sz, st, stream = w.cfg, w.sess, w.sz, w.st, w.stream
    if tune is not None:
        tune["chosen"] = sess.geometry

    def healthy(where):
        """Stop before launching on a context whose device tables changed."""
        try:
            B.hw_check_context(sess.ctx)
        except B.HwError as e:
            raise RuntimeError(f"context check failed after {where}: {e}") from None

    def barrier():
        if pg is not None:
            pg.barrier()

    w.warm(args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = B.hw_launch_count(sess.ctx)
    elapsed_ms = w.timed(args.warmup, args.steps, barrier)
    launches = B.hw_launch_count(sess.ctx) - launches0 + st.launches_per_step * args.steps
    clk = clocks.stop()
    if pg is not None:
        t = torch.tensor([elapsed_ms], device=w.dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    total_samples = 2 * bsz * args.steps * ws
    value = total_samples / (elapsed_ms / 1000.0)
    ph = w.phases(args.warmup + args.steps)
    roofline, roofline_ivp, alg = w.rooflines(ph, local, ceiling)
    healthy("the timed steps")

    key, model = w.key, w.model
    # dataset balancing (Section 3.6.1) on the same step: the label-bit IVP
    # over the training batch into the class-count ciphertext, its
    # decryption and the balanced PD-act of the test batch
    balancing = None
    if not args.no_balance:
        bal_counts = sess.new_counts()
        bal_scr = sess.words(B.hw_count_scratch_words(sess.ctx, bsz), zero=False)
        for _ in range(2):
            sess.count_classes(bal_counts, st.rgsw_train, bsz, scratch=bal_scr, stream=stream)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sess.count_classes(bal_counts, st.rgsw_train, bsz, scratch=bal_scr, stream=stream)
        e1.record(stream)
        cc = sess.class_counts(key, bal_counts, stream=stream)
        sess.pdact_balanced(st.counts, cc, bsz, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        t_count, t_post = e0.elapsed_time(e1), e1.elapsed_time(e2)
        balancing = {"count_ms_per_step": t_count, "decrypt_pdact_ms": t_post,
                     "share_of_step": (t_count + t_post) / (elapsed_ms / args.steps),
                     "ext_products_per_sample": sz["L"]}
        del bal_scr
    healthy("the balancing leg")

    # PackingKeySwitching (Section 2.4): the test batch's responses packed
    # into one RLWE per sample (what Algorithm 7 returns for PD-act)
    keyswitch = None if args.no_keyswitch else w.keyswitch(ph["infer"], ceiling)
    healthy("the key-switching leg")
    packed_main = None
    if not args.no_packing and args.config != "cfg1":
        packed_main = w.packed_inference(ph["infer"])
    healthy("the packed-inference leg")

    # inference against the model in clear (Section 3.6.2): the owner's
    # decrypted counters as plaintext tables, one blind rotation per (sample,
    # RAM) shared by the l classes; the same encrypted test batch as the
    # phase breakdown's, whose decrypted counters it must reproduce
    clear_model = None
    if not args.no_clear_model:
        W = sess.decrypt_model_counts(key, model, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plain = sess.plain_model(W, stream=stream)
        e1.record(stream)
        pbufs = sess.infer_buffers(bsz)
        sess.infer_plain(plain, st.rgsw_test, bsz, bufs=pbufs, stream=stream)  # warm-up
        torch.cuda.synchronize()
        t_load = e0.elapsed_time(e1)
        t_plain = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sess.infer_plain(plain, st.rgsw_test, bsz, bufs=pbufs, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            t_plain.append(a.elapsed_time(b))
        pc = sess.responses_counts(key, pbufs[0], bsz, stream=stream)
        same = (pc.reshape(-1) == st.counts[: pc.numel()]).float().mean().item()
        clear_model = {"inferences_per_s": bsz / (min(t_plain) / 1000.0),
                       "ms_per_batch": min(t_plain), "encrypted_model_ms_per_batch": ph["infer"],
                       "speedup_vs_encrypted_model": ph["infer"] / min(t_plain),
                       "load_ms": t_load, "plain_bytes": B.hw_plain_model_words(sess.ctx) * 8,
                       "ext_products_per_sample": {"clear": alg["ext_clear_per_sample"],
                                                   "encrypted": alg["ext_infer_per_sample"]},
                       "responses_equal_to_encrypted_path": same}
        del plain, pbufs, W
    healthy("the clear-model leg")

    # e2e through the C ABI with pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_tr = torch.from_numpy(w.tr_vals[:bsz].copy()).pin_memory()
        h_lab = torch.from_numpy(w.tr_lab[:bsz].astype(np.int32)).pin_memory()
        h_te = torch.from_numpy(w.te_vals[:bsz].copy()).pin_memory()
        h_out = torch.empty(bsz, dtype=torch.int32).pin_memory()
        host = (h_tr, h_lab, h_te, h_out)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            w.step(args.warmup + args.steps + 1 + k, host)
            torch.cuda.current_stream().synchronize()
            _ = int(h_out[0])
        t1 = time.perf_counter()
        e2e_s = t1 - t0
        if pg is not None:
            t = torch.tensor([e2e_s], device=w.dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": total_samples / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h_tr.numel() + h_lab.numel() * 4 + h_te.numel()),
               "d2h_bytes_per_step": int(h_out.numel() * 4)}
    healthy("the end-to-end leg")

    ntt = None if args.no_ntt else w.ntt()
    healthy("the NTT leg")

    # the same workload one request at a time: each request one train and one
    # test sample, encoded, encrypted, trained, inferred, decrypted, waited for
    single = None
    if not args.no_serve:
        n1 = 6
        bits1 = w.bits
        t0 = time.perf_counter()
        for k in range(n1):
            B.hw_encode(sess.ctx, w.tr_vals_d[k:k + 1], 1, bits1, stream)
            B.hw_encrypt_sample(sess.ctx, key, bits1, w.tr_lab_d[k:k + 1], 1, 9000 + k, 0, st.rgsw_train, stream)
            B.hw_train_accumulate(sess.ctx, model, st.rgsw_train, 1, st.scratch, stream)
            B.hw_encode(sess.ctx, w.te_vals_d[k:k + 1], 1, bits1, stream)
            B.hw_encrypt_sample(sess.ctx, key, bits1, None, 1, 19000 + k, 0, st.rgsw_test, stream)
            resp, sums, scr = st.ibufs
            B.hw_infer(sess.ctx, model, st.rgsw_test, 1, resp, sums, scr, stream)
            B.hw_decrypt(sess.ctx, key, B.HW_DEC_LWE, resp, cfg.n_classes * sz["k0"], st.counts, stream)
            B.hw_pdact(sess.ctx, st.counts, 1, st.scores, st.labels, stream)
            _ = int(st.labels[0].item())
        single = {"samples_per_s": 2 * n1 / (time.perf_counter() - t0), "requests": n1,
                  "request": "1 train + 1 test sample, synchronous"}
        healthy("the one-at-a-time requests")
    sample_bytes = sz["sample_words"] * 8
    del w, st, sess, key, model
    torch.cuda.synchronize()
    torch.cuda.empty_cache()

    # horizontal packing (Section 6): plain vs packed inference on the
    # Wisconsin-shaped ring (label bits low, z = 0: one VP answers both
    # classes); the digit workloads keep a stored ciphertext per class
    packing = None
    if not args.no_packing:
        packing = packing_leg(local, geo)
        if packed_main is not None:
            packing = {"cfg1": packing, args.config: packed_main}

    # the other workloads, shorter: the same step, its rooflines and the
    # batched NTT at its primes
    per_config = {}
    for nm in per_names:
        pw = Workload(nm, local, DEFAULT_BATCH[nm], geo, rank)
        pw.warm(1)
        pms = pw.timed(1, args.per_config_steps, barrier)
        per_config[nm], pph = pw.summary(pms, args.per_config_steps, ws, local, with_ntt=not args.no_ntt,
                                         ceiling=ceiling)
        if nm == "cfg2" and not args.no_keyswitch:
            per_config[nm]["packing_keyswitch"] = pw.keyswitch(pph["infer"], ceiling)
        del pw
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    serving = serve_leg(args, local) if not args.no_serve else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, 16)
        rate, wall, info = oracle_sample(args.config, cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": oracle_sample_text(info, wall)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": bench_config(cfg, bsz, ws, sample_bytes),
            "server_step": "CUDA graphs (IVP + accumulate, VP + sums, decrypt + PD-act)",
            "train_samples_per_s": bsz / (ph["train"] / 1000.0),
            "inferences_per_s": bsz / (ph["infer"] / 1000.0),
            "phases_ms": ph,
            "roofline": roofline,
            "roofline_ivp": roofline_ivp,
            "ntt": ntt,
            "per_config": per_config,
            "balancing": balancing,
            "horizontal_packing": packing,
            "packing_keyswitch": keyswitch,
            "clear_model": clear_model,
            "geometry": tune["chosen"] if tune else None,
            "autotune": tune,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "p99_ms": serving["batched"]["p99_ms"] if serving else None,
            "serving": serving,
            "one_request_at_a_time": single,
        }
        print(json.dumps(line), flush=True)


def packing_leg(local, geo):
    import torch

    from paper_2403_20190_gb300.session import Session
    from synthdata import get_config, make_dataset
    pc = get_config("cfg1")
    ps = Session(pc, local, geometry=geo)
    n_p = 100
    pv, _ = make_dataset(pc, "test", n=n_p)
    pkey = ps.keygen(pc.key_seed)
    pbits = ps.encode(torch.from_numpy(pv).to(ps.device))
    prg = ps.encrypt(pkey, pbits, None, seed=4242)
    pmodel = ps.new_model()
    pbufs = ps.infer_buffers(n_p)
    rates = {}
    for mode in (False, True):
        ts = []
        for k in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ps.infer(pmodel, prg, n_p, bufs=pbufs, packed=mode)
            b.record()
            torch.cuda.synchronize()
            if k:
                ts.append(a.elapsed_time(b))
        rates["packed" if mode else "plain"] = n_p / (min(ts) / 1000.0)
    psz = ps.sz
    groups = min(pc.n_classes, 1 << psz["z"]) if psz["z"] <= psz["L"] else pc.n_classes
    return {"workload": "cfg1", "inferences_per_s_plain": rates["plain"],
            "inferences_per_s_packed": rates["packed"],
            "vp_per_sample": {"plain": pc.n_classes * psz["k0"], "packed": groups * psz["k0"]}}


# per-request sample caps of the serving mix: what the footprint rule leaves
# for one request (786 MiB, 3.9 GiB, 15.5 GiB per encrypted cfg2/3/4 sample)
SERVE_MAX = {"cfg1": 256, "cfg2": 16, "cfg3": 2, "cfg4": 1}


def serve_leg(args, local):
    """Seeded Poisson streams (200 requests/s) of train and infer requests over
    the four workloads, served with continuous batching and, for comparison,
    one request at a time; latency is arrival to completion.  Three seeds."""
    import copy

    import torch

    from paper_2403_20190_gb300.serve import ResidentModel, Server, latency_stats, poisson_stream
    from synthdata import get_config
    cfgs = {nm: get_config(nm) for nm in ALL_CONFIGS}
    geo = "auto" if args.geometry == "auto" else None
    models = {nm: ResidentModel(c, local, key_seed=c.key_seed, geometry=geo) for nm, c in cfgs.items()}
    from paper_2403_20190_gb300.arena import DeviceArena
    budget = 120 << 30
    arena = DeviceArena(budget, torch.device("cuda", local))  # shared by every mode
    modes = {
        "batched": dict(n_streams=1, packed_infer=True, policy="fifo"),
        "batched_without_packing": dict(n_streams=1, packed_infer=False, policy="fifo"),
        "batched_sjf_2_streams": dict(n_streams=2, packed_infer=True, policy="sjf"),
    }
    warm = poisson_stream(cfgs, n_requests=4, rate=200.0, seed=1, max_samples=SERVE_MAX)
    Server(models, arena=arena).run(warm, realtime=False)
    runs = {m: [] for m in list(modes) + ["one_at_a_time"]}
    costs = None
    for seed in (2024, 2025, 2026):
        reqs = poisson_stream(cfgs, n_requests=args.serve_requests, rate=200.0, seed=seed,
                              max_samples=SERVE_MAX)
        for m, kw in modes.items():
            srv = Server(models, arena=arena, **kw)
            c = srv.calibrate()  # startup, outside the timed runs
            costs = costs or c
            runs[m].append(latency_stats(srv.run(copy.deepcopy(reqs), realtime=True)))
        runs["one_at_a_time"].append(latency_stats(
            Server(models, arena=arena, packed_infer=False).run_one_at_a_time(copy.deepcopy(reqs))))

    def summary(rs):
        keys = ("samples_per_s", "p50_ms", "p99_ms")
        out = {k: statistics.mean(r[k] for r in rs) for k in keys}
        out["runs"] = rs
        return out
    out = {"requests": args.serve_requests, "rate_per_s": 200.0, "hbm_budget_gb": budget / 2**30,
           "seeds": [2024, 2025, 2026], **{m: summary(rs) for m, rs in runs.items()},
           "policy": "batched: one stream, groups launched oldest request first, every pending request of "
                     "the same (workload, kind) joins its group (up to 256 samples), device arena, at most "
                     "one training batch in flight per model, inference with horizontal packing where the "
                     "tree layout allows (cfg1, cfg3); the one-at-a-time baseline runs the plain path",
           "calibrated_ms_per_sample": {f"{k[0]}/{k[1]}": round(v * 1e3, 3) for k, v in costs.items()},
           "max_samples_per_request": SERVE_MAX}
    out["batched_vs_one_at_a_time"] = out["batched"]["samples_per_s"] / out["one_at_a_time"]["samples_per_s"]
    del models, arena
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    ws, rank, local, pg = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, ws, rank)
    else:
        gpu_arm(args, ws, rank, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
