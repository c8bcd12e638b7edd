#!/usr/bin/env python3
"""Benchmark of the encrypted WiSARD hot path on GB300; prints one JSON line.

A step is one pass of the whole path over one batch: B training samples are
encoded, RGSW-encrypted and trained into the resident model (IVP +
accumulate), and B test samples are encoded, encrypted, inferred (VP,
ExtractLWE, class sums), decrypted and classified with PD-act.  The workload
is the batched 10-class 28x28 digit configuration (N = 4096, two ~50-bit RNS
primes, 131 RAMs of 2^12 entries).  Raw samples sit in HBM before the timed
region; encrypted batches (~50 GB per step) are far larger than L2.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="cfg2")
    ap.add_argument("--batch", type=int, default=0,
                    help="samples per step (0: the workload's default, sized to fit HBM)")
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


# DRAM bytes of k_vp_infer per test sample, from an ncu capture of the
# inference kernel on 2 cfg2 test samples (scaled by samples: the
# traffic is per item); valid only for the kernel sources it was taken on:
# the VP kernel with the device helpers it calls (the region of hw_ext.cuh
# from bit_slot to the VP kernel's end) and the headers of the external
# product and the modular arithmetic.
PROFILED_VP_TRAFFIC = {
    "config": "cfg2", "ext_loge": 3, "ext_np": 2, "ext_smem": 1, "ext_blocks_per_sm": 1, "l2_persist": 0,
    "bytes_per_test_sample": 2.1133e9,
    "sources": (("paper_2403_20190_gb300/csrc/hw_ext.cuh", "// Encrypted bit slot that drives",
                 "// EncRGSW."),
                ("paper_2403_20190_gb300/csrc/hw_ext.cuh", "// ExtractLWE(ct, k) written by the block",
                 "// Dataset balancing (Section 3.6.1)"),
                ("paper_2403_20190_gb300/csrc/hw_internal.cuh", None, None),
                ("paper_2403_20190_gb300/csrc/modarith.cuh", None, None)),
    "sha256": "1b1c5d9b6538dd97528c71efa032a025f17669d8cca0d819f28b729fc8fef19d",
}
# Register-only 64-bit lazy Cooley-Tukey butterflies per second on one GB300
# at 2070 MHz (a register-only microbenchmark): what the integer pipes issue
# for this arithmetic, beside the multiply-count peak.
BUTTERFLY_CEILING = {"ct64_t_per_s": 0.8414, "gs64_t_per_s": 0.8755,
                     "source": "microbench/bfly_ceiling.cu"}
BUTTERFLY_CEILING32 = {"ct32_t_per_s": 3.1435, "gs32_t_per_s": 3.0782,
                       "source": "microbench/bfly_ceiling.cu"}


def profiled_sources_sha(root=None):
    """sha256 over the profiled source regions (whole file where no markers)."""
    import hashlib
    h = hashlib.sha256()
    for f, start, end in PROFILED_VP_TRAFFIC["sources"]:
        with open(os.path.join(root or ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        if start is not None:
            i = text.index(start)
            text = text[i:text.index(end, i)]
        h.update(text.encode("utf-8"))
    return h.hexdigest()


def profiled_traffic(config, geometry, n_test):
    t = PROFILED_VP_TRAFFIC
    if config != t["config"] or any(geometry.get(k) != t[k] for k in
                                    ("ext_loge", "ext_np", "ext_smem", "ext_blocks_per_sm", "l2_persist")):
        return None
    if profiled_sources_sha() != t["sha256"]:
        return None  # the kernel changed since the counters were taken
    return t["bytes_per_test_sample"] * n_test


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


# -------------------------------------------------------------- the oracle
def _oracle_worker(job):
    """One worker of the CPU baseline: the oracle encrypts one train and one
    test sample's bits for its RAMs, runs the IVP of each RAM and the VP of
    each (RAM, class); returns the seconds it took."""
    cfg_name, rams = job
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import Oracle, wisard
    from synthdata import get_config, make_dataset
    cfg = get_config(cfg_name)
    t0 = time.perf_counter()
    o = Oracle(cfg)
    vals, labels = make_dataset(cfg, "train", n=1)
    tvals, _ = make_dataset(cfg, "test", n=1)
    s = o.keygen(cfg.key_seed)
    bits = wisard.encode(o.P, vals)
    tbits = wisard.encode(o.P, tvals)
    H = o.train(o.new_model(), s, 101, bits, labels, rams=rams)
    o.infer(H, s, 202, tbits, rams=rams)
    _ = np
    return time.perf_counter() - t0


def oracle_sample(cfg_name, k0, workers, rams_per_worker=1):
    import multiprocessing as mp
    jobs = []
    stride = max(1, k0 // (workers * rams_per_worker))
    r = 0
    for w in range(workers):
        rams = [(r + t * stride) % k0 for t in range(rams_per_worker)]
        r += 1
        jobs.append((cfg_name, rams))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    rams_done = workers * rams_per_worker
    samples = 2.0 * rams_done / k0  # one train + one test sample, over all k0 RAMs
    return samples / wall, wall, rams_done


def reference_arm(args, ws, rank):
    if ws > 1 and rank != 0:
        return
    from synthdata import get_config
    from oracle import Oracle
    cfg = get_config(args.config)
    k0 = Oracle(cfg).P.k0
    cores = min(os.cpu_count() or 1, 16)
    times = []
    for it in range(args.warmup + args.steps):
        rate, wall, rams = oracle_sample(args.config, k0, cores)
        if it >= args.warmup:
            times.append((rate, wall, rams))
    rate = statistics.mean(t[0] for t in times)
    sample = (f"per step: 1 train + 1 test sample restricted to {times[0][2]} of {k0} RAMs "
              f"(one RAM per worker process), scaled by {k0}/{times[0][2]}")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(t[1] for t in times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": workload_name(cfg), "sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_name(cfg):
    return (f"{cfg.name}: {cfg.n_classes}-class synthetic {cfg.data_kind}, {cfg.n_values} values x "
            f"{cfg.therm_bits}-bit thermometer, {cfg.addr_bits}-bit RAM addresses, "
            f"N=2^{cfg.log_n}, {cfg.n_primes}x{cfg.prime_bits}-bit RNS primes")


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


# samples per step: cfg1's whole test set; for the larger rings, what keeps one
# encrypted batch (786 MiB, 3.9 GiB, 15.5 GiB per sample) plus scratch well
# inside HBM
DEFAULT_BATCH = {"cfg1": 100, "cfg2": 64, "cfg3": 16, "cfg4": 4}


def gpu_arm(args, ws, rank, local, pg):
    import numpy as np
    import torch

    from paper_2403_20190_gb300 import binding as B
    from paper_2403_20190_gb300 import build as libbuild
    from paper_2403_20190_gb300.session import ServerStep, Session
    from synthdata import get_config, make_dataset

    libbuild.build()
    torch.cuda.set_device(local)
    cfg = get_config(args.config)
    tune = None
    geometry = None
    if args.geometry == "auto":
        from paper_2403_20190_gb300.tuning import tuned_geometry
        t0 = time.perf_counter()
        geometry, entries, cached = tuned_geometry(cfg, local)
        tune = {"cached": cached, "seconds": round(time.perf_counter() - t0, 2), "candidates": entries}
        # every other parameter set the legs use is tuned now, before this
        # process holds any context or buffer: the tuner's probe contexts come
        # and go while nothing else is resident, and the legs find the cache
        others = set()
        if not (args.no_ntt and args.no_packing) and args.config != "cfg1":
            others.add("cfg1")
        if not args.no_serve:
            others.update(("cfg1", "cfg2", "cfg3", "cfg4"))
        for nm in sorted(others - {args.config}):
            tuned_geometry(get_config(nm), local)
    sess = Session(cfg, local, geometry=geometry)

    def healthy(where):
        """Stop before launching on a context whose device tables changed."""
        try:
            B.hw_check_context(sess.ctx)
        except B.HwError as e:
            raise RuntimeError(f"context check failed after {where}: {e}") from None
    if tune is not None:
        tune["chosen"] = sess.geometry
    dev = sess.device
    bsz = args.batch or DEFAULT_BATCH.get(args.config, 16)
    sz = sess.sz
    n_pool = max(cfg.n_train, bsz)
    # the whole train / test sets of the workload, resident in HBM as raw bytes
    tr_vals, tr_lab = make_dataset(cfg, "train", n=n_pool)
    te_vals, _ = make_dataset(cfg, "test", n=max(cfg.n_test, bsz))
    tr_vals_d = torch.from_numpy(tr_vals).to(dev)
    tr_lab_d = torch.from_numpy(tr_lab.astype(np.int32)).to(dev)
    te_vals_d = torch.from_numpy(te_vals).to(dev)

    key = sess.keygen(cfg.key_seed)
    model = sess.new_model()
    st = ServerStep(sess, key, model, bsz, bsz)
    bits = torch.empty((bsz, sz["n_data"]), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    n_tr = tr_vals_d.shape[0]
    n_te = te_vals_d.shape[0]
    offset = rank * 7919  # replicas draw different samples

    def client(k, host=None):
        """encode + encrypt one train and one test batch (fresh seeds)"""
        i0 = min(((k * bsz + offset) % n_tr), n_tr - bsz)
        j0 = min(((k * bsz + offset) % n_te), n_te - bsz)
        if host is not None:
            tv, tl, tev = tr_vals_d[:bsz], tr_lab_d[:bsz], te_vals_d[:bsz]
            tv.copy_(host[0], non_blocking=True)
            tl.copy_(host[1], non_blocking=True)
            tev.copy_(host[2], non_blocking=True)
        else:
            tv, tl, tev = tr_vals_d[i0:i0 + bsz], tr_lab_d[i0:i0 + bsz], te_vals_d[j0:j0 + bsz]
        B.hw_encode(sess.ctx, tv, bsz, bits, stream)
        B.hw_encrypt_sample(sess.ctx, key, bits, tl, bsz, 1000 + k, 0, st.rgsw_train, stream)
        B.hw_encode(sess.ctx, tev, bsz, bits, stream)
        B.hw_encrypt_sample(sess.ctx, key, bits, None, bsz, 500000 + k, 0, st.rgsw_test, stream)

    vp_events = []  # (before, after) the inference graph of every timed step

    def step(k, host=None, time_vp=False):
        client(k, host)
        if time_vp:
            pair = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            vp_events.append(pair)
            st.replay(between=lambda i: pair[i].record(stream) if i < 2 else None)
        else:
            st.replay()
        if host is not None:
            host[3].copy_(st.labels, non_blocking=True)

    for k in range(args.warmup):
        client(k)
        st.run()
    st.capture()  # the server side of a step as CUDA graphs (train, infer, post)
    torch.cuda.synchronize()

    def barrier():
        if pg is not None:
            pg.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = B.hw_launch_count(sess.ctx)
    barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, time_vp=True)
    end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = B.hw_launch_count(sess.ctx) - launches0 + st.launches_per_step * args.steps
    clk = clocks.stop()
    elapsed_ms = start.elapsed_time(end)
    if pg is not None:
        t = torch.tensor([elapsed_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    total_samples = 2 * bsz * args.steps * ws
    value = total_samples / (elapsed_ms / 1000.0)

    # phase breakdown from one extra eager step with events between the calls
    names = ["t0", "t1", "t2", "t3", "t4", "t5"]
    evs = {nm: torch.cuda.Event(enable_timing=True) for nm in names}
    k = args.warmup + args.steps
    evs["t0"].record(stream)
    B.hw_encode(sess.ctx, tr_vals_d[:bsz], bsz, bits, stream)
    B.hw_encrypt_sample(sess.ctx, key, bits, tr_lab_d[:bsz], bsz, 1000 + k, 0, st.rgsw_train, stream)
    evs["t1"].record(stream)
    B.hw_train_accumulate(sess.ctx, model, st.rgsw_train, bsz, st.scratch, stream)
    evs["t2"].record(stream)
    B.hw_encode(sess.ctx, te_vals_d[:bsz], bsz, bits, stream)
    B.hw_encrypt_sample(sess.ctx, key, bits, None, bsz, 500000 + k, 0, st.rgsw_test, stream)
    evs["t3"].record(stream)
    resp, sums, scr = st.ibufs
    B.hw_infer(sess.ctx, model, st.rgsw_test, bsz, resp, sums, scr, stream)
    evs["t4"].record(stream)
    B.hw_decrypt(sess.ctx, key, B.HW_DEC_LWE, resp, bsz * cfg.n_classes * sz["k0"], st.counts, stream)
    B.hw_pdact(sess.ctx, st.counts, bsz, st.scores, st.labels, stream)
    evs["t5"].record(stream)
    torch.cuda.synchronize()
    keys = ["encrypt_train", "train", "encrypt_test", "infer", "decrypt_pdact"]
    ph = {kn: evs[a].elapsed_time(evs[b]) for a, b, kn in zip(names[:-1], names[1:], keys)}

    healthy("the timed steps")

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
    keyswitch = None
    if not args.no_keyswitch:
        resp = st.ibufs[0]
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        ksk = sess.ksk_gen(key, cfg.key_seed + 1, stream=stream)
        e1.record(stream)
        pscr = sess.words(B.hw_pack_scratch_words(sess.ctx), zero=False)
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
        keyswitch = {"pack_ms_per_step": min(t_pack), "ksk_gen_ms_once": e0.elapsed_time(e1),
                     "ksk_bytes": B.hw_ksk_words(sess.ctx) * 8,
                     "response_bytes_per_sample": {"lwe": sz["resp_words"] * 8, "packed": sz["rlwe_words"] * 8},
                     "share_of_infer": min(t_pack) / ph["infer"]}
        del ksk, pscr

    healthy("the key-switching leg")

    # inference against the model in clear (Section 3.6.2): the owner's
    # decrypted counters as plaintext tables, one blind rotation per (sample,
    # RAM) shared by the l classes; the same encrypted test batch as the
    # phase breakdown's, whose decrypted counters it must reproduce
    clear_model = None
    if not args.no_clear_model:
        alg_c = algorithmic_counts(sess, cfg)
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
                       "ext_products_per_sample": {"clear": alg_c["ext_clear_per_sample"],
                                                   "encrypted": alg_c["ext_infer_per_sample"]},
                       "responses_equal_to_encrypted_path": same}
        del plain, pbufs, W

    healthy("the clear-model leg")

    # e2e through the C ABI with pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        h_tr = torch.from_numpy(tr_vals[:bsz].copy()).pin_memory()
        h_lab = torch.from_numpy(tr_lab[:bsz].astype(np.int32)).pin_memory()
        h_te = torch.from_numpy(te_vals[:bsz].copy()).pin_memory()
        h_out = torch.empty(bsz, dtype=torch.int32).pin_memory()
        host = (h_tr, h_lab, h_te, h_out)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(args.warmup + args.steps + 1 + k, host)
            torch.cuda.current_stream().synchronize()
            _ = int(h_out[0])
        t1 = time.perf_counter()
        e2e_s = t1 - t0
        if pg is not None:
            t = torch.tensor([e2e_s], device=dev)
            pg.all_reduce(t, op=pg.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": total_samples / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h_tr.numel() + h_lab.numel() * 4 + h_te.numel()),
               "d2h_bytes_per_step": int(h_out.numel() * 4)}

    healthy("the end-to-end leg")

    # roofline of the dominant kernel (the VP inference kernel)
    pk, pk_kind = peaks()
    alg = algorithmic_counts(sess, cfg)
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    word_bits = sz["word_bits"]  # the external product's word width in this context
    muls = MULS_PER_MODMUL32 if word_bits == 32 else MULS_PER_MODMUL
    peak_modmul = sm_count * IMAD_PER_CLK_PER_SM * sm_mhz * 1e6 / muls
    infer_modmul = alg["ext_infer_per_sample"] * bsz * alg["per_ext_modmul"]
    # average duration of the inference graph (k_vp_infer + the per-class
    # sums, < 0.5 %) over the timed steps, CUDA events on the launching stream
    vp_ms = statistics.mean(a.elapsed_time(b) for a, b in vp_events)
    achieved = infer_modmul / (vp_ms / 1000.0)
    roofline = {"bound": "alu", "kernel": "k_vp_infer", "achieved": achieved / 1e12,
                "peak": peak_modmul / 1e12, "unit": "T modmul/s", "frac": achieved / peak_modmul,
                "traffic": profiled_traffic(args.config, sess.geometry, bsz),
                "launch_ms": vp_ms,
                "butterfly_ceiling": BUTTERFLY_CEILING32 if word_bits == 32 else BUTTERFLY_CEILING,
                "peak_kind": f"derived: {sm_count} SMs x {IMAD_PER_CLK_PER_SM} int32 multiplies/clk x "
                             f"{sm_mhz:.0f} MHz / {muls} per {word_bits}-bit modular product"}
    train_modmul = alg["ext_train_per_sample"] * bsz * alg["per_ext_modmul"]

    # batched NTT throughput (forward transforms, one read + one write per
    # polynomial): this workload's ring, and cfg1's 30-bit ring, where the
    # 32-bit transform makes the NTT bound by HBM rather than by integer
    # multiplies
    ntt = None
    if not args.no_ntt:
        def ntt_rate(ctx_sess, count):
            nn = ctx_sess.sz["n"]
            polys = ctx_sess.words(count * nn)
            for _ in range(3):
                B.hw_ntt_forward(ctx_sess.ctx, polys, count, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                B.hw_ntt_forward(ctx_sess.ctx, polys, count, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / reps / 1000.0
            gbs = 2.0 * count * nn * 8 / t / 1e9
            del polys
            g = ctx_sess.geometry
            return {"gbs": gbs, "frac_of_hbm": gbs / pk["hbm_gbs"], "polys": count, "n": nn,
                    "prime_bits": ctx_sess.cfg.prime_bits, "ms_per_launch": t * 1000.0,
                    "variant": f"radix {1 << g['ntt_loge']}, {32 * g['ntt_limbs']}-bit words"}
        ntt = {"peak_gbs": pk["hbm_gbs"], "peak_kind": pk_kind,
               args.config: ntt_rate(sess, 65536 if sz["n"] <= 4096 else 32768)}
        if args.config != "cfg1":
            s1 = Session(get_config("cfg1"), local, geometry="auto" if args.geometry == "auto" else None)
            ntt["cfg1"] = ntt_rate(s1, 262144)
            del s1

    healthy("the NTT leg")

    # horizontal packing (Section 6): plain vs packed inference on the
    # Wisconsin-shaped ring (label bits low, z = 0: one VP answers both
    # classes); the digit workloads keep a stored ciphertext per class
    packing = None
    if not args.no_packing:
        pc = cfg if args.config == "cfg1" else get_config("cfg1")
        ps = sess if args.config == "cfg1" else Session(pc, local, geometry="auto" if args.geometry == "auto" else None)
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
        packing = {"workload": "cfg1", "inferences_per_s_plain": rates["plain"],
                   "inferences_per_s_packed": rates["packed"],
                   "vp_per_sample": {"plain": pc.n_classes * psz["k0"], "packed": groups * psz["k0"]},
                   "applies_to_bench_workload": sz["z"] <= sz["L"] and min(cfg.n_classes, 1 << sz["z"]) < cfg.n_classes}
        del pbufs, prg
        if ps is not sess:
            del ps

    healthy("the packing leg")

    # the same workload one request at a time: each request one train and one
    # test sample, encoded, encrypted, trained, inferred, decrypted, waited for
    single = None
    if not args.no_serve:
        n1 = 6
        t0 = time.perf_counter()
        for k in range(n1):
            B.hw_encode(sess.ctx, tr_vals_d[k:k + 1], 1, bits, stream)
            B.hw_encrypt_sample(sess.ctx, key, bits, tr_lab_d[k:k + 1], 1, 9000 + k, 0, st.rgsw_train, stream)
            B.hw_train_accumulate(sess.ctx, model, st.rgsw_train, 1, st.scratch, stream)
            B.hw_encode(sess.ctx, te_vals_d[k:k + 1], 1, bits, stream)
            B.hw_encrypt_sample(sess.ctx, key, bits, None, 1, 19000 + k, 0, st.rgsw_test, stream)
            resp, sums, scr = st.ibufs
            B.hw_infer(sess.ctx, model, st.rgsw_test, 1, resp, sums, scr, stream)
            B.hw_decrypt(sess.ctx, key, B.HW_DEC_LWE, resp, cfg.n_classes * sz["k0"], st.counts, stream)
            B.hw_pdact(sess.ctx, st.counts, 1, st.scores, st.labels, stream)
            _ = int(st.labels[0].item())
        single = {"samples_per_s": 2 * n1 / (time.perf_counter() - t0), "requests": n1,
                  "request": "1 train + 1 test sample, synchronous"}

    serving = None
    if not args.no_serve:
        healthy("the one-at-a-time requests")
        del st, tr_vals_d, tr_lab_d, te_vals_d, bits
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        serving = serve_leg(args, local)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, 16)
        rate, wall, rams = oracle_sample(args.config, sz["k0"], cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"1 train + 1 test sample restricted to {rams} of {sz['k0']} RAMs "
                         f"(one per worker), {wall:.1f} s wall, scaled by {sz['k0']}/{rams}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": workload_name(cfg), "batch_train": bsz, "batch_test": bsz,
                       "server_step": "CUDA graph (IVP + accumulate, VP + sums, decrypt, PD-act)",
                       "l2": "inputs larger than L2 (encrypted batch ~%.0f GB)" %
                             (bsz * sz["sample_words"] * 8 / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "train_samples_per_s": bsz / (ph["train"] / 1000.0),
            "inferences_per_s": bsz / (ph["infer"] / 1000.0),
            "train_modmul_per_s": train_modmul / (ph["train"] / 1000.0),
            "phases_ms": ph,
            "balancing": balancing,
            "horizontal_packing": packing,
            "packing_keyswitch": keyswitch,
            "clear_model": clear_model,
            "roofline": roofline,
            "ntt": ntt,
            "geometry": sess.geometry,
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


# per-request sample caps of the serving mix: what the footprint rule leaves
# for one request (786 MiB, 3.9 GiB, 15.5 GiB per encrypted cfg2/3/4 sample)
SERVE_MAX = {"cfg1": 256, "cfg2": 16, "cfg3": 2, "cfg4": 1}


def serve_leg(args, local):
    """Poisson stream (200 requests/s, seeded) of train and infer requests over
    the four workloads, served with continuous batching and, for comparison,
    one request at a time; latency is arrival to completion."""
    import copy

    import torch

    from paper_2403_20190_gb300.serve import ResidentModel, Server, latency_stats, poisson_stream
    from synthdata import get_config
    cfgs = {nm: get_config(nm) for nm in ("cfg1", "cfg2", "cfg3", "cfg4")}
    geo = "auto" if args.geometry == "auto" else None
    models = {nm: ResidentModel(c, local, key_seed=c.key_seed, geometry=geo) for nm, c in cfgs.items()}
    reqs = poisson_stream(cfgs, n_requests=args.serve_requests, rate=200.0, seed=2024,
                          max_samples=SERVE_MAX)
    from paper_2403_20190_gb300.arena import DeviceArena
    budget = 120 << 30
    arena = DeviceArena(budget, torch.device("cuda", local))  # shared by both modes
    warm = copy.deepcopy(reqs[:4])
    Server(models, arena=arena).run(warm, realtime=False)
    base = copy.deepcopy(reqs)
    srv = Server(models, n_streams=2, arena=arena, packed_infer=True)
    costs = srv.calibrate()  # startup, outside the timed runs
    batched = srv.run(copy.deepcopy(reqs), realtime=True)
    srv_plain = Server(models, n_streams=2, arena=arena, packed_infer=False)
    srv_plain.calibrate()
    batched_plain = srv_plain.run(copy.deepcopy(reqs), realtime=True)
    alone = Server(models, arena=arena, packed_infer=False).run_one_at_a_time(base)
    out = {"requests": len(reqs), "rate_per_s": 200.0, "hbm_budget_gb": budget / 2**30,
           "batched": latency_stats(batched), "batched_without_packing": latency_stats(batched_plain),
           "one_at_a_time": latency_stats(alone),
           "mix": {nm: sum(1 for r in reqs if r.cfg_name == nm) for nm in cfgs},
           "policy": "2 streams, shortest expected batch first with aging 1.0, device arena, inference "
                     "with horizontal packing where the tree layout allows (cfg1, cfg3); the one-at-a-time "
                     "baseline runs the plain path",
           "calibrated_ms_per_sample": {f"{k[0]}/{k[1]}": round(v * 1e3, 3) for k, v in costs.items()},
           "max_samples_per_request": SERVE_MAX}
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
