"""Workload-level convenience over the C ABI: device buffers come from
torch's caching allocator; every step is one libhwisard call.  ServerStep
captures the server side of a step into a CUDA graph."""
import torch

from . import binding as B


class Session:
    def __init__(self, cfg, device: int = 0, geometry=None):
        """geometry: None (library defaults), "auto" (autotuned, cached per
        GPU and parameter set) or a dict of hwisard geometry fields."""
        self.cfg = cfg
        self.device = torch.device("cuda", device)
        if geometry == "auto":
            from .tuning import tuned_geometry
            geometry = tuned_geometry(cfg, device)[0]
            try:
                self.ctx = B.hw_create_tuned(cfg, geometry, device)
            except B.HwError:  # a cached choice this library cannot take: measure again
                geometry = tuned_geometry(cfg, device, refresh=True)[0]
                self.ctx = B.hw_create_tuned(cfg, geometry, device)
        elif geometry:
            self.ctx = B.hw_create_tuned(cfg, geometry, device)
        else:
            self.ctx = B.hw_create(cfg, device)
        self.geometry = B.hw_get_geometry(self.ctx)
        self.sz = B.hw_get_sizes(self.ctx)

    # --------------------------------------------------------------- buffers
    def words(self, n, zero=True):
        f = torch.zeros if zero else torch.empty
        return f(int(n), dtype=torch.int64, device=self.device)

    def keygen(self, seed, stream=None):
        key = self.words(self.sz["key_words"])
        B.hw_keygen(self.ctx, seed, key, stream)
        return key

    def new_model(self, stream=None):
        """Definition 2's model H <- {0} (hw_model_zero)."""
        model = self.words(B.hw_model_words(self.ctx), zero=False)
        B.hw_model_zero(self.ctx, model, stream)
        return model

    # ---------------------------------------------------------------- client
    def encode(self, values, stream=None):
        """values: uint8 CUDA tensor (n, n_values) -> data bits (n, n_data)."""
        n = values.shape[0]
        bits = torch.empty((n, self.sz["n_data"]), dtype=torch.uint8, device=self.device)
        B.hw_encode(self.ctx, values.contiguous(), n, bits, stream)
        return bits

    def encrypt(self, key, bits, labels, seed, first_sample=0, out=None, stream=None):
        n = bits.shape[0]
        if out is None:
            out = self.words(n * self.sz["sample_words"], zero=False)
        lab = None if labels is None else labels.to(torch.int32).contiguous()
        B.hw_encrypt_sample(self.ctx, key, bits.contiguous(), lab, n, seed, first_sample, out, stream)
        return out

    # ---------------------------------------------------------------- server
    def train_scratch(self, n):
        return self.words(B.hw_train_scratch_words(self.ctx, n), zero=False)

    def train(self, model, rgsw, n, scratch=None, stream=None):
        if scratch is None:
            scratch = self.train_scratch(n)
        B.hw_train_accumulate(self.ctx, model, rgsw, n, scratch, stream)
        return model

    def infer_buffers(self, n):
        resp = self.words(n * self.sz["resp_words"], zero=False)
        sums = self.words(n * self.sz["sums_words"], zero=False)
        scratch = self.words(B.hw_infer_scratch_words(self.ctx, n), zero=False)
        return resp, sums, scratch

    def infer(self, model, rgsw, n, bufs=None, stream=None, packed=False):
        resp, sums, scratch = bufs if bufs is not None else self.infer_buffers(n)
        fn = B.hw_infer_packed if packed else B.hw_infer
        fn(self.ctx, model, rgsw, n, resp, sums, scratch, stream)
        return resp, sums

    # -------------------------------------- unencrypted-model inference
    def plain_model(self, counts, stream=None):
        """Plaintext tables of a model in clear from its counters W[c][j][addr]
        (an int64 device tensor (l, k0, 2^a))."""
        counts = counts.to(device=self.device, dtype=torch.int64).contiguous()
        assert counts.numel() == self.cfg.n_classes * self.sz["k0"] * (1 << self.sz["a"])
        plain = self.words(B.hw_plain_model_words(self.ctx), zero=False)
        B.hw_plain_model_load(self.ctx, counts, plain, stream)
        return plain

    def infer_plain(self, plain, rgsw, n, bufs=None, stream=None):
        resp, sums, scratch = bufs if bufs is not None else self.infer_buffers(n)
        B.hw_infer_plain(self.ctx, plain, rgsw, n, resp, sums, scratch, stream)
        return resp, sums

    # ----------------------------------------------------- checkpoint
    def save_model(self, path, model, samples):
        """Checkpoint of the model after `samples` training samples
        (hw_model_export)."""
        from .checkpoint import save
        save(path, self, model, samples)

    def load_model(self, path):
        """(model on this device, samples trained) from a checkpoint of the
        same parameter set (hw_model_import); training continues from it
        bit-exactly."""
        from .checkpoint import load
        return load(path, self)

    # ---------------------------------------------------------------- client
    def decrypt_rlwe(self, key, obj, count, stream=None):
        out = torch.empty(int(count) * self.sz["n"], dtype=torch.int64, device=self.device)
        B.hw_decrypt(self.ctx, key, B.HW_DEC_RLWE, obj, count, out, stream)
        return out

    def decrypt_lwe(self, key, obj, count, stream=None):
        out = torch.empty(int(count), dtype=torch.int64, device=self.device)
        B.hw_decrypt(self.ctx, key, B.HW_DEC_LWE, obj, count, out, stream)
        return out

    # --------------------------------------------- PackingKeySwitching
    def ksk_gen(self, key, seed, stream=None):
        ksk = self.words(B.hw_ksk_words(self.ctx), zero=False)
        B.hw_ksk_gen(self.ctx, key, seed, ksk, stream)
        return ksk

    def pack_responses(self, ksk, resp, n, scratch=None, stream=None):
        """One RLWE per test sample: coefficient c * k0 + j is u[c][j]."""
        if scratch is None:
            scratch = self.words(B.hw_pack_scratch_words(self.ctx, n), zero=False)
        packed = self.words(int(n) * self.sz["rlwe_words"], zero=False)
        B.hw_pack_responses(self.ctx, ksk, resp, n, packed, scratch, stream)
        return packed

    def packed_counts(self, key, packed, n, stream=None):
        """Decrypted responses (n, l, k0) from packed RLWEs."""
        l, k0 = self.cfg.n_classes, self.sz["k0"]
        vals = self.decrypt_rlwe(key, packed, n, stream).view(int(n), self.sz["n"])
        return vals[:, : l * k0].reshape(int(n), l, k0)

    # ------------------------------------------------ dataset balancing
    def new_counts(self):
        """Class-count ciphertext (one RLWE), zero."""
        return self.words(self.sz["rlwe_words"])

    def count_classes(self, counts, rgsw, n, scratch=None, stream=None):
        if scratch is None:
            scratch = self.words(B.hw_count_scratch_words(self.ctx, n), zero=False)
        B.hw_count_classes(self.ctx, counts, rgsw, n, scratch, stream)
        return counts

    def class_counts(self, key, counts, stream=None):
        """Decrypted class counts (l,) as an int64 device tensor."""
        return self.decrypt_rlwe(key, counts, 1, stream)[: self.cfg.n_classes].contiguous()

    def pdact_balanced(self, counts, class_counts, n, stream=None):
        l = self.cfg.n_classes
        scores = torch.empty(n * l, dtype=torch.int64, device=self.device)
        labels = torch.empty(n, dtype=torch.int32, device=self.device)
        B.hw_pdact_balanced(self.ctx, counts, class_counts, n, scores, labels, stream)
        return scores.view(n, l), labels

    def pdact(self, counts, n, stream=None):
        l = self.cfg.n_classes
        scores = torch.empty(n * l, dtype=torch.int64, device=self.device)
        labels = torch.empty(n, dtype=torch.int32, device=self.device)
        B.hw_pdact(self.ctx, counts, n, scores, labels, stream)
        return scores.view(n, l), labels

    def decrypt_model_counts(self, key, model, stream=None):
        """Decrypted counters W[c][j][addr] (l, k0, 2^a) from the model
        (hw_decrypt, HW_DEC_MODEL)."""
        sz = self.sz
        out = torch.empty(self.cfg.n_classes * sz["k0"] << sz["a"], dtype=torch.int64, device=self.device)
        B.hw_decrypt(self.ctx, key, B.HW_DEC_MODEL, model, 1, out, stream)
        return out.view(self.cfg.n_classes, sz["k0"], 1 << sz["a"])

    def responses_counts(self, key, resp, n, stream=None):
        """Decrypted responses u[i][c][j] (n, l, k0)."""
        l, k0 = self.cfg.n_classes, self.sz["k0"]
        return self.decrypt_lwe(key, resp, n * l * k0, stream).view(n, l, k0)

    def export_rgsw(self, rgsw, count, stream=None):
        out = self.words(int(count) * self.sz["rgsw_words"], zero=False)
        B.hw_export_rgsw(self.ctx, rgsw, count, out, stream)
        return out

    def import_rgsw(self, canonical, count, stream=None):
        out = self.words(int(count) * self.sz["rgsw_words"], zero=False)
        B.hw_import_rgsw(self.ctx, canonical, count, out, stream)
        return out


class ServerStep:
    """The server side of one step on fixed batch sizes: train on an
    encrypted batch (IVP + accumulate into the resident model) and answer an
    encrypted test batch (VP + class sums), then decrypt the responses and
    classify them with PD-act.  The encrypted inputs live in rgsw_train /
    rgsw_test; capture() records the step once into CUDA graphs and replay()
    re-issues them (the model keeps accumulating across replays)."""

    def __init__(self, sess: Session, key, model, n_train: int, n_test: int):
        self.sess, self.key, self.model = sess, key, model
        self.n_train, self.n_test = n_train, n_test
        sz = sess.sz
        self.rgsw_train = sess.words(n_train * sz["sample_words"], zero=False)
        self.rgsw_test = sess.words(n_test * sz["sample_words"], zero=False)
        self.scratch = sess.train_scratch(max(n_train, 1))
        self.ibufs = sess.infer_buffers(max(n_test, 1))
        l, k0 = sess.cfg.n_classes, sz["k0"]
        self.counts = torch.empty(max(n_test, 1) * l * k0, dtype=torch.int64, device=sess.device)
        self.scores = torch.empty(max(n_test, 1) * l, dtype=torch.int64, device=sess.device)
        self.labels = torch.empty(max(n_test, 1), dtype=torch.int32, device=sess.device)
        self.graph = None
        self.launches_per_step = None

    def run_train(self, stream=None):
        B.hw_train_accumulate(self.sess.ctx, self.model, self.rgsw_train, self.n_train, self.scratch, stream)

    def run_infer(self, stream=None):
        resp, sums, scr = self.ibufs
        B.hw_infer(self.sess.ctx, self.model, self.rgsw_test, self.n_test, resp, sums, scr, stream)

    def run_post(self, stream=None):
        s, ctx = self.sess, self.sess.ctx
        resp = self.ibufs[0]
        l, k0 = s.cfg.n_classes, s.sz["k0"]
        B.hw_decrypt(ctx, self.key, B.HW_DEC_LWE, resp, self.n_test * l * k0, self.counts, stream)
        B.hw_pdact(ctx, self.counts, self.n_test, self.scores, self.labels, stream)

    def run(self, stream=None):
        self.run_train(stream)
        self.run_infer(stream)
        self.run_post(stream)

    def capture(self):
        """Capture the step as three CUDA graphs (train, infer, decrypt +
        PD-act) replayed back to back, so a caller can time the parts."""
        before = B.hw_launch_count(self.sess.ctx)
        graphs = []
        for part in (self.run_train, self.run_infer, self.run_post):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="relaxed"):
                part()
            graphs.append(g)
        self.launches_per_step = B.hw_launch_count(self.sess.ctx) - before
        self.graphs = graphs
        self.graph = graphs[0]
        return graphs

    def replay(self, between=None):
        """Replay the step; between(i) runs after part i (0: train, 1: infer)."""
        for i, g in enumerate(self.graphs):
            g.replay()
            if between is not None:
                between(i)
