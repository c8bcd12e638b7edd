"""hw_import_rgsw is the inverse of hw_export_rgsw, bit for bit, and makes
ciphertexts portable: RGSW encrypted by the CPU oracle, imported, trains a
model on the GPU equal to the oracle's own training; RGSW exported from a
context of one kernel geometry and imported into another trains the same
model.  Integer results: tolerance 0."""
import numpy as np
import pytest
import torch

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset
from test_gpu_parity import tiny_cfg, u64

pytestmark = pytest.mark.gpu


def _session(cfg, geometry=None):
    from paper_2403_20190_gb300.session import Session
    return Session(cfg, 0, geometry=geometry)


@pytest.mark.parametrize("name", ["zL", "r2_beta1024"])
def test_export_import_roundtrip(name):
    cfg = tiny_cfg(name)
    s = _session(cfg)
    dev = s.device
    vals, labels = make_dataset(cfg, "train", n=3)
    key = s.keygen(5)
    bits = s.encode(torch.from_numpy(vals).to(dev))
    rg = s.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(dev), seed=9)
    count = 3 * s.sz["n_slots"]
    canon = s.export_rgsw(rg, count)
    back = s.import_rgsw(canon, count)
    torch.cuda.synchronize()
    assert torch.equal(back, rg)
    # words above q are reduced on entry; in place is allowed
    q = np.array(s.sz["q"], dtype=np.uint64)
    n, r = s.sz["n"], s.sz["r"]
    c = u64(canon).reshape(-1, r, n).copy()
    c += q[None, :, None]  # same residues, not reduced
    dev_c = torch.from_numpy(c.reshape(-1).view(np.int64)).to(dev)
    from paper_2403_20190_gb300 import binding as B
    B.hw_import_rgsw(s.ctx, dev_c, count, dev_c)
    torch.cuda.synchronize()
    assert torch.equal(dev_c, rg)


def test_oracle_ciphertexts_train_on_the_gpu():
    cfg = tiny_cfg("zgtL")
    o = Oracle(cfg)
    P = o.P
    n = 4
    vals, labels = make_dataset(cfg, "train", n=n)
    bits = wisard.encode(P, vals)
    sk = o.keygen(7)
    canon = []
    for i in range(n):
        for b in range(P.n_slots):
            val = (int(labels[i]) >> b) & 1 if b < P.L else int(bits[i, b - P.L])
            canon.append(o.export_rgsw(o.encrypt_bit(sk, 13, i * P.n_slots + b, val)))
    canon = np.ascontiguousarray(np.stack(canon)).reshape(-1)
    s = _session(cfg)
    rg = s.import_rgsw(torch.from_numpy(canon.view(np.int64)).to(s.device), n * P.n_slots)
    model = s.train(s.new_model(), rg, n)
    torch.cuda.synchronize()
    H = o.train(o.new_model(), sk, 13, bits, labels)
    assert np.array_equal(u64(model).reshape(H.shape), H)


def test_ciphertexts_move_between_geometries():
    from paper_2403_20190_gb300 import binding as B
    cfg = get_config("cfg1")
    geos = B.hw_list_geometries(cfg)
    a = _session(cfg, geos[0])
    b = _session(cfg, next(g for g in geos if g["ext_loge"] != geos[0]["ext_loge"]))
    assert a.geometry["ext_loge"] != b.geometry["ext_loge"]
    vals, labels = make_dataset(cfg, "train", n=4)
    key = a.keygen(3)
    bits = a.encode(torch.from_numpy(vals).to(a.device))
    rg = a.encrypt(key, bits, torch.from_numpy(labels.astype(np.int32)).to(a.device), seed=21)
    count = 4 * a.sz["n_slots"]
    moved = b.import_rgsw(a.export_rgsw(rg, count), count)
    ma = a.train(a.new_model(), rg, 4)
    mb = b.train(b.new_model(), moved, 4)
    torch.cuda.synchronize()
    assert torch.equal(ma, mb)
