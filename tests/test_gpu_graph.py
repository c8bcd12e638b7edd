"""The CUDA-graph-captured server step (IVP + accumulate, VP + class sums,
decryption, PD-act) gives bit-identical results to the same calls issued
eagerly, replay after replay (the model keeps accumulating)."""
import numpy as np
import pytest
import torch

from synthdata import get_config, make_dataset

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,over", [
    ("cfg1", {}),
    ("cfg1", dict(log_n=6, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3,
                  n_values=4, therm_bits=2, addr_bits=7, tuple_bits=7, data_kind="uniform")),
])
def test_graph_replay_equals_eager(name, over):
    from paper_2403_20190_gb300 import build
    from paper_2403_20190_gb300.session import ServerStep, Session
    build.build()
    cfg = get_config(name, **over)
    sess = Session(cfg, 0)
    dev = sess.device
    key = sess.keygen(3)
    n_tr, n_te = 6, 4
    vals, labels = make_dataset(cfg, "train", n=3 * n_tr)
    tvals, _ = make_dataset(cfg, "test", n=n_te)
    steps = []
    for mode in ("eager", "graph"):
        model = sess.new_model()
        st = ServerStep(sess, key, model, n_tr, n_te)
        tb = sess.encode(torch.from_numpy(tvals).to(dev))
        sess.encrypt(key, tb, None, seed=77, out=st.rgsw_test)
        outs = []
        for k in range(3):
            b = sess.encode(torch.from_numpy(vals[k * n_tr:(k + 1) * n_tr]).to(dev))
            lab = torch.from_numpy(labels[k * n_tr:(k + 1) * n_tr].astype(np.int32)).to(dev)
            sess.encrypt(key, b, lab, seed=100 + k, out=st.rgsw_train)
            if mode == "eager":
                st.run()
            else:
                if st.graph is None:
                    st.capture()
                st.replay()
            torch.cuda.synchronize()
            outs.append((model.clone(), st.ibufs[0].clone(), st.labels.clone()))
        steps.append(outs)
    for (m0, r0, l0), (m1, r1, l1) in zip(*steps):
        assert torch.equal(m0, m1) and torch.equal(r0, r1) and torch.equal(l0, l1)
