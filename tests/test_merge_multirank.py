"""Data-parallel training across ranks: each rank trains on its shard of the
samples, the partial models are summed mod q in one all-reduce, and the
merged model is bit-identical to the model trained centrally (Section 3.6.2).
Runs two gloo ranks on the CPU; the shard models come from the oracle."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import Oracle, wisard
from synthdata import get_config, make_dataset

CFG = dict(log_n=4, n_primes=3, prime_bits=55, log_beta=0, log_p=22, n_classes=3, n_values=4,
           therm_bits=2, addr_bits=4, tuple_bits=4, data_kind="uniform", act="log", act_arg=0)
N_SAMPLES = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_models():
    cfg = get_config("cfg1", **CFG)
    o = Oracle(cfg)
    vals, labels = make_dataset(cfg, "train", n=N_SAMPLES)
    bits = wisard.encode(o.P, vals)
    s = o.keygen(4)
    central = o.train(o.new_model(), s, 17, bits, labels)
    half = N_SAMPLES // 2
    shards = [o.train(o.new_model(), s, 17, bits[:half], labels[:half]),
              o.train(o.new_model(), s, 17, bits[half:], labels[half:], sample_offset=half)]
    return o.P, central, shards


def _rank(rank, world, port, shards, q, n, out):
    import torch.distributed as dist
    from paper_2403_20190_gb300.merge import all_reduce_model
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = torch.from_numpy(shards[rank].reshape(-1).view(np.int64).copy())
        all_reduce_model(m, q, n)
        out[rank] = m.numpy().view(np.uint64).copy()
    finally:
        dist.destroy_process_group()


def test_two_rank_merge_equals_central_training():
    P, central, shards = _shard_models()
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, port, shards, P.q, P.n, out), nprocs=2, join=True,
                           start_method="spawn")
        for rank in range(2):
            assert np.array_equal(out[rank].reshape(central.shape), central)


def test_add_models_is_addition_mod_q():
    from paper_2403_20190_gb300.merge import add_models
    P, central, shards = _shard_models()
    a = torch.from_numpy(shards[0].reshape(-1).view(np.int64).copy())
    b = torch.from_numpy(shards[1].reshape(-1).view(np.int64).copy())
    s = add_models(a, b, P.q, P.n).numpy().view(np.uint64)
    assert np.array_equal(s.reshape(central.shape), central)
    with pytest.raises(Exception):
        add_models(a, b[:-1], P.q, P.n)
