"""Merging partial models: the federated / data-parallel step of the method.

An Integer WiSARD trained on disjoint shards of the samples is merged by
adding the models (Section 3.6.2): every RAM counter is a sum over samples,
so the sum of shard models equals the model trained on all samples.  Under
encryption the addition is ciphertext addition, residue by residue mod q_i,
and the merged model is bit-identical to central training because addition
mod q is associative and commutative.

The model layout is [RAM][ciphertext][component][prime][N] residues; the
prime of a word is (word // N) mod r within each RLWE block.
"""
import torch


def prime_of_words(n_words: int, n: int, r: int, device=None) -> torch.Tensor:
    """Index of the RNS prime of every word of a model / RLWE array."""
    idx = torch.arange(n_words, device=device, dtype=torch.int64)
    return (idx // n) % r


def add_models(a: torch.Tensor, b: torch.Tensor, q, n: int) -> torch.Tensor:
    """(a + b) mod q_i, element-wise, for int64 tensors holding residues
    below 2^62 (so the sum cannot overflow)."""
    qs = torch.tensor([int(v) for v in q], dtype=torch.int64, device=a.device)
    qw = qs[prime_of_words(a.numel(), n, len(q), a.device)].view_as(a)
    s = a + b
    return torch.where(s >= qw, s - qw, s)


def all_reduce_model(model: torch.Tensor, q, n: int, group=None) -> torch.Tensor:
    """Sum the ranks' partial models mod q_i in place (one all-reduce).

    Residues are below 2^55 and a group holds fewer than 2^7 ranks, so the
    plain int64 sum is exact; one reduction mod q_i follows."""
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    if ws >= 128:
        raise ValueError("more than 127 ranks could overflow the int64 sum")
    dist.all_reduce(model, op=dist.ReduceOp.SUM, group=group)
    qs = torch.tensor([int(v) for v in q], dtype=torch.int64, device=model.device)
    qw = qs[prime_of_words(model.numel(), n, len(q), model.device)].view_as(model)
    model.remainder_(qw)
    return model
