"""Failures made on the host (nothing faults the GPU): a device allocation
of context creation that fails -- injected with HW_FAULT_ALLOC=k, the k-th
allocation of each hw_create -- returns an error, frees what was already
allocated, and leaves the device usable for the next context."""
import gc

import pytest
import torch

from synthdata import get_config

pytestmark = pytest.mark.gpu


def test_allocation_failures_leave_nothing_behind(monkeypatch):
    from paper_2403_20190_gb300 import binding as B
    cfg = get_config("cfg2")
    B.hw_create(cfg, 0)  # module loading and tables once, before measuring
    gc.collect()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    for k in (1, 2) * 8:
        monkeypatch.setenv("HW_FAULT_ALLOC", str(k))
        with pytest.raises(B.HwError, match="allocation failed"):
            B.hw_create(cfg, 0)
    monkeypatch.delenv("HW_FAULT_ALLOC")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert free0 - free1 < (8 << 20), "a failed creation leaked device memory"
    ctx = B.hw_create(cfg, 0)  # the device still serves a new context
    assert B.hw_get_sizes(ctx)["n"] == 4096


def test_context_self_check_passes_after_work():
    """hw_check_context: the tables a context uploaded are unchanged after a
    full encrypt / train / infer pipeline on it and on another context."""
    from paper_2403_20190_gb300 import binding as B
    from test_gpu_parity import run_pipeline, tiny_cfg
    R = run_pipeline(get_config("cfg1"), 3, 2)
    B.hw_check_context(R["sess"].ctx)
    other = run_pipeline(tiny_cfg("zgtL"), 3, 2)
    B.hw_check_context(other["sess"].ctx)
    B.hw_check_context(R["sess"].ctx)
