"""The caller's allocator (pq_set_allocator): with PyTorch's caching allocator
owning the library's device memory, a propagation gives the same numbers as
with cudaMalloc, every buffer is returned when the state is freed, and the
allocator cannot change while a state exists.  Collected late so that the
states of the other test files are gone."""
import gc

import numpy as np
import pytest

import workloads as W
from gpu_helpers import lib

pytestmark = pytest.mark.gpu


def _run(pq, cfg, n):
    b = pq.build_model(cfg)
    s = pq.State(b, cfg["q0"], cfg["p0"], cfg["width"], cfg["theta"], precision=pq.FP64)
    s.propagate(cfg["K"], cfg["dt"], cfg["theta"], n)
    return s, s.observables()


def test_torch_caching_allocator_owns_library_memory():
    import torch
    pq = lib()
    cfg = W.MORSE2D
    gc.collect()
    s, ref = _run(pq, cfg, 20)
    s.free()
    counts = {"alloc": 0, "free": 0}
    live = {}

    def alloc(n, stream, ctx):
        p = torch.cuda.caching_allocator_alloc(int(n), stream=int(stream or 0))
        counts["alloc"] += 1
        live[p] = n
        return p

    def free(p, stream, ctx):
        counts["free"] += 1
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    base = torch.cuda.memory_allocated()
    pq.set_allocator(alloc, free)
    try:
        s, o = _run(pq, cfg, 20)
        assert counts["alloc"] > 10
        assert torch.cuda.memory_allocated() > base
        with pytest.raises(pq.PQError) as e:   # a state exists
            pq.set_allocator()
        assert e.value.status == pq.EINVAL
        s.free()
        torch.cuda.synchronize()
        assert not live and counts["free"] == counts["alloc"]
        assert torch.cuda.memory_allocated() == base
        np.testing.assert_array_equal(o["n_active"], ref["n_active"])
        np.testing.assert_array_equal(o["C"], ref["C"])
    finally:
        gc.collect()
        pq.set_allocator()
