"""Failure handling on the host side: no test here faults, traps or hangs a GPU.

Allocation failures come from a fake allocator installed through the library's allocator hook;
invalid inputs are rejected before any device work. After each failure the handle (or a new
one) keeps working.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _install(allocs_before_failure):
    """A PyTorch-backed device allocator that returns NULL after a number of successes."""
    import torch

    from paper_1910_13874_gb300 import gedwalk

    lib = gedwalk.load()
    state = {"left": allocs_before_failure, "live": {}}

    def alloc(nbytes, stream, ctx):
        if state["left"] == 0:
            return None
        state["left"] -= 1
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, nbytes, stream, ctx):
        state["live"].pop(ptr, None)

    hooks = (gedwalk._ALLOC_FN(alloc), gedwalk._FREE_FN(free))
    gedwalk._hook_refs.append(hooks)  # blocks are freed through the hooks that made them
    assert lib.gedwalk_set_allocator(hooks[0], hooks[1], None) == gedwalk.OK
    return hooks, state


def _restore():
    from paper_1910_13874_gb300 import gedwalk

    lib = gedwalk.load()
    assert lib.gedwalk_set_allocator(gedwalk._ALLOC_FN(), gedwalk._FREE_FN(), None) == gedwalk.OK
    gedwalk._torch_hooks = None
    gedwalk.use_torch_allocator()  # back to the binding's default


def test_upload_reports_oom_and_recovers(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = gg.erdos_renyi(2000, 8, 3)
    hooks, _ = _install(0)
    try:
        with pytest.raises(gedwalk.GedWalkError) as e:
            gedwalk.Graph.from_host(g)
        assert e.value.status == gedwalk.ERR_OOM
    finally:
        _restore()
    G = gedwalk.Graph.from_host(g)  # the binding's default allocator works again
    assert G.score([1, 2, 3], precision="fp64", L=4)[0] > 0


def test_oom_midway_leaves_the_graph_usable(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = gg.erdos_renyi(2000, 8, 4)
    hooks, state = _install(10 ** 6)
    try:
        G = gedwalk.Graph.from_host(g)
        state["left"] = 0  # every later allocation fails
        with pytest.raises(gedwalk.GedWalkError) as e:
            G.maximize(5, precision="fp32", epsilon=1e-4)
        assert e.value.status == gedwalk.ERR_OOM
        state["left"] = 10 ** 6
        grp, gains, _, L = G.maximize(5, precision="fp32", epsilon=1e-4)
        ogrp, _, _ = oracle.greedy(g, 5, oracle.default_alpha(g), L, "lazy")
        assert list(grp) == list(ogrp)
        G.free()
    finally:
        _restore()


def test_torch_allocator_hook(cuda_device):
    import gc

    import torch

    from paper_1910_13874_gb300 import gedwalk

    gedwalk.use_torch_allocator()  # the binding's default; a no-op when installed
    g = gg.barabasi_albert(5000, 3, 9)
    gc.collect()
    gc.disable()  # nothing else may release PyTorch memory while the upload is measured
    try:
        before = torch.cuda.memory_allocated()
        G = gedwalk.Graph.from_host(g)
        grown = torch.cuda.memory_allocated() - before
    finally:
        gc.enable()
    assert grown >= 4 * g.nnz  # at least the relabelled CSR lives in PyTorch's allocations
    try:
        s, L, _ = G.score([0, 1, 2], precision="fp32", epsilon=1e-4)
        assert abs(s - oracle.score(g, [0, 1, 2], oracle.default_alpha(g), L)) <= 1e-5 * s
        G.free()
    finally:
        _restore()


def test_invalid_arguments_are_rejected(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    g = gg.erdos_renyi(500, 6, 5)
    G = gedwalk.Graph.from_host(g)
    cases = [
        lambda: G.maximize(-1),
        lambda: G.maximize(g.n + 1),
        lambda: G.maximize(3, init=[g.n]),
        lambda: G.score([0], epsilon=-1.0),
        lambda: G.score([0], L=-3),
        lambda: G.score_batch([1, 2], [0, 1]),  # offsets must start at 0
        lambda: G.score_batch([0, 3, 2], [0, 1, 2]),  # offsets decrease
        lambda: G.gains([0], alpha=-0.5),
    ]
    for f in cases:
        with pytest.raises(gedwalk.GedWalkError) as e:
            f()
        assert e.value.status == gedwalk.ERR_INVALID
    # the handle still works
    assert G.score([0, 1], precision="fp64", L=3)[0] > 0
    assert np.isfinite(G.maximize(2)[2])
