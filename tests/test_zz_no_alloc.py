"""The allocation-free two-state step, called through the C ABI on caller-owned device memory.

Callers that cannot allocate device memory (a framework that has pooled the whole GPU, a
service that forbids allocation while serving) use gedwalk_score_step_noalloc with buffers
they already own. This test owns its buffers through PyTorch, runs the step repeatedly and
compares every partial sum with the regular scoring entry point (gedwalk_score, FP32) and the
whole score with the CPU oracle's two-state recurrence, within the FP32 tolerance of the other
parity tests (1e-5 relative). It runs two scorings in a row so
that the scratch kept from the previous call cannot leak into the next one, and it must pass
alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _mask(n, S):
    words = np.zeros((n + 31) // 32, dtype=np.uint32)
    for v in S:
        words[v >> 5] |= np.uint32(1) << np.uint32(v & 31)
    return words


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_noalloc_step_matches_score_two_calls_in_a_row(cuda_device):
    import torch

    from paper_1910_13874_gb300 import gedwalk

    g = gg.rmat(13, 16, seed=21)  # rows split over many warps, hubs, isolated vertices
    G = gedwalk.Graph.from_host(g)
    alpha = G.alpha_default
    n = g.n
    rp = torch.from_numpy(g.row_ptr).to(cuda_device)
    ci = torch.from_numpy(g.col_idx).to(cuda_device)
    out = torch.zeros(16, dtype=torch.float64, device=cuda_device)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(5)
    for trial in range(2):  # two scorings in a row share the library's scratch
        S = rng.choice(n, size=40, replace=False)
        mask = torch.from_numpy(_mask(n, S)).to(cuda_device)
        x = torch.zeros((n, 2), dtype=torch.float32, device=cuda_device)
        x[:, 1] = 1.0
        x[torch.from_numpy(S).long().to(cuda_device), 0] = 1.0
        x[torch.from_numpy(S).long().to(cuda_device), 1] = 0.0
        y = torch.empty_like(x)
        total = 0.0
        L = 6
        for step in range(1, L + 1):
            first_call = trial == 0 and step == 1
            free_before = torch.cuda.mem_get_info()[0]
            gedwalk.score_step_noalloc(rp.data_ptr(), ci.data_ptr(), n, mask.data_ptr(), x.data_ptr(),
                                       y.data_ptr(), alpha, out.data_ptr() + 8 * step, stream)
            torch.cuda.synchronize()
            if not first_call:  # once the first call has set up the scratch address, nothing is allocated
                assert torch.cuda.mem_get_info()[0] == free_before
            total += float(out[step].item())
            if step <= 2:  # every one of the first two calls checked on its own
                want, _, _ = G.score(S, precision="fp32", L=step)
                assert _rel(total, want) < TOL, (trial, step, total, want)
            x, y = y, x
        want, _, _ = G.score(S, precision="fp32", L=L)
        assert _rel(total, want) < TOL, (trial, total, want)
        want_oracle = oracle.score(g, S, alpha, L)  # independent of the library: the CPU oracle
        assert _rel(total, want_oracle) < TOL, (trial, total, want_oracle)
    G.free()


def test_noalloc_rejects_oversized_input(cuda_device):
    import torch

    from paper_1910_13874_gb300 import gedwalk

    buf = torch.zeros(64, dtype=torch.float64, device=cuda_device)
    p = buf.data_ptr()
    with pytest.raises(gedwalk.GedWalkError) as e:
        gedwalk.score_step_noalloc(p, p, 16_777_217, p, p, p + 256, 0.1, p + 128)
    assert e.value.status == gedwalk.ERR_INVALID
    assert "16777216" in str(e.value)
    lib = gedwalk.load()
    assert lib.gedwalk_score_step_noalloc(None, None, 10, None, None, None, ctypes.c_double(0.1), None, 0) \
        == gedwalk.ERR_INVALID
