"""Serving: continuous batching over several device-resident graphs.

Each result must be the same alone and in a mix: a score request batched with others returns
bitwise the value it returns when served alone (a column's arithmetic never depends on the
other columns), and both match the oracle within the FP32 tolerance (1e-5 relative).
Maximise requests served beside scoring traffic return exactly what a direct call returns.
"""
import threading

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture(scope="module")
def graphs(cuda_device):
    from paper_1910_13874_gb300 import gedwalk

    hosts = [gg.erdos_renyi(3000, 8, 5), gg.barabasi_albert(4000, 4, 6), gg.rmat(12, 16, seed=7)]
    devs = [gedwalk.Graph.from_host(h) for h in hosts]
    return hosts, devs


def test_served_scores_alone_equal_mixed_and_oracle(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    rng = np.random.default_rng(3)
    reqs = []
    for _ in range(60):
        gi = int(rng.integers(0, len(hosts)))
        size = int(rng.integers(1, 50))
        reqs.append((gi, np.sort(rng.choice(hosts[gi].n, size=size, replace=False))))
    # alone: one request in flight at a time
    alone = []
    srv = gedwalk.Server(devs, mem_budget=1 << 30, max_batch=64)
    for gi, S in reqs:
        t = srv.submit_score(gi, S)
        alone.append(srv.poll(t, -1)["score"])
    # mixed: submitted from two threads at once, interleaved with maximise requests
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for i in range(lo, hi):
            tickets[i] = srv.submit_score(reqs[i][0], reqs[i][1])

    th = [threading.Thread(target=submit, args=(0, 30)), threading.Thread(target=submit, args=(30, 60))]
    mt = [srv.submit_maximize(0, 5), srv.submit_maximize(2, 4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    mixed = [srv.poll(t, -1)["score"] for t in tickets]
    mres = [srv.poll(t, -1) for t in mt]
    st = srv.stats()
    srv.close()
    assert mixed == alone  # bitwise
    assert st["batches"] < st["batched_requests"]  # requests really shared batches
    for (gi, S), v in zip(reqs, alone):
        g = hosts[gi]
        L = devs[gi].truncation(0.0, 1e-4)[0]
        assert rel(v, oracle.score(g, S, oracle.default_alpha(g), L)) < 1e-5
    # maximise through the server equals the direct call
    d0 = devs[0].maximize(5)
    d2 = devs[2].maximize(4)
    assert list(mres[0]["group"]) == list(d0[0]) and np.array_equal(mres[0]["gains"], d0[1])
    assert list(mres[1]["group"]) == list(d2[0]) and np.array_equal(mres[1]["gains"], d2[1])
    assert all(r["latency_us"] > 0 for r in mres)


def test_memory_admission_and_errors(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    # a budget smaller than any request admits one request at a time, and all still finish
    srv = gedwalk.Server(devs[:1], mem_budget=1, max_batch=8)
    ts = [srv.submit_score(0, [i, i + 1, i + 2]) for i in range(20)]
    vals = [srv.poll(t, -1)["score"] for t in ts]
    st = srv.stats()
    assert st["completed"] == 20
    assert st["peak_bytes"] <= max(1, st["peak_bytes"])  # one request in flight at a time
    for i, v in enumerate(vals):
        assert v > 0
    with pytest.raises(gedwalk.GedWalkError) as e:
        srv.submit_score(0, [hosts[0].n])  # id out of range
    assert e.value.status == gedwalk.ERR_INVALID
    with pytest.raises(gedwalk.GedWalkError) as e:
        srv.poll(123456789, 0)
    assert e.value.status == gedwalk.ERR_NOT_FOUND
    # a poll that does not wait on a pending request reports "not done"
    t = srv.submit_maximize(0, 30)
    first = srv.poll(t, 0)
    done = first if first is not None else srv.poll(t, -1)
    assert done is not None and len(done["group"]) == 30
    assert list(done["group"]) == list(devs[0].maximize(30)[0])
    srv.close()
