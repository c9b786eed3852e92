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


def test_maximise_footprint_covers_the_memory_held(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    for gi, k in ((0, 10), (2, 12)):
        srv = gedwalk.Server(devs[gi:gi + 1], mem_budget=1 << 34)
        r = srv.poll(srv.submit_maximize(0, k), -1)
        st = srv.stats()
        srv.close()
        assert len(r["group"]) == k
        # the charge of the run (its footprint) covers what the worker's buffers hold afterwards,
        # and is not grossly above it
        assert 0 < st["idle_held_bytes"] <= st["peak_bytes"] <= 2 * st["idle_held_bytes"], st


def test_budget_below_two_maximise_footprints_never_runs_two(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    srv = gedwalk.Server(devs[:1], mem_budget=1 << 34)
    alone = srv.poll(srv.submit_maximize(0, 10), -1)
    F = srv.stats()["peak_bytes"]
    srv.close()
    budget = int(1.5 * F)
    srv = gedwalk.Server(devs[:1], mem_budget=budget)
    ts = [srv.submit_maximize(0, 10) for _ in range(4)]
    res = [srv.poll(t, -1) for t in ts]
    st = srv.stats()
    srv.close()
    assert st["peak_maximize_running"] == 1, st
    assert st["peak_bytes"] <= budget, st
    assert st["admitted_after_wait"] >= 3 and st["completed"] == 4, st
    for r in res:
        assert list(r["group"]) == list(alone["group"]) and np.array_equal(r["gains"], alone["gains"])
    # with room for four footprints the same requests run side by side, with the same results
    srv = gedwalk.Server(devs[:1], mem_budget=8 * F)
    ts = [srv.submit_maximize(0, 10) for _ in range(4)]
    res = [srv.poll(t, -1) for t in ts]
    st = srv.stats()
    srv.close()
    assert st["peak_maximize_running"] >= 2 and st["peak_bytes"] <= 8 * F, st
    for r in res:
        assert list(r["group"]) == list(alone["group"]) and np.array_equal(r["gains"], alone["gains"])


def test_tiny_budget_releases_idle_workspaces(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    reqs = [(i % 2, [3 * i, 3 * i + 1, 3 * i + 2]) for i in range(12)]
    srv = gedwalk.Server(devs[:2], mem_budget=1 << 34)
    want = [srv.poll(srv.submit_score(gi, S), -1)["score"] for gi, S in reqs]
    srv.close()
    # a budget below any request: the two lanes never hold memory at once, the idle one is
    # released to admit the other, and every result is unchanged
    srv = gedwalk.Server(devs[:2], mem_budget=1, max_batch=8)
    ts = [srv.submit_score(gi, S) for gi, S in reqs]
    vals = [srv.poll(t, -1)["score"] for t in ts]
    st = srv.stats()
    srv.close()
    assert vals == want
    assert st["completed"] == 12 and st["releases"] >= 1, st


def test_served_alpha_is_fixed_per_graph(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    srv = gedwalk.Server(devs[:1])
    a0 = devs[0].alpha_default
    t = srv.submit_score(0, [1, 2, 3])
    with pytest.raises(gedwalk.GedWalkError) as e:
        srv.submit_score(0, [1, 2, 3], alpha=a0 / 2)
    assert e.value.status == gedwalk.ERR_INVALID
    with pytest.raises(gedwalk.GedWalkError) as e:
        srv.submit_maximize(0, 3, alpha=a0 / 2)
    assert e.value.status == gedwalk.ERR_INVALID
    # the requests with the served alpha are unaffected
    v = srv.poll(t, -1)["score"]
    assert v == srv.poll(srv.submit_score(0, [1, 2, 3], alpha=a0), -1)["score"] and v > 0
    srv.close()


def test_memory_admission_and_errors(graphs):
    from paper_1910_13874_gb300 import gedwalk

    hosts, devs = graphs
    # a budget smaller than any request: each runs when nothing else holds memory; all finish
    srv = gedwalk.Server(devs[:1], mem_budget=1, max_batch=8)
    ts = [srv.submit_score(0, [i, i + 1, i + 2]) for i in range(20)]
    vals = [srv.poll(t, -1)["score"] for t in ts]
    st = srv.stats()
    assert st["completed"] == 20
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
