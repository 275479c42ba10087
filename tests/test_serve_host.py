"""Host logic of the serving loop (no GPU): admission by the memory budget, first fit in
arrival order, the in-flight cap, rejection of requests larger than the budget, and the
latency report. Execution is replaced by a host function."""
import random
import threading
import time

import numpy as np
import pytest

from paper_2207_03711_gb300.serve import Request, Server


def _req(tag):
    return Request("energy", np.eye(2), np.zeros((2, 2, 2, 2)), 2, 4, np.zeros(3), tag=tag)


def test_admission_respects_budget_and_inflight_cap():
    lock = threading.Lock()
    live = {"bytes": 0, "n": 0, "max_bytes": 0, "max_n": 0}
    needs = {}

    def run(req):
        with lock:
            live["bytes"] += needs[req.tag]
            live["n"] += 1
            live["max_bytes"] = max(live["max_bytes"], live["bytes"])
            live["max_n"] = max(live["max_n"], live["n"])
        time.sleep(random.Random(req.tag).uniform(0.002, 0.02))
        with lock:
            live["bytes"] -= needs[req.tag]
            live["n"] -= 1
        return 2 * req.tag

    rng = random.Random(0)
    with Server(budget_bytes=1000, max_inflight=3, run_fn=run) as srv:
        futs = []
        for t in range(40):
            needs[t] = rng.randint(50, 600)
            futs.append(srv.submit(_req(t), need_bytes=needs[t]))
        assert [f.result(timeout=30) for f in futs] == [2 * t for t in range(40)]
        st = srv.stats()
    assert live["max_bytes"] <= 1000 and st["peak_used_bytes"] <= 1000
    assert live["max_n"] <= 3 and st["peak_inflight"] <= 3
    assert st["peak_inflight"] >= 2          # requests do overlap
    assert st["completed"] == 40
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"]


def test_small_requests_pass_a_waiting_large_one():
    gate = threading.Event()
    order = []

    def run(req):
        if req.tag == 0:
            gate.wait(5)
        order.append(req.tag)
        return req.tag

    with Server(budget_bytes=100, max_inflight=4, run_fn=run) as srv:
        f0 = srv.submit(_req(0), need_bytes=60)     # holds 60 until released
        f1 = srv.submit(_req(1), need_bytes=70)     # does not fit next to request 0
        f2 = srv.submit(_req(2), need_bytes=30)     # fits: admitted before request 1
        assert f2.result(timeout=5) == 2
        assert not f1.done()
        gate.set()
        assert f0.result(timeout=5) == 0 and f1.result(timeout=5) == 1
    assert order.index(2) < order.index(1)


def test_request_larger_than_budget_is_rejected():
    with Server(budget_bytes=100, run_fn=lambda r: 0) as srv:
        f = srv.submit(_req(0), need_bytes=101)
        with pytest.raises(MemoryError):
            f.result(timeout=5)


def test_cancelled_request_never_runs():
    gate = threading.Event()
    ran = []

    def run(req):
        if req.tag == 0:
            gate.wait(5)
        ran.append(req.tag)
        return req.tag

    with Server(budget_bytes=100, max_inflight=4, run_fn=run) as srv:
        f0 = srv.submit(_req(0), need_bytes=80)     # occupies the budget
        f1 = srv.submit(_req(1), need_bytes=50)     # waits for memory
        f2 = srv.submit(_req(2), need_bytes=50)
        assert f1.cancel()                           # still queued: cancellable
        gate.set()
        assert f0.result(timeout=5) == 0 and f2.result(timeout=5) == 2
        assert f1.cancelled()
        st = srv.stats()
    assert 1 not in ran and st["completed"] == 2


def test_large_request_is_not_starved_by_a_stream_of_small_ones():
    """Budget 100: a request needing 70 never fits next to the small ones (40 each) that
    keep arriving; after max_wait_s it reserves the head of the line and completes while
    the small stream is still arriving."""
    stop = threading.Event()

    def run(req):
        time.sleep(0.02)
        return req.tag

    with Server(budget_bytes=100, max_inflight=4, run_fn=run, max_wait_s=0.1) as srv:
        first = [srv.submit(_req(100 + i), need_bytes=40) for i in range(2)]   # fill the budget
        big = srv.submit(_req(0), need_bytes=70)

        def feeder():
            i = 0
            while not stop.is_set():
                srv.submit(_req(200 + i), need_bytes=40)
                i += 1
                time.sleep(0.005)
        t = threading.Thread(target=feeder, daemon=True)
        t.start()
        assert big.result(timeout=3) == 0
        stop.set()
        t.join()
        assert all(f.result(timeout=5) >= 100 for f in first)
