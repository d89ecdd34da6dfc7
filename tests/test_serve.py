"""Host logic of the serving loop (CPU): admission by the memory budget and
free slots, arrival times, retry of a request whose allocation failed, and
bookkeeping.  The gradient itself is replaced by a stand-in that sleeps;
the GPU path is covered by test_gpu_serve.py."""
import threading
import time

import numpy as np

from paper_2512_21909_gb300 import cdcc
from paper_2512_21909_gb300.serve import (GradientServer, Request, footprint,
                                          latency_stats)


def _req(i, arrival, o=2, v=4, nchol=6):
    occ, vir, chol = [o], [v], [nchol]
    n = o + v
    return Request(i, arrival, 1, occ, vir, chol,
                   np.zeros(n, np.int32), np.arange(n, dtype=float),
                   np.zeros(nchol, np.int32), np.full(nchol * n * n, i * 1.0),
                   np.ones((2, nchol * n * n)))


class FakeServer(GradientServer):
    def __init__(self, *a, fail_once=(), **k):
        super().__init__(*a, **k)
        self.running = 0
        self.peak = 0
        self.peak_bytes = 0
        self.inflight_bytes = 0
        self.fail_once = set(fail_once)
        self.mu = threading.Lock()
        self.order = []

    def execute(self, req, slot):
        with self.mu:
            self.running += 1
            self.inflight_bytes += req.est_bytes
            self.peak = max(self.peak, self.running)
            self.peak_bytes = max(self.peak_bytes, self.inflight_bytes)
            self.order.append(req.index)
        try:
            time.sleep(0.02 + 0.01 * (req.index % 3))
            if req.index in self.fail_once:
                self.fail_once.discard(req.index)
                raise cdcc.CdccError(cdcc.CDCC_ENOMEM, "fake allocation failure")
            return float(req.L[0]), req.dL.sum(axis=1)
        finally:
            with self.mu:
                self.running -= 1
                self.inflight_bytes -= req.est_bytes


def test_all_requests_served_with_slot_limit():
    reqs = [_req(i, 0.0) for i in range(10)]
    srv = FakeServer(max_active=3, budget_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert srv.peak <= 3 and srv.peak >= 2
    assert [r.e for r in reqs] == [float(i) for i in range(10)]
    st = latency_stats(reqs, srv.wall)
    assert st["done"] == 10 and st["p50_s"] <= st["p99_s"]


def test_memory_budget_limits_concurrency():
    reqs = [_req(i, 0.0) for i in range(8)]
    one = footprint(reqs[0], cdcc.PREC_TC, cdcc.LADDER_STORED)["bytes"]
    srv = FakeServer(max_active=8, budget_bytes=int(2.5 * one),
                     stored_max_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert srv.peak == 2
    assert srv.peak_bytes <= 2.5 * one


def test_oversized_request_runs_alone():
    small = [_req(i, 0.0) for i in range(3)]
    big = _req(3, 0.0, o=4, v=12, nchol=30)
    srv = FakeServer(max_active=4,
                     budget_bytes=footprint(small[0], cdcc.PREC_TC,
                                            cdcc.LADDER_STORED)["bytes"] * 2)
    srv.run(small + [big], realtime=False)
    assert big.status == "done"


def test_arrivals_are_respected():
    reqs = [_req(0, 0.0), _req(1, 0.15), _req(2, 0.3)]
    srv = FakeServer(max_active=4, budget_bytes=1 << 50)
    srv.run(reqs, realtime=True)
    for r in reqs:
        assert r.status == "done"
        assert r.t_admit >= r.arrival - 1e-3
        assert r.latency > 0


def test_failed_allocation_is_retried_alone():
    reqs = [_req(i, 0.0) for i in range(5)]
    srv = FakeServer(max_active=3, budget_bytes=1 << 50, fail_once={1})
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert reqs[1].retries == 1
    assert srv.order.count(1) == 2


def test_ladder_policy_depends_on_size_only():
    srv = FakeServer(max_active=1, stored_max_bytes=1 << 20)
    small, big = _req(0, 0.0, o=2, v=4), _req(1, 0.0, o=4, v=40, nchol=40)
    assert srv.ladder_for(small) == cdcc.LADDER_STORED
    assert srv.ladder_for(big) == cdcc.LADDER_OTF
    f_st = footprint(big, cdcc.PREC_TC, cdcc.LADDER_STORED)
    assert f_st["w"] == 40 ** 4 and f_st["t2"] == 16 * 1600


class FailingServer(FakeServer):
    def execute(self, req, slot):
        if req.index == 2:
            raise cdcc.CdccError(cdcc.CDCC_ENUMERIC, "fake divergence")
        return super().execute(req, slot)


def test_other_failures_are_reported_per_request():
    reqs = [_req(i, 0.0) for i in range(5)]
    srv = FailingServer(max_active=2, budget_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert reqs[2].status.startswith("error")
    assert all(r.status == "done" for k, r in enumerate(reqs) if k != 2)
    st = latency_stats(reqs, srv.wall)
    assert st["done"] == 4 and st["failed"] == 1
