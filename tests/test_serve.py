"""Host logic of the native serving loop (CPU): admission by the memory
budget and free slots, arrival times, retry of a request whose allocation
failed, per-request failures and bookkeeping, through the serving entry
points of the C ABI (cdcc_server_create / cdcc_submit / cdcc_poll).  The
gradient itself is replaced by a host executor that sleeps; the GPU path is
covered by test_gpu_serve.py."""
import threading
import time

import numpy as np

from paper_2512_21909_gb300 import cdcc
from paper_2512_21909_gb300.serve import (GradientServer, Request,
                                          footprint_bytes, latency_stats)


def _req(i, arrival, o=2, v=4, nchol=6):
    occ, vir, chol = [o], [v], [nchol]
    n = o + v
    return Request(i, arrival, 1, occ, vir, chol,
                   np.zeros(n, np.int32), np.arange(n, dtype=float),
                   np.zeros(nchol, np.int32), np.full(nchol * n * n, i * 1.0),
                   np.ones((2, nchol * n * n)))


class Recorder:
    """Host executor: sleeps, records concurrency and bytes in flight."""

    def __init__(self, fail_once=(), fail_always=(), precision=cdcc.PREC_TC):
        self.running = 0
        self.peak = 0
        self.peak_bytes = 0
        self.inflight = 0
        self.fail_once = set(fail_once)
        self.fail_always = set(fail_always)
        self.mu = threading.Lock()
        self.order = []
        self.precision = precision

    def __call__(self, req, slot):
        est = footprint_bytes(req, self.precision, cdcc.LADDER_STORED)
        with self.mu:
            self.running += 1
            self.inflight += est
            self.peak = max(self.peak, self.running)
            self.peak_bytes = max(self.peak_bytes, self.inflight)
            self.order.append(req.index)
        try:
            time.sleep(0.02 + 0.01 * (req.index % 3))
            if req.index in self.fail_once:
                self.fail_once.discard(req.index)
                raise cdcc.CdccError(cdcc.CDCC_ENOMEM, "fake allocation")
            if req.index in self.fail_always:
                raise cdcc.CdccError(cdcc.CDCC_ENUMERIC, "fake divergence")
            return float(req.L[0]), req.dL.sum(axis=1), 1e-12 * req.index
        finally:
            with self.mu:
                self.running -= 1
                self.inflight -= est


def _server(rec, **kw):
    kw.setdefault("stored_max_bytes", 1 << 50)
    return GradientServer(executor=rec, **kw)


def test_all_requests_served_with_slot_limit():
    reqs = [_req(i, 0.0) for i in range(10)]
    rec = Recorder()
    srv = _server(rec, max_active=3, budget_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs), [r.status for r in reqs]
    assert 2 <= rec.peak <= 3
    assert srv.max_seen_active <= 3
    assert [r.e for r in reqs] == [float(i) for i in range(10)]
    assert all(np.array_equal(r.g, np.full(2, r.L.size * 1.0)) for r in reqs)
    assert [r.err_dE for r in reqs] == [1e-12 * i for i in range(10)]
    st = latency_stats(reqs, srv.wall)
    assert st["done"] == 10 and st["p50_s"] <= st["p99_s"]


def test_memory_budget_limits_concurrency():
    reqs = [_req(i, 0.0) for i in range(8)]
    one = footprint_bytes(reqs[0], cdcc.PREC_TC, cdcc.LADDER_STORED)
    rec = Recorder()
    srv = _server(rec, max_active=8, budget_bytes=int(2.5 * one))
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert rec.peak == 2
    assert rec.peak_bytes <= 2.5 * one


def test_oversized_request_runs_alone():
    small = [_req(i, 0.0) for i in range(3)]
    big = _req(3, 0.0, o=4, v=12, nchol=30)
    rec = Recorder()
    srv = _server(rec, max_active=4,
                  budget_bytes=footprint_bytes(small[0], cdcc.PREC_TC,
                                               cdcc.LADDER_STORED) * 2)
    srv.run(small + [big], realtime=False)
    assert big.status == "done"
    assert all(r.status == "done" for r in small)


def test_arrivals_are_respected():
    reqs = [_req(0, 0.0), _req(1, 0.15), _req(2, 0.3)]
    srv = _server(Recorder(), max_active=4, budget_bytes=1 << 50)
    srv.run(reqs, realtime=True)
    for r in reqs:
        assert r.status == "done"
        assert r.t_admit >= r.arrival - 1e-3
        assert r.latency > 0


def test_failed_allocation_is_retried_alone():
    reqs = [_req(i, 0.0) for i in range(5)]
    rec = Recorder(fail_once={1})
    srv = _server(rec, max_active=3, budget_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert all(r.status == "done" for r in reqs)
    assert reqs[1].retries == 1
    assert rec.order.count(1) == 2


def test_ladder_policy_depends_on_size_only():
    # stored integrals of the small request fit 1 MB, the big one's do not
    small, big = _req(0, 0.0, o=2, v=4), _req(1, 0.0, o=4, v=40, nchol=40)
    rec = Recorder()
    srv = GradientServer(executor=rec, max_active=1, budget_bytes=1 << 50,
                         stored_max_bytes=1 << 20)
    srv.run([small, big], realtime=False)
    assert small.ladder == cdcc.LADDER_STORED
    assert big.ladder == cdcc.LADDER_OTF
    # the estimate grows with the stored (ab|cd) integrals: v^4 doubles,
    # 36 bytes per element in TC; on the fly keeps two BF16 slices of W+
    # and W- (the +/- packed ladder: canonical pairs c >= d, 40*41/2 of
    # them in C1) from one ladder application to the next
    st = footprint_bytes(big, cdcc.PREC_TC, cdcc.LADDER_STORED)
    otf = footprint_bytes(big, cdcc.PREC_TC, cdcc.LADDER_OTF, 0.0)
    assert st - otf == int(8 * 40 ** 4 * 4.5) - 8 * (40 * 41 // 2) ** 2


def test_other_failures_are_reported_per_request():
    reqs = [_req(i, 0.0) for i in range(5)]
    rec = Recorder(fail_always={2})
    srv = _server(rec, max_active=2, budget_bytes=1 << 50)
    srv.run(reqs, realtime=False)
    assert reqs[2].status.startswith("error")
    assert "CDCC_ENUMERIC" in reqs[2].status
    assert all(r.status == "done" for k, r in enumerate(reqs) if k != 2)
    st = latency_stats(reqs, srv.wall)
    assert st["done"] == 4 and st["failed"] == 1


def test_native_entry_points_poll_and_wait():
    # the C ABI directly: submit, non-blocking poll, blocking wait
    rec = Recorder()
    by = {}
    r0 = _req(7, 0.0)
    by[1] = r0

    def run(ticket, desc, slot, e_ptr, g_ptr, err_ptr, _u):
        d = desc.contents
        assert (d.nocc, d.nvir, d.nchol, d.nx) == (2, 4, 6, 2)
        e, g, de = rec(by[int(ticket)], slot)
        e_ptr[0], err_ptr[0] = e, de
        g_ptr[0], g_ptr[1] = g[0], g[1]
        return cdcc.CDCC_OK
    fn = cdcc.EXECUTOR_FN(run)
    so = cdcc.cdcc_server_default_options()
    so.max_active = 2
    so.executor = fn
    srv = cdcc.Server(None, so)
    try:
        d, keep = r0.desc()
        tk = srv.submit(d, keep)
        assert tk == 1
        res, _ = srv.poll(tk, 2)
        assert res.state in (cdcc.JOB_QUEUED, cdcc.JOB_RUNNING,
                             cdcc.JOB_DONE)
        res, g = srv.wait(tk, 2, 10.0)
        assert res.state == cdcc.JOB_DONE and res.status == cdcc.CDCC_OK
        assert res.e_corr == 7.0 and np.array_equal(g, [216.0, 216.0])
        try:
            srv.poll(99, 2)
            raise AssertionError("unknown ticket accepted")
        except cdcc.CdccError as err:
            assert err.status == cdcc.CDCC_EINVAL
    finally:
        srv.close()
