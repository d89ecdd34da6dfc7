"""Serving loop for gradient requests of mixed sizes and point groups.

A thin driver over the native serving entry points of include/cdcc.h
(cdcc_server_create / cdcc_submit / cdcc_poll): requests are submitted at
their arrival times and their results collected; admission (by free slots
and the estimated device footprint), residency of each admitted request's
state in its own context, concurrent execution on per-slot CUDA streams,
retry of requests whose allocation failed and the error report attached to
every result all happen inside the library.

Every result is independent of the mix it ran in: the arithmetic of a
request depends only on its own data and options (the ladder mode is chosen
from the request's size, never from the free memory of the moment), so a
request gives the same energy and gradient alone and in the mix.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import cdcc


@dataclass
class Request:
    """One gradient request (host arrays; the layout of cd_ccsd_init)."""
    index: int
    arrival: float
    nirrep: int
    occ: list
    vir: list
    chol: list
    orb_irrep: np.ndarray
    eps: np.ndarray
    chol_irrep: np.ndarray
    L: np.ndarray
    dL: np.ndarray
    # filled by the server
    e: float | None = None
    g: np.ndarray | None = None
    err_dE: float | None = None
    status: str = "pending"
    t_admit: float | None = None
    t_done: float | None = None
    ladder: int = 0
    retries: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nocc(self):
        return int(sum(self.occ))

    @property
    def nvir(self):
        return int(sum(self.vir))

    @property
    def nchol(self):
        return int(sum(self.chol))

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival

    @classmethod
    def from_system(cls, index, arrival, s, dL):
        return cls(index, arrival, s.nirrep, list(s.occ), list(s.vir),
                   list(s.chol), s.orb_irrep, s.eps, s.chol_irrep, s.L,
                   np.ascontiguousarray(dL))

    def desc(self):
        return cdcc.job_desc(self.nirrep, self.nocc, self.nvir, self.nchol,
                             self.orb_irrep, self.eps, self.chol_irrep,
                             self.L, self.dL)


def footprint_bytes(req: Request, precision: int, ladder: int,
                    batch_gb: float = 2.0) -> int:
    """The library's admission estimate of a request's peak device bytes."""
    d, _keep = req.desc()
    return cdcc.cdcc_job_footprint(d, precision, ladder, batch_gb)


class GradientServer:
    """Continuous-batching server on one GPU (native request loop).

    precision        cdcc.PREC_* of every request
    max_active       slots (concurrent requests, one stream each)
    reserve_bytes    device memory kept free
    stored_max_bytes largest stored-ladder footprint; bigger requests build
                     their ladder integrals on the fly
    budget_bytes     device memory the requests may use (default: free
                     memory at start minus reserve_bytes)
    executor         optional host stand-in f(request, slot) -> (e, g, dE)
                     (raising cdcc.CdccError reports its status), for tests
                     of the scheduling without a GPU
    """

    def __init__(self, device=0, precision=cdcc.PREC_TC, max_active=4,
                 reserve_bytes=8 << 30, stored_max_bytes=24 << 30,
                 conv_tol=1e-10, batch_gb=2.0, budget_bytes=None,
                 executor=None, error_report=True):
        self.device = device
        self.precision = precision
        self.max_active = max_active
        self.reserve = reserve_bytes
        self.stored_max = stored_max_bytes
        self.conv_tol = conv_tol
        self.batch_gb = batch_gb
        self.budget = budget_bytes
        self.executor = executor
        self.error_report = error_report
        self.max_seen_active = 0
        self.wall = 0.0

    def _native(self, by_ticket):
        o = cdcc.cdcc_default_options()
        o.device = self.device
        o.precision = self.precision
        o.conv_tol = self.conv_tol
        o.ladder_batch_gb = self.batch_gb
        so = cdcc.cdcc_server_default_options()
        so.max_active = self.max_active
        so.reserve_gb = self.reserve / 1e9
        so.stored_max_gb = self.stored_max / 1e9
        so.error_report = 1 if self.error_report else 0
        if self.budget is not None:
            so.budget_gb = self.budget / 1e9
        keep = None
        if self.executor is not None:
            user = self.executor

            def run(ticket, desc, slot, e_ptr, g_ptr, err_ptr, _u):
                req = by_ticket[int(ticket)]
                try:
                    e, g, de = user(req, slot)
                except cdcc.CdccError as err:
                    return err.status
                e_ptr[0] = float(e)
                err_ptr[0] = float(de)
                for k, x in enumerate(np.asarray(g, dtype=float)):
                    g_ptr[k] = x
                return cdcc.CDCC_OK
            keep = cdcc.EXECUTOR_FN(run)
            so.executor = keep
        else:
            import torch
            if torch.cuda.is_available():
                torch.cuda.empty_cache()   # the library allocates natively
        srv = cdcc.Server(o, so)
        srv._executor_keep = keep
        return srv

    def run(self, requests, realtime=True):
        """Serve `requests` (arrival times in seconds from the start);
        returns them with results and times filled in."""
        by_ticket = {}
        srv = self._native(by_ticket)
        pending = sorted(requests, key=lambda r: r.arrival)
        live = {}
        t0 = time.perf_counter()
        try:
            while pending or live:
                now = time.perf_counter() - t0
                while pending and (not realtime or pending[0].arrival <= now):
                    r = pending.pop(0)
                    if not realtime:
                        r.arrival = now
                    d, keep = r.desc()
                    # register before submitting: a worker may start at once
                    tk_probe = len(by_ticket) + 1
                    by_ticket[tk_probe] = r
                    tk = srv.submit(d, keep)
                    if tk != tk_probe:
                        by_ticket.pop(tk_probe, None)
                        by_ticket[tk] = r
                    r.extra["t_submit"] = time.perf_counter() - t0
                    r.status = "queued"
                    live[tk] = r
                for tk in list(live):
                    r = live[tk]
                    res, g = srv.poll(tk, r.dL.shape[0])
                    if res.state == cdcc.JOB_RUNNING and r.t_admit is None:
                        r.status = "running"
                    if res.state in (cdcc.JOB_DONE, cdcc.JOB_FAILED):
                        ts = r.extra["t_submit"]
                        r.t_admit = ts + res.t_wait
                        r.ladder = res.ladder
                        r.retries = res.retries
                        if res.state == cdcc.JOB_DONE:
                            r.e, r.g, r.err_dE = res.e_corr, g.copy(), \
                                res.err_dE
                            r.extra["dE"] = res.err_dE
                            r.t_done = r.t_admit + res.t_run
                            r.status = "done"
                        else:
                            msg = res.message.decode(errors="replace")
                            r.status = (f"error {res.status}: "
                                        f"{cdcc.STATUS.get(res.status)} {msg}")
                        del live[tk]
                if pending or live:
                    nxt = 0.002
                    if pending and realtime:
                        nxt = min(nxt, max(0.0, pending[0].arrival -
                                           (time.perf_counter() - t0)))
                    time.sleep(max(nxt, 0.0005))
        finally:
            self.max_seen_active = srv.max_active_seen()
            srv.close()
        self.wall = time.perf_counter() - t0
        return requests


def latency_stats(requests, wall=None):
    """p50 / p99 time-to-gradient (completion - arrival) and jobs/s."""
    done = [r for r in requests if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(0)
    span = wall if wall is not None else (
        max(r.t_done for r in done) - min(r.arrival for r in requests)
        if done else 0.0)
    return dict(done=len(done), failed=len(requests) - len(done),
                p50_s=float(np.percentile(lat, 50)) if len(lat) else None,
                p99_s=float(np.percentile(lat, 99)) if len(lat) else None,
                jobs_per_s=len(done) / span if span > 0 else None,
                wall_s=span)
