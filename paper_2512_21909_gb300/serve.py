"""Serving loop for gradient requests of mixed sizes and point groups.

Requests arrive over time (for instance from many geometry-optimisation
steps).  The loop admits a request when a slot is free and its estimated
device footprint fits the memory not yet promised to running requests; the
request then lives on the device (its context holds the amplitudes, Lambda,
DIIS histories and all intermediates) and is driven to its gradient by a
worker thread on the slot's own CUDA stream.  Requests that arrive while
others run are admitted as slots and memory free up, and their kernels
overlap with those of the running requests on the GPU.  A request whose
allocation still fails (the estimate was low) is put back at the head of
the queue and retried when the device is otherwise idle.

Every result is independent of the mix it ran in: the arithmetic of a
request depends only on its own data and options (the ladder mode is chosen
from the request's size, never from the free memory of the moment), so a
request gives the same energy and gradient alone and in the mix.

Host-side scheduling is plain Python threads; every gradient runs in the
CUDA library through `cdcc` (the worker releases the GIL inside each call).
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import cdcc


# ------------------------------------------------------------------ sizes
def _pairs(n_a, n_b, h, gamma):
    return sum(n_a[g] * n_b[g ^ gamma] for g in range(h))


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
    status: str = "pending"
    t_admit: float | None = None
    t_done: float | None = None
    ladder: int = 0
    est_bytes: int = 0
    retries: int = 0
    slot: int = -1
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


def footprint(req: Request, precision: int, ladder: int,
              batch_gb: float = 2.0) -> dict:
    """Element counts of the large device arrays of one request and an
    upper estimate of its peak device memory in bytes."""
    h = req.nirrep
    o, v = req.occ, req.vir
    n = [o[g] + v[g] for g in range(h)]
    t2 = sum(_pairs(o, o, h, G) * _pairs(v, v, h, G) for G in range(h))
    w = sum(_pairs(v, v, h, G) ** 2 for G in range(h))
    ovvv = sum(_pairs(o, v, h, G) * _pairs(v, v, h, G) for G in range(h))
    nnz = sum(req.chol[G] * _pairs(n, n, h, G) for G in range(h))
    # ~64 doubles-sized arrays (amplitudes, residuals, multipliers, two DIIS
    # histories, the recorded residual intermediates and their adjoints),
    # (mc|bd) and its adjoint and slices, L in its blocks, adjoint and slices
    base = 8 * (64 * t2 + 4 * ovvv + 10 * nnz) + (512 << 20)
    if ladder == cdcc.LADDER_STORED:
        k = {cdcc.PREC_TC: 4.5, cdcc.PREC_MIXED: 3.5}.get(precision, 2.0)
        lad = int(8 * w * k)
    else:
        # two batch buffers, the batch slices and, in the density sweep, the
        # slices of the adjoint batch (measured peaks: <= 5 batches)
        lad = int(5.5 * batch_gb * 1e9)
    return dict(t2=t2, w=w, ovvv=ovvv, nnz=nnz, bytes=base + lad)


# ----------------------------------------------------------------- server
class GradientServer:
    """Continuous-batching server on one GPU.

    precision        cdcc.PREC_* of every request
    max_active       slots (concurrent requests, one stream each)
    reserve_bytes    device memory kept free
    stored_max_bytes largest stored-ladder footprint; bigger requests build
                     their ladder integrals on the fly
    """

    def __init__(self, device=0, precision=cdcc.PREC_TC, max_active=4,
                 reserve_bytes=8 << 30, stored_max_bytes=24 << 30,
                 conv_tol=1e-10, batch_gb=2.0, budget_bytes=None):
        import torch
        self.torch = torch
        self.device = device
        self.precision = precision
        self.max_active = max_active
        self.reserve = reserve_bytes
        self.stored_max = stored_max_bytes
        self.conv_tol = conv_tol
        self.batch_gb = batch_gb
        self.budget = budget_bytes
        self.streams = ([torch.cuda.Stream(device) for _ in range(max_active)]
                        if torch.cuda.is_available() else [None] * max_active)
        self.lock = threading.Condition()
        self.max_seen_active = 0

    # --------------------------------------------------------- policy
    def ladder_for(self, req: Request) -> int:
        f = footprint(req, self.precision, cdcc.LADDER_STORED)
        w_bytes = f["bytes"] - footprint(req, self.precision,
                                         cdcc.LADDER_OTF, 0.0)["bytes"]
        return cdcc.LADDER_STORED if w_bytes <= self.stored_max \
            else cdcc.LADDER_OTF

    def _device_budget(self):
        if self.budget is not None:
            return self.budget
        torch = self.torch
        free, _ = torch.cuda.mem_get_info(self.device)
        cached = (torch.cuda.memory_reserved(self.device)
                  - torch.cuda.memory_allocated(self.device))
        return free + cached - self.reserve

    # --------------------------------------------------------- worker
    def execute(self, req: Request, slot: int):
        """One gradient on the slot's stream: (E_corr, g)."""
        torch = self.torch
        st = self.streams[slot]
        if st is None:
            raise RuntimeError("the CUDA library needs a GPU")
        with torch.cuda.stream(st):
            o = cdcc.cdcc_default_options()
            o.device = self.device
            o.precision = self.precision
            o.conv_tol = self.conv_tol
            o.ladder = req.ladder
            o.ladder_batch_gb = self.batch_gb
            ctx = cdcc.cd_ccsd_init(req.nirrep, req.nocc, req.nvir, req.nchol,
                                    req.orb_irrep, req.eps, req.chol_irrep,
                                    req.L, options=o, stream=st.cuda_stream)
            try:
                return cdcc.gradient(ctx, req.dL)
            finally:
                ctx.close()

    def _work(self, req: Request, slot: int, t0: float):
        try:
            req.e, req.g = self.execute(req, slot)
            req.status = "done"
        except cdcc.CdccError as err:
            req.status = ("nomem" if err.status == cdcc.CDCC_ENOMEM
                          else f"error {err.status}: {err}")
        except Exception as err:                      # host-side failure
            req.status = f"error: {err}"
        t = time.perf_counter() - t0
        with self.lock:
            if req.status == "done":
                req.t_done = t
            self._active.pop(req.index, None)
            self._free_slots.append(slot)
            self._committed -= req.est_bytes
            self.lock.notify_all()

    # ------------------------------------------------------------ loop
    def run(self, requests, realtime=True):
        """Serve `requests` (arrival times in seconds from the start);
        returns them with results and times filled in."""
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            r.ladder = self.ladder_for(r)
            r.est_bytes = footprint(r, self.precision, r.ladder,
                                    self.batch_gb)["bytes"]
        queue = []
        self._active = {}
        self._free_slots = list(range(self.max_active))
        self._committed = 0
        budget = self._device_budget()
        threads = []
        t0 = time.perf_counter()
        self.t0 = t0
        with self.lock:
            while pending or queue or self._active:
                now = time.perf_counter() - t0
                while pending and (not realtime or pending[0].arrival <= now):
                    r = pending.pop(0)
                    if not realtime:
                        r.arrival = now
                    queue.append(r)
                # requeue allocation failures at the head
                for r in requests:
                    if r.status == "nomem":
                        r.status = "pending"
                        r.retries += 1
                        queue.insert(0, r)
                admitted = True
                while admitted and queue and self._free_slots:
                    admitted = False
                    for k, r in enumerate(queue):
                        # a retried request runs alone
                        if r.retries and self._active:
                            break
                        if r.retries > 2:
                            r.status = "error: out of device memory"
                            queue.pop(k)
                            admitted = True
                            break
                        fits = self._committed + r.est_bytes <= budget
                        if fits or not self._active:
                            queue.pop(k)
                            slot = self._free_slots.pop(0)
                            r.slot = slot
                            r.status = "running"
                            r.t_admit = time.perf_counter() - t0
                            self._committed += r.est_bytes
                            self._active[r.index] = r
                            self.max_seen_active = max(self.max_seen_active,
                                                       len(self._active))
                            th = threading.Thread(target=self._work,
                                                  args=(r, slot, t0),
                                                  daemon=True)
                            threads.append(th)
                            th.start()
                            admitted = True
                            break
                        if k >= 3:        # bounded look-ahead past the head
                            break
                timeout = 0.5
                if pending and realtime:
                    timeout = max(0.0, min(timeout, pending[0].arrival -
                                           (time.perf_counter() - t0)))
                if pending or queue or self._active:
                    self.lock.wait(timeout=timeout if timeout > 0 else 0.001)
        for th in threads:
            th.join()
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
