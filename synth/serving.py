"""Seeded serving workload: gradient requests of mixed sizes and point groups
arriving as a Poisson stream (the c4 workload).

  * 64 requests; inter-arrival times ~ Exp(mean 0.5 s) from their own
    generator (seed BASE_SEED + 4).
  * Request j draws, from a generator seeded BASE_SEED + 4 + 1009 (j + 1):
    o ~ U{4..40}, v = 9 o, nL = 4 (o + v) = 40 o, and the point group
    uniformly from C1, C2v, D2h.  Orbitals are split over irreps as for the
    fixed workloads (C1: one irrep; D2h: even over 8; C2v: 40/25/20/15 %;
    floor + largest remainder, so small D2h requests have empty irreps), the
    Cholesky vectors in proportion to the orbital pairs of each irrep.
  * The arrays are those of random_system with seed BASE_SEED + 4 +
    1009 (j + 1) + 1, scaled by the per-request s (table below); 6
    displacements per request.

The per-request scale s = min(1, (0.04 o / |E_MP2(s=1)|)^(1/4)) targets the
same ~-0.04 Eh of correlation energy per occupied orbital as the fixed
workloads.  It is a stored constant (serving_scales.json), written by
`python -m oracle.calibrate_scale --serving`; nothing here computes it.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

from .gen import BASE_SEED, irrep_split, chol_split, random_system, System

GROUPS = {"C1": (1, "even"), "C2v": (4, (0.40, 0.25, 0.20, 0.15)),
          "D2h": (8, "even")}
GROUP_ORDER = ("C1", "C2v", "D2h")
NJOBS = 64
MEAN_INTERARRIVAL = 0.5
NX = 6
_HERE = os.path.dirname(os.path.abspath(__file__))
SCALES_FILE = os.path.join(_HERE, "serving_scales.json")


@dataclass
class JobSpec:
    index: int
    arrival: float      # seconds after the start of the stream
    group: str
    o: int
    v: int
    nchol: int
    seed: int

    @property
    def occ_vir_chol(self):
        h, split = GROUPS[self.group]
        occ = irrep_split(self.o, h, split)
        vir = irrep_split(self.v, h, split)
        norb = [occ[g] + vir[g] for g in range(h)]
        return occ, vir, chol_split(self.nchol, h, norb)


def serving_jobs(njobs: int = NJOBS) -> list:
    """The request list (sizes, groups, arrival times); no arrays."""
    ra = np.random.Generator(np.random.PCG64(BASE_SEED + 4))
    arrivals = np.cumsum(ra.exponential(MEAN_INTERARRIVAL, njobs))
    jobs = []
    for j in range(njobs):
        seed = BASE_SEED + 4 + 1009 * (j + 1)
        r = np.random.Generator(np.random.PCG64(seed))
        o = int(r.integers(4, 41))
        group = GROUP_ORDER[int(r.integers(0, 3))]
        jobs.append(JobSpec(j, float(arrivals[j]), group, o, 9 * o, 40 * o,
                            seed + 1))
    return jobs


def _scales():
    if not os.path.exists(SCALES_FILE):
        return {}
    with open(SCALES_FILE) as f:
        return {int(k): float(v) for k, v in json.load(f).items()}


def job_system(spec: JobSpec, scale: float | None = None) -> System:
    """Arrays of one request (scale None: the stored per-request s)."""
    if scale is None:
        tab = _scales()
        if spec.index not in tab:
            raise KeyError(f"no stored scale for request {spec.index}; run "
                           "python -m oracle.calibrate_scale --serving")
        scale = tab[spec.index]
    occ, vir, chol = spec.occ_vir_chol
    s = random_system(occ, vir, chol, seed=spec.seed, scale=scale,
                      name=f"c4-job{spec.index}")
    s.extra["group"] = spec.group
    return s
