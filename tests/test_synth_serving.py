"""The serving workload generator follows its stated recipe (CPU)."""
import numpy as np

from synth.serving import (serving_jobs, job_system, GROUPS, NJOBS,
                           MEAN_INTERARRIVAL, _scales)
from synth.gen import pair_count


def test_requests_follow_the_recipe():
    jobs = serving_jobs()
    assert len(jobs) == NJOBS
    arr = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(arr) > 0) and arr[0] > 0
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - MEAN_INTERARRIVAL) < 0.25   # 64 draws of Exp(0.5)
    for j in jobs:
        assert 4 <= j.o <= 40 and j.v == 9 * j.o and j.nchol == 40 * j.o
        assert j.group in GROUPS
        occ, vir, chol = j.occ_vir_chol
        h = GROUPS[j.group][0]
        assert len(occ) == h and sum(occ) == j.o and sum(vir) == j.v
        assert sum(chol) == j.nchol
    assert {j.group for j in jobs} == set(GROUPS)


def test_requests_are_deterministic_and_scaled():
    a, b = serving_jobs(), serving_jobs()
    assert [(x.o, x.group, x.arrival, x.seed) for x in a] == \
        [(x.o, x.group, x.arrival, x.seed) for x in b]
    tab = _scales()
    assert sorted(tab) == list(range(NJOBS))
    assert all(0 < v <= 1 for v in tab.values())
    small = min(a, key=lambda j: j.o)
    s1, s2 = job_system(small), job_system(small)
    assert np.array_equal(s1.L, s2.L) and s1.scale == tab[small.index]
    # Cholesky vectors split in proportion to the orbital pairs of each irrep
    norb = [s1.occ[g] + s1.vir[g] for g in range(s1.nirrep)]
    npp = [pair_count(s1.nirrep, norb, g) for g in range(s1.nirrep)]
    share = np.array(s1.chol) / sum(s1.chol)
    assert np.abs(share - np.array(npp) / sum(npp)).max() < 2.0 / sum(s1.chol)
