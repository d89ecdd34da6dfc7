"""The Lagrangian check of tests/lagcheck.py (used at c2, where the dense
oracle cannot solve the amplitude and Lambda equations) accepts the oracle's
own converged (t, lambda, Gamma^P) and rejects planted mistakes in lambda
and in Gamma^P (CPU only; c0 and a ragged C2v case)."""
import numpy as np
import pytest
import torch

from synth import make_system, random_system, make_displacements, unpack_dense
from oracle import model, lagrangian
from lagcheck import random_direction, lagrangian_difference

T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa


@pytest.mark.parametrize("which", ["c0", "ragged"])
def test_lagrangian_check_on_the_oracle_solution(which):
    s = (make_system(0) if which == "c0" else
         random_system([3, 2, 2, 1], [7, 5, 4, 3], [12, 10, 9, 8],
                       seed=211, scale=0.4))
    o = s.nocc
    dL = make_displacements(s, 3)
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    r = lagrangian.run_all(h, L, o, tol=1e-12, e_tol=1e-13)
    t1, t2 = r["cc"]["t1"].numpy(), r["cc"]["t2"].numpy()
    l1, l2 = r["lam"]["l1"].numpy(), r["lam"]["l2"].numpy()
    w = np.random.default_rng(5).standard_normal(dL.shape[0])
    D = w @ dL
    gD = float(lagrangian.gradient_from_density(
        r["G"], T(unpack_dense(s, D))[None])[0])
    dt1, dt2 = random_direction(s, t1, t2)
    step = 1e-4   # truncation ~3e-11 at c0 (3e-9 at 1e-3)
    fd = lagrangian_difference(s, t1, t2, l1, l2, dt1, dt2, D, step)
    tol = 1e-8 * max(1.0, abs(gD))
    assert abs(fd - gD) <= tol, (fd, gD)
    # a Lambda off by 1 % breaks the stationarity in t
    bad = lagrangian_difference(s, t1, t2, l1, 1.01 * l2, dt1, dt2, D, step)
    assert abs(bad - gD) > 100 * tol, (bad, gD)
    bad = lagrangian_difference(s, t1, t2, 1.01 * l1, l2, dt1, dt2, D, step)
    assert abs(bad - gD) > 100 * tol, (bad, gD)
    # a Gamma^P off by 1 %
    assert abs(fd - 1.01 * gD) > 100 * tol
