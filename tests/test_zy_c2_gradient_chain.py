"""Full-size C2v workload c2 (o = 40, v = 360, nL = 1600, 24 displacements):
the gradient chain of the tensor-core schedule -- amplitudes t, Lambda
multipliers, Cholesky-basis density Gamma^P and the gradient -- against the
oracle's Lagrangian (Sec. 2.2; check in tests/lagcheck.py).

The dense oracle cannot solve the c2 amplitude and Lambda equations (its
reverse-mode Lambda needs the dense O(v^4) integrals), but it evaluates the
Lagrangian Lag(t, lambda; h, L) = E + lambda1 . R1 + lambda2 . R2 at given
(t, lambda).  One central difference of Lag at the GPU's (t, lambda) along
a random amplitude direction dt together with a random combination D of the
24 displacements must equal the GPU's <Gamma^P, D>:

  * the dt part vanishes only if lambda solves the Lambda equations
    (Lag stationary in t);
  * the D part is dLag/dL . D at fixed h, exactly (Lag is quadratic in L),
    which is what Gamma^P contracts to.

The amplitude equations themselves are checked against the oracle's
residual rows in test_gpu_c2.py.  Tolerance |FD - <Gamma^P, D>| <= 1e-6
max(1, |<Gamma^P, D>|), as for the finite difference of test_gpu_c2.py:
at c2 the step 1e-4 leaves a truncation and rounding error of about 1e-11
(steps 1e-4 and 2e-4 differ by 3.6e-11 on MP2-like amplitudes), and the
Lambda residual (converged to max |G/D| <= 1e-10) and the exact-slice
arithmetic are expected to contribute about 1e-9.  A 1 % error in lambda2
moves the difference by about 1e-4 (c0 and c1), one in lambda1 by 5e-6 at
c0 (tests/test_oracle_lagcheck.py) and 3e-7 at c1, below this tolerance.
The two Lagrangian evaluations take about four minutes of host time
(symmetry-blocked oracle), so this file runs after the others.
"""
import numpy as np
import pytest
import torch

from synth import make_system, make_displacements
from lagcheck import random_direction, lagrangian_difference

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def test_c2_gradient_chain_against_oracle_lagrangian(cd):
    s = make_system(2)
    o, v = s.nocc, s.nvir
    dL = make_displacements(s)
    w = np.random.default_rng(3).standard_normal(dL.shape[0])
    D = w @ dL
    opt = cd.cdcc_default_options()
    opt.precision = cd.PREC_TC
    ctx = cd.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol, s.orb_irrep,
                          s.eps, s.chol_irrep, s.L, options=opt)
    cd.ccsd_solve(ctx)
    t1 = cd.cdcc_get_amplitudes(ctx, 0, o, v)
    t2 = cd.cdcc_get_amplitudes(ctx, 1, o, v)
    cd.lambda_solve(ctx)
    l1 = cd.cdcc_get_amplitudes(ctx, 2, o, v)
    l2 = cd.cdcc_get_amplitudes(ctx, 3, o, v)
    cd.build_density(ctx, s.n)
    g = cd.contract_dL(ctx, dL)
    gD = float(cd.contract_dL(ctx, D[None])[0])
    cd.cd_ccsd_free(ctx)
    # the contraction is linear in the displacement
    assert abs(gD - float(w @ g)) <= 1e-10 * max(1.0, abs(gD))
    dt1, dt2 = random_direction(s, t1, t2)
    fd = lagrangian_difference(s, t1, t2, l1, l2, dt1, dt2, D, 1e-4)
    assert abs(fd - gD) <= 1e-6 * max(1.0, abs(gD)), (fd, gD)
