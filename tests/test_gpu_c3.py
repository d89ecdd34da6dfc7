"""Full-size D2h workload at the paper's scale (o = 60, v = 540, nL = 2400,
36 displacements) in the tensor-core schedule with the ladder assembled on
the fly (the stored ladder integrals alone would be 85 GB).

The dense oracle cannot run at this size; what holds at any size is
checked instead: the gradient along two displacements equals a central
difference of the GPU's total energy (the library rebuilds h = diag(eps) -
G(L) from the L it is given, so the prediction adds -sum_pq D_pq dG_pq/dx
with the one-particle density D the GPU returns; G is quadratic in L and its
central difference exact).  Step 1e-3; |dg| <= 1e-6.  The amplitude
equations at full size are checked against the oracle on the C2v workload
(test_gpu_c2.py).
"""
import numpy as np
import pytest
import torch

from synth import make_system, make_displacements, unpack_dense
from oracle import model

pytestmark = pytest.mark.gpu

T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def _init(cd, s, L):
    o = cd.cdcc_default_options()
    o.precision = cd.PREC_TC
    return cd.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol, s.orb_irrep,
                           s.eps, s.chol_irrep, L, options=o)


def test_c3_gradient_matches_finite_difference(cd):
    s = make_system(3)
    dL = make_displacements(s, 2)
    o = s.nocc
    ctx = _init(cd, s, s.L)
    assert cd.cdcc_ladder_mode(ctx) == cd.LADDER_OTF
    e, _, _ = cd.ccsd_solve(ctx)
    cd.lambda_solve(ctx)
    D = cd.build_density(ctx, s.n)
    g = cd.contract_dL(ctx, dL)
    cd.cd_ccsd_free(ctx)
    assert np.isfinite(e) and np.all(np.isfinite(g))
    eps = s.eps
    step = 1e-3
    for x in range(2):
        Ex, Gx = [], []
        for sgn in (1.0, -1.0):
            Lx = s.L + sgn * step * dL[x]
            ctx = _init(cd, s, Lx)
            ec, _, _ = cd.ccsd_solve(ctx)
            cd.cd_ccsd_free(ctx)
            G = model.two_electron_fock(T(unpack_dense(s, Lx)), o).numpy()
            Ex.append(ec + float(np.sum(2.0 * eps[:o] - np.diag(G)[:o])))
            Gx.append(G)
        fd = (Ex[0] - Ex[1]) / (2 * step)
        pred = g[x] - float(np.sum(D * (Gx[0] - Gx[1]) / (2 * step)))
        assert abs(pred - fd) <= 1e-6, (x, pred, fd)
