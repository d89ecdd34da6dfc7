"""Full-size C2v workload (o = 40, v = 360, nL = 1600, split 40/25/20/15 %)
in the tensor-core schedule, checked where the dense FP64 oracle still
answers at this size:

  * energy: the correlation energy returned by the GPU equals the oracle's
    energy functional (oracle.rows.energy) at the GPU's amplitudes;
  * amplitude equations: the oracle's residual at the GPU's amplitudes
    vanishes to the convergence threshold on all of R1 and on sampled rows
    R2[i, j, :, :] (pairs inside one irrep and across irreps);
  * gradient (a property at any size): g_x equals a central difference of
    the GPU's total energy along dL_x.  The library builds
    h = diag(eps) - G(L) from the L it is given, so the displaced runs move
    h as well; the prediction adds that term, - sum_pq D_pq dG_pq/dx, with
    D the one-particle density the GPU returns (G is quadratic in L, so its
    central difference is exact).

Tolerances: |dE| <= 1e-9 Eh; max |R/D| <= 1e-8 (converged to 1e-10 in the
exact-slice arithmetic; a missing or wrong term leaves ~1e-3); finite
difference with step 1e-3: |dg| <= 1e-6 (energy noise ~1e-10 / 1e-3).
"""
import numpy as np
import pytest
import torch

from synth import make_system, make_displacements, unpack_dense
from oracle import model, rows

pytestmark = pytest.mark.gpu

T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


@pytest.fixture(scope="module")
def c2():
    s = make_system(2)
    return s, make_displacements(s, 2)


def _opts(cd):
    o = cd.cdcc_default_options()
    o.precision = cd.PREC_TC
    return o


def _init(cd, s, L):
    return cd.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol, s.orb_irrep,
                           s.eps, s.chol_irrep, L, options=_opts(cd))


def test_c2_tensor_core_schedule_against_oracle(cd, c2):
    s, dL = c2
    o, v = s.nocc, s.nvir
    ctx = _init(cd, s, s.L)
    e, it, res = cd.ccsd_solve(ctx)
    t1 = cd.cdcc_get_amplitudes(ctx, 0, o, v)
    t2 = cd.cdcc_get_amplitudes(ctx, 1, o, v)
    cd.lambda_solve(ctx)
    D = cd.build_density(ctx, s.n)
    g = cd.contract_dL(ctx, dL)
    cd.cd_ccsd_free(ctx)

    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    eref = model.e_ref(h, L, o).item()
    t1t, t2t = T(t1), T(t2)
    del t2
    # energy functional at the GPU amplitudes
    e_or = rows.energy(t1t, t2t, h, L, o) - eref
    assert abs(e - e_or) <= 1e-9, (e, e_or)
    # residual rows: occupied irreps are 0..15, 16..25, 26..33, 34..39
    pairs = [(0, 0), (3, 20), (35, 17), (28, 29)]
    R1, R2 = rows.residual_rows(t1t, t2t, h, L, o, pairs)
    eps = s.eps
    D1 = eps[:o, None] - eps[None, o:]
    assert np.abs(R1.numpy() / D1).max() <= 1e-8
    for (i, j) in pairs:
        Dij = eps[i] + eps[j] - eps[o:, None] - eps[None, o:]
        r = np.abs(R2[(i, j)].numpy() / Dij).max()
        assert r <= 1e-8, ((i, j), r)
    del t2t, R2

    # gradient vs a central difference of the total energy along dL_0
    step = 1e-3
    Ex, Gx = [], []
    for sgn in (1.0, -1.0):
        Lx = s.L + sgn * step * dL[0]
        ctx = _init(cd, s, Lx)
        ec, _, _ = cd.ccsd_solve(ctx)
        cd.cd_ccsd_free(ctx)
        G = model.two_electron_fock(T(unpack_dense(s, Lx)), o).numpy()
        # E_ref = sum_i (h_ii + f_ii) with f = diag(eps) at every L
        Ex.append(ec + float(np.sum(2.0 * eps[:o] - np.diag(G)[:o])))
        Gx.append(G)
    fd = (Ex[0] - Ex[1]) / (2 * step)
    dG = (Gx[0] - Gx[1]) / (2 * step)
    pred = g[0] - float(np.sum(D * dG))
    assert abs(pred - fd) <= 1e-6, (pred, fd)
