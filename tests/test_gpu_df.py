"""The density-fitting / Cholesky three-term gradient (contract_df) on the
GPU: metric factorisation, transformed density and vectors, W matrix and the
two contractions (Sec. 2.1 Eqs. dfcd, cv_2ndstep, eri_cddf_der; Sec. 2.6
Eq. 2el_grad_cont).

  * small C1 and C2v-like systems (one of them with an irrep without
    Cholesky vectors), FP64 schedule: against the oracle's three-term
    gradient (oracle/df.py) from the oracle's own density, |dg| <= 1e-9;
  * the D2h o=16 v=144 nL=640 workload, FP64 and tensor-core schedules:
    against contract_dL of the finite-difference derivative of
    chol(M + x dM)^{-1} (B + x dB) (computed here with numpy), i.e. the
    chain rule through the metric factorisation, |dg| <= 1e-9 (FP64) and
    1e-6 (tensor cores);
  * a metric that is not positive definite is rejected.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

from synth import make_system, random_system, unpack_dense, pack_dense
from synth.df import make_df_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def _gpu(cd, s, M, dB, dM, prec=None, dL=None):
    o = cd.cdcc_default_options()
    o.conv_tol = 1e-12
    o.energy_tol = 1e-13
    if prec is not None:
        o.precision = prec
        o.conv_tol = 1e-10
        o.energy_tol = 1e-12
    ctx = cd.init_from_system(s, options=o)
    cd.ccsd_solve(ctx)
    cd.lambda_solve(ctx)
    cd.build_density(ctx)
    assert cd.cdcc_metric_size(ctx) == M.size
    g = cd.contract_df(ctx, M, dB, dM)
    g2 = cd.contract_dL(ctx, dL) if dL is not None else None
    cd.cd_ccsd_free(ctx)
    return g, g2


@pytest.mark.parametrize("case", ["c0", "sym", "no_chol_irrep"])
def test_contract_df_matches_oracle(cd, case):
    from oracle import model, lagrangian, df
    s = {"c0": lambda: make_system(0),
         "sym": lambda: random_system([3, 2, 2, 1], [7, 5, 4, 3],
                                      [12, 10, 9, 8], seed=221, scale=0.4),
         "no_chol_irrep": lambda: random_system([2, 1, 1, 1], [4, 3, 3, 2],
                                                [7, 0, 6, 5], seed=222,
                                                scale=0.4)}[case]()
    M, _, dB, dM = make_df_inputs(s, 3)
    g, _ = _gpu(cd, s, M, dB, dM)
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
    r = lagrangian.run_all(h, L, s.nocc, tol=1e-12, e_tol=1e-13)
    dBd = torch.as_tensor(np.stack([unpack_dense(s, x) for x in dB]))
    g_or = df.df_gradient(r["G"], L, M, s.chol, dBd,
                          torch.as_tensor(dM)).numpy()
    assert np.abs(g - g_or).max() <= 1e-9, (g, g_or)


def _chain_rule_dL(s, M, dB, dM):
    """d/dx [chol(M + x dM)^{-1} (B + x dB)] with B = K L (packed), central
    differences with Richardson extrapolation."""
    Ld = unpack_dense(s, s.L)
    B = np.zeros_like(Ld)
    P0, off = 0, 0
    blocks = []
    for n in s.chol:
        K = np.linalg.cholesky(M[off:off + n * n].reshape(n, n))
        B[P0:P0 + n] = (K @ Ld[P0:P0 + n].reshape(n, -1)).reshape(
            n, *Ld.shape[1:])
        blocks.append((P0, off, n))
        P0 += n
        off += n * n

    def vec(Mx, Bx):
        out = np.zeros_like(Bx)
        for P0, off, n in blocks:
            K = np.linalg.cholesky(Mx[off:off + n * n].reshape(n, n))
            out[P0:P0 + n] = scipy.linalg.solve_triangular(
                K, Bx[P0:P0 + n].reshape(n, -1), lower=True).reshape(
                    n, *Bx.shape[1:])
        return out
    res = []
    for x in range(dB.shape[0]):
        dBx = unpack_dense(s, dB[x])
        fd = []
        for st in (1e-3, 5e-4):
            fd.append((vec(M + st * dM[x], B + st * dBx)
                       - vec(M - st * dM[x], B - st * dBx)) / (2 * st))
        res.append(pack_dense(s, (4.0 * fd[1] - fd[0]) / 3.0))
    return np.stack(res)


@pytest.mark.parametrize("prec", ["fp64", "tc"])
def test_contract_df_chain_rule_d2h_workload(cd, prec):
    s = make_system(1)
    M, _, dB, dM = make_df_inputs(s, 3)
    dL = _chain_rule_dL(s, M, dB, dM)
    p = cd.PREC_TC if prec == "tc" else None
    g, g_dl = _gpu(cd, s, M, dB, dM, prec=p, dL=dL)
    tol = 1e-6 if prec == "tc" else 1e-9
    assert np.abs(g - g_dl).max() <= tol, (g, g_dl)


def test_contract_df_rejects_indefinite_metric(cd):
    s = random_system([2, 1], [5, 4], [8, 6], seed=223, scale=0.4)
    M, _, dB, dM = make_df_inputs(s, 1)
    M = M.copy()
    M[0] = -1.0                     # first diagonal element negative
    o = cd.cdcc_default_options()
    ctx = cd.init_from_system(s, options=o)
    cd.ccsd_solve(ctx)
    cd.lambda_solve(ctx)
    cd.build_density(ctx)
    with pytest.raises(cd.CdccError) as ei:
        cd.contract_df(ctx, M, dB, dM)
    assert ei.value.status == cd.CDCC_EINVAL
    # the context stays usable
    g = cd.contract_df(ctx, make_df_inputs(s, 1)[0], dB, dM)
    assert np.all(np.isfinite(g))
    cd.cd_ccsd_free(ctx)
