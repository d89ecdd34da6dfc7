"""Symmetry-adapted two-step Cholesky decomposition on the GPU
(cdcc_cd_two_step; Sec. 3.2, Algorithm 1, Eq. cv_2ndstep) against the
oracle (oracle/cd.py) on the same seeded synthetic factored matrices:

  * pivots: the same pairs in the same order per irrep (an integer
    decision both sides take in FP64), and the same numbers of macro and
    micro iterations;
  * vectors: the second-step vectors element by element, |dL| <= 1e-9
    sqrt(max |(r|s)|);
  * properties at sizes the oracle does not run: every residual
    |(r|s) - sum_P L^P_r L^P_s| below tau (full blocks, or sampled rows of
    the largest case), the metric identity L[:, Q] = K^T (upper triangular
    with a positive diagonal on the pivots);
  * edge cases: irreps without pairs, an irrep without factor columns,
    tau above every diagonal (no vectors), device-resident B.
"""
import numpy as np
import pytest
import torch

from synth.cd import make_cd_system
from oracle import cd as ocd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cdc():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def _run(cdc, s, tau, sigma, qmax, B=None):
    return cdc.cd_two_step(s.npair, s.naux, s.B if B is None else B, tau,
                           sigma=sigma, qmax=qmax)


CASES = [
    # nbasis, nirrep, naux, seed, tau, sigma, qmax
    (14, 1, 40, 11, 1e-7, 1.0, 1),       # textbook pivoted Cholesky
    (24, 8, 30, 5, 1e-5, 1e-2, 1000),    # one macro iteration per batch
    (24, 8, 30, 5, 1e-5, 1e-2, 7),       # many small batches
    (40, 4, 60, 17, 1e-6, 0.3, 25),
    (36, 2, 90, 23, 1e-8, 1e-2, 1000),
]


@pytest.mark.parametrize("nb,h,naux,seed,tau,sigma,qmax", CASES)
def test_matches_oracle(cdc, nb, h, naux, seed, tau, sigma, qmax):
    s = make_cd_system(nb, h, naux, seed=seed)
    blocks = [s.block(g) for g in range(h)]
    piv_o, _, _, info = ocd.first_step(blocks, tau, sigma, qmax)
    L_o = ocd.second_step(blocks, piv_o)
    piv, L, stats = _run(cdc, s, tau, sigma, qmax)
    assert piv == piv_o
    assert (int(stats[0]), int(stats[1])) == (info["macro"], info["micro"])
    for g, B in enumerate(blocks):
        if B.shape[0] == 0:
            continue
        scale = np.sqrt(np.abs(B @ B.T).max())
        assert L[g].shape == L_o[g].shape
        if L[g].size:
            assert np.abs(L[g] - L_o[g]).max() <= 1e-9 * scale, g


def test_residual_and_metric_identity_at_a_larger_size(cdc):
    s = make_cd_system(120, 8, 150, seed=31)
    tau = 1e-6
    piv, L, stats = _run(cdc, s, tau, 1e-2, 1000)
    assert sum(len(p) for p in piv) > 0
    for g in range(s.nirrep):
        B = s.block(g)
        if B.shape[0] == 0:
            continue
        M = B @ B.T
        R = M - L[g].T @ L[g]
        assert np.abs(R).max() <= tau * (1 + 1e-8), g
        q = np.array(piv[g])
        if q.size:
            Kt = L[g][:, q]                    # = K^T
            assert np.abs(np.tril(Kt, -1)).max() <= 1e-10 * np.sqrt(M.max())
            assert (np.diag(Kt) > 0).all()


def test_paper_sized_case_sampled_rows(cdc):
    # 678 basis functions in D2h (the hexabenzocoronene basis size of the
    # paper's first test; tau = 1e-4 keeps 3770 vectors, the paper reports
    # 3710): the residual on sampled rows, evaluated from the factor
    s = make_cd_system(678, 8, 600, seed=41, decay=19.5)
    tau = 1e-4
    piv, L, stats = _run(cdc, s, tau, 1e-2, 1000)
    rng = np.random.default_rng(0)
    for g in range(s.nirrep):
        B = s.block(g)
        rows = rng.choice(B.shape[0], 16, replace=False)
        R = B[rows] @ B.T - L[g][:, rows].T @ L[g]
        assert np.abs(R).max() <= tau * (1 + 1e-8), g
        assert len(set(piv[g])) == len(piv[g])


def test_edge_cases(cdc):
    # nbasis 3 in D2h: irreps without pairs
    s = make_cd_system(3, 8, 4, seed=2)
    assert 0 in s.npair
    piv, L, _ = _run(cdc, s, 1e-8, 1e-2, 1000)
    piv_o, L_o, _ = ocd.two_step(s, 1e-8)
    assert piv == piv_o
    # tau above every diagonal: no vectors
    s = make_cd_system(20, 4, 10, seed=4)
    piv, L, stats = _run(cdc, s, 1e6, 1e-2, 1000)
    assert all(len(p) == 0 for p in piv) and stats[0] == 0
    # an irrep without factor columns (zero block) next to the others
    s = make_cd_system(20, 2, 10, seed=6)
    s.naux[1] = 0
    s.B = s.B[:s.npair[0] * s.naux[0]]
    piv, L, _ = _run(cdc, s, 1e-8, 1e-2, 1000)
    assert len(piv[1]) == 0 and len(piv[0]) == 10
    # device-resident B gives the same result
    s = make_cd_system(24, 8, 30, seed=5)
    a = _run(cdc, s, 1e-5, 1e-2, 7)
    b = _run(cdc, s, 1e-5, 1e-2, 7, B=torch.as_tensor(s.B, device="cuda"))
    assert a[0] == b[0]
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
