"""Pins of the two-step Cholesky decomposition oracle (oracle/cd.py,
Sec. 3.2, Algorithm 1 and eq. cv_2ndstep) against what the mathematics
fixes (CPU only):

  * sigma = 1, Q_max = 1 is the textbook pivoted Cholesky decomposition:
    the pivots and vectors of LAPACK's dpstrf;
  * every residual |(r|s) - sum_P L^P_r L^P_s| stays below tau (the
    residual matrix is positive semidefinite and its diagonal below tau);
  * a matrix of exact rank k per irrep gives k vectors per irrep and
    reproduces the matrix;
  * the symmetry-blocked decomposition equals the one of the same matrix
    with the irrep labels dropped;
  * the second-step vectors reproduce the Nystrom form M[:, Q] V^-1 M[Q, :]
    from numpy's general solver and equal the first-step vectors;
  * a planted mistake (a wrong diagonal) is caught.
"""
import numpy as np
import pytest
import scipy.linalg.lapack as lapack

from synth.cd import make_cd_system, as_c1
from oracle import cd


def _blocks(s):
    return [s.block(g) for g in range(s.nirrep)]


def _full(B):
    return B @ B.T


def test_pivoted_cholesky_limit_matches_dpstrf():
    s = make_cd_system(14, 1, 40, seed=11)
    B = s.block(0)
    M = _full(B)
    tau = 1e-7
    piv, L, _, info = cd.first_step([B], tau, sigma=1.0, qmax=1)
    c, perm, rank, err = lapack.dpstrf(M, tol=tau, lower=1)
    assert err in (0, 1)
    perm = perm - 1                             # full row permutation
    assert piv[0] == list(perm[:rank]), (piv[0][:10], list(perm[:10]))
    Lc = np.tril(c)[:, :rank]                   # rows in pivot order
    ours = L[0].T[perm]                         # same row order
    assert np.abs(ours - Lc).max() <= 1e-10 * np.abs(M).max()
    assert info["macro"] == rank


@pytest.mark.parametrize("qmax,sigma", [(1000, 1e-2), (7, 1e-2), (3, 0.3)])
def test_residual_below_tau(qmax, sigma):
    s = make_cd_system(24, 8, 30, seed=5)
    tau = 1e-5
    blocks = _blocks(s)
    piv, L1, _, info = cd.first_step(blocks, tau, sigma=sigma, qmax=qmax)
    L2 = cd.second_step(blocks, piv)
    assert info["macro"] >= 1
    for g, B in enumerate(blocks):
        if B.shape[0] == 0:
            continue
        M = _full(B)
        for L in (L1[g], L2[g]):
            R = M - L.T @ L
            assert np.diag(R).max() < tau * (1 + 1e-9)
            assert np.abs(R).max() <= tau * (1 + 1e-9)
        assert len(set(piv[g])) == len(piv[g])


def test_exact_rank_is_found_and_reproduced():
    s = make_cd_system(20, 4, 5, seed=7, decay=0.0)
    blocks = _blocks(s)
    piv, L2, _ = cd.two_step(s, 1e-10)
    for g, B in enumerate(blocks):
        M = _full(B)
        assert len(piv[g]) == min(5, B.shape[0])
        assert np.abs(M - L2[g].T @ L2[g]).max() <= 1e-10 * np.abs(M).max()


def test_symmetry_blocked_equals_c1():
    s = make_cd_system(16, 4, 12, seed=3)
    c1 = as_c1(s)
    tau = 1e-6
    piv, L, _ = cd.two_step(s, tau, sigma=1.0, qmax=1)
    piv1, L1, _ = cd.two_step(c1, tau, sigma=1.0, qmax=1)
    offs = np.cumsum([0] + s.npair)
    blocked = sorted(int(offs[g] + q) for g in range(s.nirrep)
                     for q in piv[g])
    assert blocked == sorted(piv1[0])
    # same approximation of the same matrix
    M1 = np.zeros((offs[-1], offs[-1]))
    for g in range(s.nirrep):
        a, b = offs[g], offs[g + 1]
        M1[a:b, a:b] = L[g].T @ L[g]
    assert np.abs(M1 - L1[0].T @ L1[0]).max() <= 1e-11


def test_second_step_is_nystrom_and_equals_first_step():
    s = make_cd_system(18, 2, 25, seed=9)
    blocks = _blocks(s)
    piv, L1, _, _ = cd.first_step(blocks, 1e-6, sigma=1e-2, qmax=5)
    L2 = cd.second_step(blocks, piv)
    for g, B in enumerate(blocks):
        M = _full(B)
        q = np.array(piv[g])
        ny = M[:, q] @ np.linalg.solve(M[np.ix_(q, q)], M[q, :])
        assert np.abs(L2[g].T @ L2[g] - ny).max() <= 1e-10 * np.abs(M).max()
        assert np.abs(L2[g] - L1[g]).max() <= 1e-9 * np.sqrt(np.abs(M).max())


def test_planted_mistake_is_caught(monkeypatch):
    s = make_cd_system(24, 8, 30, seed=5)
    good = cd.diagonal
    monkeypatch.setattr(cd, "diagonal", lambda B: 1.01 * good(B))
    blocks = _blocks(s)
    piv, L, _, _ = cd.first_step(blocks, 1e-5, qmax=7)
    worst = max(np.abs(_full(B) - L[g].T @ L[g]).max()
                for g, B in enumerate(blocks) if B.shape[0])
    assert worst > 1e-5
