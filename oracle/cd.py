"""Oracle: symmetry-adapted two-step Cholesky decomposition of the ERI
matrix (Sec. 3.2, Algorithm 1, and the second step, eq. cv_2ndstep).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this module; the library never does.

Plain numpy in FP64, the steps in the paper's order.  The integral source
is the synthetic factored matrix of synth/cd.py: (r|s) = B_G[r] . B_G[s]
for pairs r, s of irrep G (zero across irreps); integrals are evaluated
from that definition whenever a step needs them, one column per pivot
candidate (the synthetic integrals have no shell structure, so a "shell
quartet" is a single pair column).

First step (Cholesky basis).  Pairs whose diagonal (r|r) reaches tau form
the list P.  Each macro iteration takes, over all irreps, the at most
Q_max largest diagonals of P that reach sigma * D_max (D_max the largest
diagonal of P), evaluates the columns (t|u) of these candidates u for all
t of the same irrep and subtracts the vectors found so far,
M~_tu = (t|u) - sum_p L^p_t L^p_u.  Micro iterations then pivot, inside
the candidate set, on the largest current diagonal q while it reaches
tau_mic = max(tau, sigma * D_max) (each pair is a pivot at most
once): the new vector is
L^q_r = (M~_rq - sum over this macro iteration's earlier vectors
L^p_r L^p_q) / sqrt(D_q) for every r of q's irrep, and D_r -= (L^q_r)^2.
The new vectors join the irrep's list, and pairs whose diagonal fell below
tau leave P.  The loop ends when P is empty.  (tau_mic is not defined in
the paper's text; the reading max(tau, sigma * D_max) is the span-factor
rule of the two-step method the paper follows.)

Second step.  With the pivots q of irrep G as the Cholesky basis, the
metric V_G = (Q|R) is factored V = K K^T and the vectors are
L^P_rs = sum_R (K^-1)_PR (R|rs) for every pair rs of G.

Pinned in tests/test_oracle_cd.py: with sigma = 1 and Q_max = 1 the
first step is the textbook pivoted Cholesky decomposition and picks the
pivots of LAPACK's dpstrf; every residual |(r|s) - sum L_r L_s| stays
below tau; a matrix of exact rank k gives k vectors per irrep and
reproduces it; the symmetry-blocked decomposition equals the one of the
same matrix with the irrep labels dropped; the second-step vectors
reproduce the Nystrom form M[:, Q] V^-1 M[Q, :] of numpy's solver.
"""
from __future__ import annotations

import numpy as np


def integral_columns(Bg: np.ndarray, cols) -> np.ndarray:
    """(t|u) for all pairs t of one irrep and the pairs u in cols."""
    return Bg @ Bg[np.asarray(cols, dtype=np.int64)].T


def diagonal(Bg: np.ndarray) -> np.ndarray:
    """(r|r) for every pair r of one irrep."""
    return np.einsum("rk,rk->r", Bg, Bg)


def first_step(blocks, tau: float, sigma: float = 1e-2, qmax: int = 1000,
               max_macro: int = 100000):
    """Cholesky basis of the block-diagonal matrix with factors
    blocks[G] (npair(G) x naux(G)).  Returns (pivots, vectors, diag, info):
    pivots[G] the pivot pairs of irrep G in the order they were taken,
    vectors[G] their first-step vectors (ncv(G) x npair(G), every row
    filled), diag[G] the final updated diagonals, info the number of macro
    and micro iterations."""
    h = len(blocks)
    D = [diagonal(B) for B in blocks]
    # list P: pairs whose diagonal reaches tau (per irrep, a mask)
    P = [D[g] >= tau for g in range(h)]
    L = [np.zeros((0, blocks[g].shape[0])) for g in range(h)]
    piv = [[] for _ in range(h)]
    # a pair is a pivot at most once (exactly: its diagonal is then 0)
    taken = [np.zeros(blocks[g].shape[0], bool) for g in range(h)]
    n_macro = n_micro = 0
    while any(P[g].any() for g in range(h)):
        n_macro += 1
        if n_macro > max_macro:
            raise RuntimeError("two-step CD: no progress")
        dmax = max(D[g][P[g]].max() for g in range(h) if P[g].any())
        # qualified candidates over all irreps: the Q_max largest diagonals
        # of P that reach sigma * D_max (ties: lower irrep, lower pair)
        cand = [(D[g][r], g, r) for g in range(h)
                for r in np.nonzero(P[g])[0] if D[g][r] >= sigma * dmax]
        cand.sort(key=lambda c: (-c[0], c[1], c[2]))
        cand = cand[:qmax]
        Q = [[r for (_, gg, r) in cand if gg == g] for g in range(h)]
        # columns of the candidates minus the vectors found so far
        Mt = []
        for g in range(h):
            if not Q[g]:
                Mt.append(None)
                continue
            M = integral_columns(blocks[g], Q[g])
            if L[g].shape[0]:
                M = M - L[g].T @ L[g][:, Q[g]]
            Mt.append(M)
        # micro iterations inside the candidate set
        tau_mic = max(tau, sigma * dmax)
        Lmic = [[] for _ in range(h)]
        while True:
            best = None
            for g in range(h):
                for j, r in enumerate(Q[g]):
                    if not taken[g][r] and (best is None or D[g][r] > best[0]):
                        best = (D[g][r], g, j)
            if best is None or best[0] < tau_mic:
                break
            dq, g, j = best
            q = Q[g][j]
            col = Mt[g][:, j].copy()
            for v in Lmic[g]:
                col -= v * v[q]
            lq = col / np.sqrt(dq)
            D[g] = D[g] - lq * lq
            Lmic[g].append(lq)
            piv[g].append(int(q))
            taken[g][q] = True
            n_micro += 1
        for g in range(h):
            if Lmic[g]:
                L[g] = np.vstack([L[g], np.array(Lmic[g])])
            # pairs whose diagonal fell below tau (and the pivots) leave P
            P[g] &= (D[g] >= tau) & ~taken[g]
    return piv, L, D, dict(macro=n_macro, micro=n_micro)


def second_step(blocks, pivots):
    """Vectors L^P_rs = sum_R (K^-1)_PR (R|rs) with V = K K^T the metric of
    the pivots of each irrep (eq. cv_2ndstep)."""
    out = []
    for g, B in enumerate(blocks):
        q = np.asarray(pivots[g], dtype=np.int64)
        if q.size == 0:
            out.append(np.zeros((0, B.shape[0])))
            continue
        V = integral_columns(B[q], np.arange(q.size))      # (Q|R)
        K = np.linalg.cholesky(V)
        C = integral_columns(B, q).T                        # (R|rs)
        out.append(np.linalg.solve(K, C))                   # K^-1 (R|rs)
    return out


def two_step(sysm, tau: float, sigma: float = 1e-2, qmax: int = 1000):
    """Both steps on a synth.cd.CdSystem: (pivots, vectors, info)."""
    blocks = [sysm.block(g) for g in range(sysm.nirrep)]
    piv, _, _, info = first_step(blocks, tau, sigma, qmax)
    return piv, second_step(blocks, piv), info
