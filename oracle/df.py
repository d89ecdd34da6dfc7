"""Gradient in the density-fitting / Cholesky three-term form (oracle).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Sec. 2.1 writes the
Cholesky vectors through a metric: with three-index integrals B^R_pq =
(R|pq) and the metric M_PQ = (P|Q) = (K K^T)_PQ (K its Cholesky factor),
Eq. dfcd / Eq. cv_2ndstep give L^P = sum_R K^{-1}_PR B^R, and Eq.
eri_cddf_der writes the integral derivative with the transformed vectors
Ltilde = K^{-T} L as
    (pq|rs)^x = sum_P B^{x,P}_pq Ltilde^P_rs + sum_P Ltilde^P_pq B^{x,P}_rs
                - sum_PQ Ltilde^P_pq M^x_PQ Ltilde^Q_rs.
Contracted with the two-particle density (Sec. 2.6, Eq. 2el_grad_cont) this
is the three-term gradient
    dE/dx = sum_P <Jt^P, B^{x,P}> - sum_PQ W_PQ M^x_PQ,
    Jt^P = sum_Q (K^{-T})_PQ Gamma^Q,   W_PQ = 1/2 sum_pq Ltilde^P_pq Jt^Q_pq,
where Gamma^P_pq = dLag/dL^P_pq is the Cholesky-basis density of
oracle/lagrangian.py (twice the paper's Gamma^P_pr of Eq. d2xtl1 summed
with its Gammabar, J^P = 1/2 Jt^P; the two paper terms with J and Jbar are
equal here because Gamma^P is symmetrised in pq).  The metric is block
diagonal by the irrep of the Cholesky vectors (Sec. 3.1).

Steps follow the paper: Cholesky factor of each metric block, triangular
solves for Ltilde and Jt, the W matrix, then the two contractions.  Pinned
(tests/test_oracle_pins.py) against the differentiated-vector form
<Gamma, dL/dx> with dL/dx a central finite difference of
chol(M + x dM)^{-1} (B + x dB), and against a finite difference of the
CCSD energy in x.
"""
from __future__ import annotations

import torch

from .model import DT


def metric_blocks(M, chol):
    """Packed metric -> list of dense (n, n) blocks, one per irrep."""
    out, off = [], 0
    M = torch.as_tensor(M, dtype=DT)
    for n in chol:
        out.append(M[off:off + n * n].reshape(n, n))
        off += n * n
    return out


def transformed(X, M_blocks, chol):
    """K^{-T} X over the Cholesky index of a dense (nchol, n, n) array,
    irrep block by irrep block (K the Cholesky factor of each block)."""
    Y = torch.zeros_like(X)
    P0 = 0
    for Mb, n in zip(M_blocks, chol):
        if n == 0:
            continue
        K = torch.linalg.cholesky(Mb)
        rhs = X[P0:P0 + n].reshape(n, -1)
        Y[P0:P0 + n] = torch.linalg.solve_triangular(
            K.T, rhs, upper=True).reshape(n, *X.shape[1:])
        P0 += n
    return Y


def df_gradient(G, L, M, chol, dB, dM):
    """Three-term gradient g_x for each displacement.
    G, L: dense (nchol, n, n); M: packed metric; dB: (nx, nchol, n, n)
    dense; dM: (nx, metric size) packed."""
    Mb = metric_blocks(M, chol)
    Lt = transformed(torch.as_tensor(L, dtype=DT), Mb, chol)
    Jt = transformed(torch.as_tensor(G, dtype=DT), Mb, chol)
    dB = torch.as_tensor(dB, dtype=DT)
    dM = torch.as_tensor(dM, dtype=DT)
    g = torch.einsum("Ppq,xPpq->x", Jt, dB)
    P0, off = 0, 0
    for n in chol:
        if n == 0:
            continue
        W = 0.5 * Lt[P0:P0 + n].reshape(n, -1) @ Jt[P0:P0 + n].reshape(n, -1).T
        g = g - torch.einsum("PQ,xPQ->x", W,
                             dM[:, off:off + n * n].reshape(-1, n, n))
        P0 += n
        off += n * n
    return g
