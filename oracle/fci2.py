"""Exact two-electron singlet FCI (pin for o = 1).

For two electrons CCSD is exact.  The singlet wavefunction is
Psi = sum_pq C_pq phi_p(1) phi_q(2) x (singlet spin), C symmetric,
sum_pq C_pq^2 = 1, and
    (H C)_pq = sum_r h_pr C_rq + sum_r C_pr h_rq + sum_rs (pr|qs) C_rs ,
    (pr|qs) = sum_P L^P_pr L^P_qs  (Sec. 2.1, Eq. 1).
The root returned is the lowest singlet.  With h held fixed, Hellmann-Feynman
gives the exact derivative along dL (Eq. 2 for the ERI derivative):
    dE/dx = 2 sum_P tr(dL^P C L^P C).
"""
from __future__ import annotations

import numpy as np


def singlet_fci(h: np.ndarray, L: np.ndarray):
    n = h.shape[0]
    g = np.einsum("Ppr,Pqs->pqrs", L, L)      # index [p,q,r,s] = (pr|qs)
    eye = np.eye(n)
    M = (np.einsum("pr,qs->pqrs", h, eye) + np.einsum("pr,qs->pqrs", eye, h)
         + g).reshape(n * n, n * n)
    # orthonormal basis of symmetric C
    cols = []
    for p in range(n):
        for q in range(p, n):
            c = np.zeros((n, n))
            if p == q:
                c[p, p] = 1.0
            else:
                c[p, q] = c[q, p] = 1.0 / np.sqrt(2.0)
            cols.append(c.reshape(-1))
    B = np.array(cols).T
    Ms = B.T @ M @ B
    w, V = np.linalg.eigh(0.5 * (Ms + Ms.T))
    C = (B @ V[:, 0]).reshape(n, n)
    if C[0, 0] < 0:
        C = -C
    return w[0], C


def hellmann_feynman(C: np.ndarray, L: np.ndarray, dL: np.ndarray):
    """dE/dx = 2 sum_P tr(dL^P C L^P C) for each displacement in dL."""
    return np.array([2.0 * sum(np.trace(dLx[P] @ C @ L[P] @ C)
                               for P in range(L.shape[0])) for dLx in dL])
