"""Seeded inputs of the density-fitting (DF) form of a workload.

In the DF/CD-equivalent form the Cholesky vectors are L = K^{-1} B with
B^R_pq = (R|pq) three-index integrals and K the Cholesky factor of the
metric M_PQ = (P|Q) (block diagonal by the irrep of P).  A displacement
changes B and M.  This module draws, for a workload whose L is given, a
metric M = K K^T from a drawn lower-triangular K with positive diagonal
(the usual way to draw a well-conditioned symmetric positive definite
matrix), and the displacement derivatives dB (with L's block pattern) and
dM (symmetric per irrep block).  It computes none of the method's
arithmetic: B itself is never formed here.

Packed metric layout: for each irrep G of the Cholesky vectors, the
nchol(G) x nchol(G) block, row-major, blocks back to back.
"""
from __future__ import annotations

import numpy as np

from .gen import System, _draw_symmetric_pattern


def metric_size(sysm: System) -> int:
    return int(sum(n * n for n in sysm.chol))


def make_df_inputs(sysm: System, nx: int = 2, sigma: float = 0.05,
                   sigma_m: float = 0.05):
    """(M, K, dB, dM): packed metric, its drawn factor (for pins only),
    nx packed three-index derivatives and nx packed metric derivatives."""
    rng = np.random.Generator(np.random.PCG64(sysm.seed + 52711))
    Ms, Ks = [], []
    for n in sysm.chol:
        K = np.tril(rng.standard_normal((n, n)) * (0.2 / np.sqrt(max(n, 1))),
                    -1)
        K[np.diag_indices(n)] = rng.uniform(0.8, 1.2, n)
        Ks.append(K.reshape(-1))
        Ms.append((K @ K.T).reshape(-1))
    M = np.concatenate(Ms) if Ms else np.zeros(0)
    Kp = np.concatenate(Ks) if Ks else np.zeros(0)
    norb = sysm.norb_irrep()

    def amp_of(gP, nP):
        return np.full(nP, sigma * sysm.scale)

    dB = np.stack([_draw_symmetric_pattern(rng, sysm.nirrep, norb, sysm.chol,
                                           amp_of) for _ in range(nx)])
    dM = np.zeros((nx, M.size))
    for x in range(nx):
        parts = []
        for n in sysm.chol:
            X = rng.standard_normal((n, n)) * sigma_m
            parts.append((0.5 * (X + X.T)).reshape(-1))
        dM[x] = np.concatenate(parts) if parts else np.zeros(0)
    return M, Kp, dB, dM
