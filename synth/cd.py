"""Seeded inputs of the two-step Cholesky decomposition of the ERI matrix.

A synthetic "AO basis" of n functions with irrep labels; the basis pairs
r = (mu, nu), mu >= nu, carry the irrep of mu x nu.  The two-electron
integral matrix (r|s) of the pairs is block diagonal by that irrep, and
block G is drawn in factored form

    (r|s) = sum_k B_G[r, k] B_G[s, k],      B_G: npair(G) x naux(G),

which makes it symmetric positive semidefinite, as the ERI matrix is.
B_G[r, k] = g_r w_k z_rk with z ~ N(0, 1), pair magnitudes g_r spread over
orders of magnitude (like the diagonal of real integrals) and column
weights w_k decaying geometrically (a decaying spectrum, so that a
threshold tau keeps a number of vectors that grows with the basis).

This module only draws and lays out numbers: the integrals themselves are
formed by whoever evaluates them (the oracle, the library), from B.

Layout: the pairs of each irrep are numbered in the order nu = 0, 1, ...
and inside it mu = nu, nu + 1, ... (mu >= nu); B holds the irrep blocks
back to back, each row-major (npair(G) rows of naux(G) columns).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CdSystem:
    name: str
    nirrep: int
    orb_irrep: np.ndarray           # (nbasis,)
    pairs: list                     # per irrep: (npair_G, 2) int array
    npair: list                     # per irrep
    naux: list                      # per irrep
    B: np.ndarray                   # packed, blocks back to back
    seed: int

    def block(self, g: int) -> np.ndarray:
        off = sum(self.npair[h] * self.naux[h] for h in range(g))
        n, k = self.npair[g], self.naux[g]
        return self.B[off:off + n * k].reshape(n, k)


def make_cd_system(nbasis: int, nirrep: int, naux: int, seed: int,
                   spread: float = 6.0, decay: float = 9.0,
                   name: str = "") -> CdSystem:
    """nbasis functions spread evenly over nirrep irreps (largest-remainder
    split), naux factor columns per irrep; pair magnitudes g_r =
    exp(-spread * u_r / 2) with u ~ U(0, 1); column weights
    w_k = exp(-decay * k / (2 naux))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = [nbasis // nirrep] * nirrep
    for g in range(nbasis - sum(base)):
        base[g] += 1
    orb = np.concatenate([np.full(n, g, np.int32) for g, n in enumerate(base)])
    rng.shuffle(orb)
    pair_lists = [[] for _ in range(nirrep)]
    for nu in range(nbasis):
        for mu in range(nu, nbasis):
            pair_lists[orb[mu] ^ orb[nu]].append((mu, nu))
    pairs = [np.array(p, dtype=np.int32).reshape(-1, 2) for p in pair_lists]
    npair = [len(p) for p in pairs]
    nax = [naux if npair[g] > 0 else 0 for g in range(nirrep)]
    w = np.exp(-decay * np.arange(naux) / (2.0 * naux))
    blocks = []
    for g in range(nirrep):
        n = npair[g]
        gr = np.exp(-spread * rng.uniform(0.0, 1.0, n) / 2.0)
        z = rng.standard_normal((n, nax[g]))
        blocks.append((gr[:, None] * w[None, :nax[g]] * z).reshape(-1))
    B = np.concatenate(blocks) if blocks else np.zeros(0)
    return CdSystem(name or f"cd n={nbasis} h={nirrep} naux={naux}", nirrep,
                    orb, pairs, npair, nax, B, seed)


def as_c1(s: CdSystem) -> CdSystem:
    """The same integral matrix with every irrep label dropped: one block,
    the blocks' pairs stacked in irrep order, B block diagonal (columns of
    block G placed after those of the blocks before it)."""
    n = sum(s.npair)
    k = sum(s.naux)
    B = np.zeros((n, k))
    r0 = c0 = 0
    for g in range(s.nirrep):
        B[r0:r0 + s.npair[g], c0:c0 + s.naux[g]] = s.block(g)
        r0 += s.npair[g]
        c0 += s.naux[g]
    pairs = [np.concatenate(s.pairs, axis=0)] if n else [np.zeros((0, 2))]
    return CdSystem(s.name + " (C1)", 1, np.zeros_like(s.orb_irrep), pairs,
                    [n], [k], B.reshape(-1), s.seed)
