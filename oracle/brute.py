"""Brute-force coupled-cluster projections in a determinant basis (pin).

The CCSD equations are the projections  <mu| exp(-T) H exp(T) |0> = 0
(standard CC theory; Sec. 2.2 writes the Lagrangian in these terms).  This
module evaluates them literally for tiny systems: the Hamiltonian and the
spin-free excitation operators E_pq = a+_{p alpha} a_{q alpha} + a+_{p beta} a_{q beta}
are built as matrices on all determinants with 2*nocc electrons, T is the
closed-shell cluster operator
    T = sum_ia t1[i,a] E_ai + 1/2 sum_ijab t2[i,j,a,b] E_ai E_bj,
and exp(+-T) is the terminating power series.  Cost grows exponentially; use
n <= 6 spatial orbitals.

Spin orbital 2p is p alpha, 2p+1 is p beta.  Creation/annihilation signs use
the Jordan-Wigner ordering of spin orbitals.
"""
from __future__ import annotations

from itertools import combinations
import numpy as np


def _parity_below(bits: int, k: int) -> int:
    return bin(bits & ((1 << k) - 1)).count("1") & 1


class DeterminantSpace:
    def __init__(self, nspatial: int, nelec: int):
        self.n = nspatial
        self.nso = 2 * nspatial
        self.dets = [sum(1 << k for k in c)
                     for c in combinations(range(self.nso), nelec)]
        self.index = {d: i for i, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self._exc = {}

    def spin_exc(self, p: int, q: int, spin: int) -> np.ndarray:
        """Matrix of a+_{p,spin} a_{q,spin} on this space."""
        key = (p, q, spin)
        if key in self._exc:
            return self._exc[key]
        P, Q = 2 * p + spin, 2 * q + spin
        M = np.zeros((self.dim, self.dim))
        for col, d in enumerate(self.dets):
            if not (d >> Q) & 1:
                continue
            s = _parity_below(d, Q)
            d1 = d ^ (1 << Q)
            if (d1 >> P) & 1:
                continue
            s ^= _parity_below(d1, P)
            d2 = d1 | (1 << P)
            M[self.index[d2], col] += -1.0 if s else 1.0
        self._exc[key] = M
        return M

    def E(self, p: int, q: int) -> np.ndarray:
        return self.spin_exc(p, q, 0) + self.spin_exc(p, q, 1)

    def hf(self, nocc: int) -> np.ndarray:
        d = sum(1 << (2 * p + s) for p in range(nocc) for s in (0, 1))
        v = np.zeros(self.dim)
        v[self.index[d]] = 1.0
        return v


def hamiltonian(space: DeterminantSpace, h: np.ndarray, L: np.ndarray):
    """H = sum h_pq E_pq + 1/2 sum (pq|rs) (E_pq E_rs - delta_qr E_ps) with
    (pq|rs) = sum_P L^P_pq L^P_rs (Eq. 1)."""
    n = space.n
    Es = [[space.E(p, q) for q in range(n)] for p in range(n)]
    H = np.zeros((space.dim, space.dim))
    for p in range(n):
        for q in range(n):
            if h[p, q] != 0.0:
                H += h[p, q] * Es[p][q]
    for P in range(L.shape[0]):
        O = np.zeros_like(H)
        for p in range(n):
            for q in range(n):
                if L[P, p, q] != 0.0:
                    O += L[P, p, q] * Es[p][q]
        H += 0.5 * O @ O
    K = np.einsum("Ppq,Pqs->ps", L, L)
    for p in range(n):
        for s in range(n):
            if K[p, s] != 0.0:
                H -= 0.5 * K[p, s] * Es[p][s]
    return H


def cluster_operator(space, t1, t2, nocc):
    o, v = t1.shape
    T = np.zeros((space.dim, space.dim))
    for i in range(o):
        for a in range(v):
            if t1[i, a] != 0.0:
                T += t1[i, a] * space.E(nocc + a, i)
    Eai = {(a, i): space.E(nocc + a, i) for a in range(v) for i in range(o)}
    for i in range(o):
        for j in range(o):
            for a in range(v):
                for b in range(v):
                    c = t2[i, j, a, b]
                    if c != 0.0:
                        T += 0.5 * c * (Eai[(a, i)] @ Eai[(b, j)])
    return T


def _exp_apply(T, vec, sign=1.0, kmax=64):
    out = vec.copy()
    term = vec.copy()
    for k in range(1, kmax):
        term = sign * (T @ term) / k
        if not np.any(term):
            break
        out += term
    return out


def projections(h, L, nocc, t1, t2):
    """Return (E_total, R1[i,a], R2[i,j,a,b]) by literal projection."""
    n = h.shape[0]
    space = DeterminantSpace(n, 2 * nocc)
    H = hamiltonian(space, h, L)
    T = cluster_operator(space, t1, t2, nocc)
    ref = space.hf(nocc)
    u = _exp_apply(T, H @ _exp_apply(T, ref, 1.0), -1.0)
    o, v = nocc, n - nocc
    R1 = np.zeros((o, v))
    R2 = np.zeros((o, o, v, v))
    for i in range(o):
        for a in range(v):
            phi = space.spin_exc(o + a, i, 0) @ ref
            R1[i, a] = phi @ u
    for i in range(o):
        for j in range(o):
            for a in range(v):
                for b in range(v):
                    phi = space.spin_exc(o + a, i, 0) @ (
                        space.spin_exc(o + b, j, 1) @ ref)
                    R2[i, j, a, b] = phi @ u
    return ref @ u, R1, R2


def fci_ground_energy(h, L, nocc):
    """Lowest eigenvalue of H in the full determinant space (any spin)."""
    space = DeterminantSpace(h.shape[0], 2 * nocc)
    H = hamiltonian(space, h, L)
    return np.linalg.eigvalsh(0.5 * (H + H.T))[0]
