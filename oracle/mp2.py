"""Closed-form closed-shell MP2 energy with canonical orbitals (pin).

E_MP2 = sum_ijab (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b),
(ia|jb) = sum_P L^P_ia L^P_jb (Sec. 2.1, Eq. 1).  It equals the CCSD energy
expression at t1 = 0 and the first-order doubles t2 = (ai|bj)/D.
"""
from __future__ import annotations

import numpy as np


def mp2_energy(eps: np.ndarray, L: np.ndarray, o: int) -> float:
    Lov = L[:, :o, o:]
    g = np.einsum("Pia,Pjb->iajb", Lov, Lov)
    e_o, e_v = eps[:o], eps[o:]
    D = (e_o[:, None, None, None] - e_v[None, :, None, None]
         + e_o[None, None, :, None] - e_v[None, None, None, :])
    return float(np.sum(g * (2.0 * g - g.transpose(0, 3, 2, 1)) / D))
