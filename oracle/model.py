"""Model Hamiltonian of the synthetic CD-CCSD workloads (oracle side).

The electron-repulsion integrals are given by their Cholesky representation,
Sec. 2.1 Eq. 1:  (pq|rs) = sum_P L^P_pq L^P_rs.

The paper works with AO integrals, SCF orbitals and orbital relaxation
(Sec. 2.5); the synthetic workloads have none of these.  Reading adopted
for the model Hamiltonian:
  * the core Hamiltonian is fixed so that at the reference geometry the
    closed-shell Fock matrix is diag(eps):
        h_pq = eps_p delta_pq - sum_k [ 2 (pq|kk) - (pk|kq) ]
  * a displacement changes only the Cholesky vectors (L -> L + x dL/dx),
    h stays fixed ("FIXED_CORE"), the MOs are the basis (no relaxation, no
    overlap derivative: the S^x and Z-vector terms of Eq. gradcc_mo vanish;
    the variant with orbitals relaxed by the SCF condition is in
    oracle/zvector.py);
  * the energy differentiated is E = E_ref + E_corr with
        E_ref = sum_i (h_ii + f_ii),   f = h + G(L).
All functions take torch float64 tensors (dense, symmetry ignored).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def to_t(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def eri(L: torch.Tensor) -> torch.Tensor:
    """(pq|rs) = sum_P L^P_pq L^P_rs  (Sec. 2.1, Eq. 1)."""
    return torch.einsum("Ppq,Prs->pqrs", L, L)


def two_electron_fock(L: torch.Tensor, nocc: int) -> torch.Tensor:
    """G_pq = sum_k [2 (pq|kk) - (pk|kq)] over the doubly occupied k."""
    J = torch.einsum("Pkk->P", L[:, :nocc, :nocc])
    return (2.0 * torch.einsum("Ppq,P->pq", L, J)
            - torch.einsum("Ppk,Pkq->pq", L[:, :, :nocc], L[:, :nocc, :]))


def core_from_eps(eps: torch.Tensor, L: torch.Tensor, nocc: int):
    """h = diag(eps) - G(L): the fixed core Hamiltonian of the model."""
    return torch.diag(eps) - two_electron_fock(L, nocc)


def fock(h: torch.Tensor, L: torch.Tensor, nocc: int) -> torch.Tensor:
    return h + two_electron_fock(L, nocc)


def e_ref(h: torch.Tensor, L: torch.Tensor, nocc: int) -> torch.Tensor:
    """Closed-shell determinant energy sum_i (h_ii + f_ii)."""
    f = fock(h, L, nocc)
    return torch.trace(h[:nocc, :nocc]) + torch.trace(f[:nocc, :nocc])


def dense_inputs(sysm, packed_L=None):
    """(eps, L_dense) as torch float64 from a synth.System."""
    from synth import unpack_dense
    L = unpack_dense(sysm, sysm.L if packed_L is None else packed_L)
    return to_t(sysm.eps), to_t(L)
