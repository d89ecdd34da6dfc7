"""Orbital relaxation: Z-vector equations and the relaxed gradient
(Sec. 2.5, Eq. z_vector) for the relaxed variant of the model (oracle).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this module; the library never does.

Model with orbital rotations (reading).  The fixed-core model (model.py)
keeps the orbitals of the reference: a displacement changes L only.  In its
relaxed variant the orbitals follow the closed-shell SCF condition of the
same Hamiltonian: at every displacement x they are rotated, phi' = phi U
with U = exp(K) orthogonal (the basis is orthonormal and fixed, so the
overlap derivative S^x of the paper vanishes), K antisymmetric with only
the virtual-occupied block K_ai = kappa_ai free (CCSD is invariant to
occupied-occupied and virtual-virtual rotations), and kappa(x) chosen so
that the rotated Fock matrix has no virtual-occupied block (Brillouin):
    f'_ai(kappa, x) = 0,   f' = h' + G(L'),  h' = U^T h U,  L'^P = U^T L^P U.
At x = 0, kappa = 0 solves it (f = diag(eps) in the model).  The relaxed
energy is E_rel(x) = E(t, lambda; h'(x), L'(x)) with the CCSD amplitudes
re-solved in the rotated orbitals.

Gradient (Sec. 2.5).  With the Lagrangian Lag of lagrangian.py at the
converged (t, lambda) and kappa = 0,
    dE_rel/dx = dLag/dx + sum_ai Z_ai d f_ai / dx   (orbitals fixed)
where Z solves the Z-vector equations
    sum_bj Z_bj A_bj,ai = - dLag/dkappa_ai,   A_bj,ai = d f_bj / d kappa_ai,
A being the closed-shell orbital Hessian of Eq. z_vector and the right-hand
side the orbital gradient of the Lagrangian (the I'_IA - I'_AI of the paper
in this model).  The orbital terms are written out from the densities:
    dLag/dkappa_ai = 2 W_ai,   W = [h, D] + sum_P [L^P, Gamma^P]
(D = dLag/dh, Gamma^P = dLag/dL^P, both symmetric), and the relaxation adds
Gamma_Z^P = d/dL^P (sum_ai Z_ai f_ai) to Gamma^P, so the relaxed gradient
is <Gamma^P + Gamma_Z^P, dL^P/dx>.  Every written-out term is checked
against the reverse-mode derivative it stands for, and the relaxed
gradient against a central difference of E_rel (tests/test_oracle_zvector.py).
"""
from __future__ import annotations

import torch

from .model import DT, fock
from .ccsd import solve_ccsd
from .lagrangian import lagrangian


def generator(kappa, n, o):
    """Antisymmetric K with K[a, i] = kappa[a - o, i] (a virtual, i
    occupied) and K[i, a] = -kappa[a - o, i]."""
    K = torch.zeros((n, n), dtype=DT)
    K[o:, :o] = kappa
    K[:o, o:] = -kappa.T
    return K


def rotate(h, L, kappa, o):
    """h' = U^T h U, L'^P = U^T L^P U with U = exp(K(kappa))."""
    U = torch.linalg.matrix_exp(generator(kappa, h.shape[0], o))
    return U.T @ h @ U, U.T @ L @ U


def brillouin(h, L, o):
    """f_ai of the closed-shell Fock matrix (virtual x occupied)."""
    return fock(h, L, o)[o:, :o]


def orbital_hessian(h, L, o):
    """A[b,j,a,i] = d f_bj / d kappa_ai at kappa = 0 (reverse mode)."""
    n = h.shape[0]
    v = n - o

    def f(kappa):
        hr, Lr = rotate(h, L, kappa, o)
        return brillouin(hr, Lr, o)

    return torch.autograd.functional.jacobian(
        f, torch.zeros((v, o), dtype=DT))


def orbital_hessian_eq(eps, L, o):
    """The bracket of Eq. z_vector, with <pq|rs> = (pr|qs):
    H[a,i,e,m] = (eps_a - eps_i) d_ea d_mi + 2<Ei|Ma> - <Ei|Am>
                 + 2<Ea|Mi> - <Ea|Im>
               = (eps_a - eps_i) d_ea d_mi + 2(em|ia) - (ea|im)
                 + 2(em|ai) - (ei|am)."""
    n = L.shape[1]
    v = n - o
    Lvo, Lov = L[:, o:, :o], L[:, :o, o:]
    Lvv, Loo = L[:, o:, o:], L[:, :o, :o]
    H = (2.0 * torch.einsum("Pem,Pia->aiem", Lvo, Lov)
         - torch.einsum("Pea,Pim->aiem", Lvv, Loo)
         + 2.0 * torch.einsum("Pem,Pai->aiem", Lvo, Lvo)
         - torch.einsum("Pei,Pam->aiem", Lvo, Lvo))
    d = eps[o:, None] - eps[None, :o]
    H = H + torch.diag_embed(d.reshape(-1)).reshape(v, o, v, o)
    return H


def lagrangian_orbital_gradient(t1, t2, l1, l2, h, L, o):
    """dLag/dkappa_ai at kappa = 0 (reverse mode), (t, lambda) fixed."""
    n = h.shape[0]
    with torch.enable_grad():
        kappa = torch.zeros((n - o, o), dtype=DT, requires_grad=True)
        hr, Lr = rotate(h, L, kappa, o)
        lag = lagrangian(t1, t2, l1, l2, hr, Lr, o)
        (g,) = torch.autograd.grad(lag, kappa)
    return g


def orbital_gradient(D, G, h, L, o):
    """2 W_ai with W = [h, D] + sum_P [L^P, Gamma^P] (D, Gamma^P symmetric):
    the orbital gradient from the densities."""
    W = h @ D - D @ h + torch.einsum("Ppr,Prq->pq", L, G) \
        - torch.einsum("Ppr,Prq->pq", G, L)
    return 2.0 * W[o:, :o]


def z_vector(A, rhs):
    """Solve sum_bj Z_bj A[b,j,a,i] = -rhs[a,i]."""
    v, o = rhs.shape
    M = A.reshape(v * o, v * o)
    return torch.linalg.solve(M.T, -rhs.reshape(-1)).reshape(v, o)


def relaxation_density(Z, h, L, o):
    """Gamma_Z^P = d/dL^P sum_ai Z_ai f_ai (reverse mode, symmetrised)."""
    with torch.enable_grad():
        Lg = L.detach().clone().requires_grad_(True)
        s = (Z * brillouin(h, Lg, o)).sum()
        (g,) = torch.autograd.grad(s, Lg)
    return 0.5 * (g + g.transpose(1, 2))


def relaxation_density_eq(Z, L, o):
    """Gamma_Z^P written out: with f_ai = h_ai + sum_k [2 (ai|kk) -
    (ak|ki)], the derivative of sum_ai Z_ai f_ai with respect to L^P_pq,
    symmetrised in pq."""
    J = torch.einsum("Pkk->P", L[:, :o, :o])
    g = torch.zeros_like(L)
    g[:, o:, :o] += 2.0 * J[:, None, None] * Z[None]                # L_ai
    zl = torch.einsum("ai,Pai->P", Z, L[:, o:, :o])
    g[:, :o, :o] += 2.0 * zl[:, None, None] * torch.eye(o, dtype=DT)  # L_kk
    g[:, o:, :o] -= torch.einsum("ai,Pki->Pak", Z, L[:, :o, :o])    # L_ak
    g[:, :o, :o] -= torch.einsum("ai,Pak->Pki", Z, L[:, o:, :o])    # L_ki
    return 0.5 * (g + g.transpose(1, 2))


def scf_rotation(h, L, o, tol=1e-13, maxiter=50):
    """kappa with f'_ai(kappa) = 0 by Newton iterations from kappa = 0
    (the relaxed orbitals of a displaced model)."""
    n = h.shape[0]
    kappa = torch.zeros((n - o, o), dtype=DT)

    def f(k):
        hr, Lr = rotate(h, L, k, o)
        return brillouin(hr, Lr, o)

    for _ in range(maxiter):
        r = f(kappa)
        if float(r.abs().max()) <= tol:
            return kappa
        J = torch.autograd.functional.jacobian(f, kappa)
        m = r.numel()
        step = torch.linalg.solve(J.reshape(m, m), r.reshape(-1))
        kappa = kappa - step.reshape(kappa.shape)
    raise RuntimeError("relaxed orbitals: Newton iterations did not converge")


def relaxed_energy(h, L, o, tol=1e-13, e_tol=1e-14):
    """E_rel: total CCSD energy in the relaxed orbitals of (h, L)."""
    kappa = scf_rotation(h, L, o)
    hr, Lr = rotate(h, L, kappa, o)
    return solve_ccsd(hr, Lr, o, tol=tol, e_tol=e_tol)["E"]


def relaxed_gradient(r, h, L, o, dL):
    """Relaxed gradient from a lagrangian.run_all result r at (h, L):
    (g_rel[x], Z, Gamma_rel) with g_rel = <Gamma^P + Gamma_Z^P, dL_x>."""
    A = orbital_hessian(h, L, o)
    rhs = orbital_gradient(r["D"], r["G"], h, L, o)
    Z = z_vector(A, rhs)
    Grel = r["G"] + relaxation_density_eq(Z, L, o)
    return torch.einsum("Ppq,xPpq->x", Grel, dL), Z, Grel
