"""Lambda equations, Cholesky-basis densities and the gradient (oracle).

Sec. 2.2 defines the CC Lagrangian; for the model Hamiltonian (no orbital
relaxation, no overlap, see oracle/model.py) it reduces to
    Lag(t, lambda; h, L) = E(t; h, L) + sum_ia l1[i,a] R1[i,a]
                                       + sum_ijab l2[i,j,a,b] R2[i,j,a,b]
with E, R1, R2 from oracle/ccsd.py.  (The paper's Lambda-operator
normalisation differs by constant factors per block; the gradient does not
depend on it.)

  * Lambda equations (Sec. 2.3): dLag/dt = 0.  The printed spin-adapted
    equations (Eqs. lambda_singles / lambda_doubles, App. A) contain
    undefined and inconsistent symbols, so the oracle does not transcribe
    them: it takes the transpose products lambda . dR/dt by reverse-mode
    differentiation of the residual, which is the definition.
  * Cholesky-basis density (Sec. 2.6, Gamma^P_pr of Eq. d2xtl1 summed with
    the 1-particle and reference parts):
        Gamma^P_pq = d Lag / d L^P_pq   at converged (t, lambda), h fixed,
    symmetrised in pq.  Then, with the differentiated-CV form of the ERI
    derivative (Sec. 2.1, Eq. 2),
        dE/dx = sum_P sum_pq Gamma^P_pq dL^P_pq/dx.
  * One-particle density D_pq = d Lag / d h_pq (symmetrised): the full
    (reference + correlation) 1-RDM of the Lagrangian.
"""
from __future__ import annotations

import torch

from .model import DT, fock
from .ccsd import residual, denominators, DIIS, pack_amps, unpack_amps, sym2


def lagrangian(t1, t2, l1, l2, h, L, o, ein=None):
    """Lag at (t, lambda); `ein` as in oracle.ccsd.residual."""
    R1, R2, E = residual(t1, t2, h, L, o, ein)
    return E + (l1 * R1).sum() + (l2 * R2).sum()


def lambda_gradient(t1, t2, l1, l2, h, L, o):
    """dLag/dt1, dLag/dt2 (the Lambda-equation residuals)."""
    with torch.enable_grad():
        a1 = t1.detach().clone().requires_grad_(True)
        a2 = t2.detach().clone().requires_grad_(True)
        lag = lagrangian(a1, a2, l1, l2, h, L, o)
        g1, g2 = torch.autograd.grad(lag, (a1, a2))
    return g1, g2


def solve_lambda(t1, t2, h, L, o, tol=1e-10, maxiter=200, ndiis=8,
                 diis_start=2, verbose=False):
    """Jacobi iterations  lambda <- lambda + G/D  with DIIS, from lambda = 0
    (the first step gives dE/dt / D).  Convergence: max |G/D| <= tol."""
    n = h.shape[0]
    v = n - o
    f = fock(h, L, o)
    Dia, Dijab = denominators(f, o)
    l1 = torch.zeros((o, v), dtype=DT)
    l2 = torch.zeros((o, o, v, v), dtype=DT)
    diis = DIIS(ndiis)
    hist = []
    for it in range(1, maxiter + 1):
        g1, g2 = lambda_gradient(t1, t2, l1, l2, h, L, o)
        s1, s2 = g1 / Dia, g2 / Dijab
        rmax = max(s1.abs().max().item() if s1.numel() else 0.0,
                   s2.abs().max().item() if s2.numel() else 0.0)
        hist.append((it, rmax))
        if verbose:
            print(f"lambda it {it:3d} rmax {rmax:.3e}")
        if rmax <= tol:
            break
        l1 = l1 + s1
        l2 = l2 + s2
        if ndiis and it >= diis_start:
            diis.push(pack_amps(l1, l2), pack_amps(s1, s2))
            if len(diis.vecs) >= 2:
                l1, l2 = unpack_amps(diis.extrapolate(), o, v)
    else:
        raise RuntimeError(f"Lambda did not converge in {maxiter} iterations")
    return dict(l1=l1, l2=sym2(l2), iterations=it, rmax=rmax, history=hist)


def densities(t1, t2, l1, l2, h, L, o):
    """Return (Gamma^P_pq, D_pq, Lag) at the given amplitudes; both
    derivatives symmetrised in pq."""
    with torch.enable_grad():
        Lv = L.detach().clone().requires_grad_(True)
        hv = h.detach().clone().requires_grad_(True)
        lag = lagrangian(t1, t2, l1, l2, hv, Lv, o)
        gL, gh = torch.autograd.grad(lag, (Lv, hv))
    G = 0.5 * (gL + gL.transpose(1, 2))
    D = 0.5 * (gh + gh.T)
    return G.detach(), D.detach(), lag.item()


def density_frozen_fock(t1, t2, l1, l2, eps, L, o):
    """Gamma^P of the FROZEN_FOCK model (the alternative reading of the model
    Hamiltonian): the Fock matrix stays diag(eps) under a displacement, i.e.
    h follows L as h(L) = diag(eps) - G(L), and the energy differentiated is
    the correlation energy:
        Gamma_FF^P = d/dL [Lag(t, lambda; h(L), L) - E_ref(h(L), L)],
    symmetrised in pq.  The amplitude and Lambda equations at x = 0 are
    those of the default model (same h, same L); only Gamma changes."""
    from .model import core_from_eps, e_ref
    with torch.enable_grad():
        Lv = L.detach().clone().requires_grad_(True)
        hv = core_from_eps(torch.as_tensor(eps, dtype=DT), Lv, o)
        lag = lagrangian(t1, t2, l1, l2, hv, Lv, o) - e_ref(hv, Lv, o)
        (gL,) = torch.autograd.grad(lag, (Lv,))
    return (0.5 * (gL + gL.transpose(1, 2))).detach()


def gradient_from_density(G, dL):
    """g_x = sum_P sum_pq Gamma^P_pq dL^P_pq/dx for each displacement x."""
    return torch.einsum("Ppq,xPpq->x", G, dL)


def run_all(h, L, o, tol=1e-10, e_tol=1e-12, verbose=False):
    """CCSD -> Lambda -> densities.  Returns a dict with everything."""
    from .ccsd import solve_ccsd
    cc = solve_ccsd(h, L, o, tol=tol, e_tol=e_tol, verbose=verbose)
    lam = solve_lambda(cc["t1"], cc["t2"], h, L, o, tol=tol, verbose=verbose)
    G, D, lag = densities(cc["t1"], cc["t2"], lam["l1"], lam["l2"], h, L, o)
    return dict(cc=cc, lam=lam, G=G, D=D, lag=lag)
