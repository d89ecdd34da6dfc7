"""Closed-shell CCSD with Cholesky-vector integrals (oracle, FP64, dense).

The paper does not print the amplitude equations (Sec. 2.3 refers the PPL
strategy to earlier work).  The oracle writes them from coupled-cluster
theory in the T1-similarity-transformed form:

  * T1 dressing.  With the n x n matrix t (t_ai = t1[i,a], zero elsewhere),
    exp(-T1) H exp(T1) has one-electron integrals (1-t) h (1+t) and
    Cholesky vectors  Lhat^P = (1 - t) L^P (1 + t).  These are the
    t1-contracted Cholesky intermediates t^P_ia, t^P_ai, t^P_ij, t^P_ab of
    App. A, summed into one dressed vector.
  * On the dressed Hamiltonian the singles and doubles projections are those
    of CCD with a general (non-Hermitian) Hamiltonian plus the singles
    projection.  Conventions:
        t2[i,j,a,b] = amplitude of  a^+_{a alpha} a^+_{b beta} a_{j beta} a_{i alpha}
        R1[i,a]     = < Phi_{i alpha}^{a alpha} | exp(-T) H exp(T) | 0 >
        R2[i,j,a,b] = < Phi_{i alpha j beta}^{a alpha b beta} | exp(-T) H exp(T) | 0 >
    (pinned against the brute-force determinant projection in
    oracle/brute.py by tests/test_oracle_pins.py).
  * Particle-particle ladder (Sec. 2.3, PPL):  sum_cd t[i,j,c,d] (ac|bd) with
    (ac|bd) = sum_P Lhat^P_ac Lhat^P_bd assembled on the fly per block of a;
    W_abcd is never stored whole.

Integrals (pq|rs) are Mulliken; <pq|rs> = (pr|qs).
"""
from __future__ import annotations

import math
import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

from .model import DT, fock, e_ref

einsum = torch.einsum


def sym2(t2):
    """Symmetrise a doubles array under the simultaneous swap (i,a)<->(j,b)."""
    return 0.5 * (t2 + t2.permute(1, 0, 3, 2))


def P_ij_ab(x):
    """P^{ab}_{ij} X[i,j,a,b] = X[i,j,a,b] + X[j,i,b,a]."""
    return x + x.permute(1, 0, 3, 2)


def dressing_matrices(t1, n, o):
    X = torch.eye(n, dtype=DT)
    Y = torch.eye(n, dtype=DT)
    if t1.numel():
        X = X.clone()
        Y = Y.clone()
        X[o:, :o] = -t1.T
        Y[o:, :o] = t1.T
    return X, Y


def dress(L, h, t1, o):
    """Lhat^P = (1-t) L^P (1+t),  hhat = (1-t) h (1+t)."""
    n = h.shape[0]
    X, Y = dressing_matrices(t1, n, o)
    return X @ L @ Y, X @ h @ Y


def dressed_fock(hh, Lh, o):
    """F_pq = hhat_pq + sum_k [2 (pq|kk)^ - (pk|kq)^] from dressed vectors."""
    J = einsum("Pkk->P", Lh[:, :o, :o])
    return (hh + 2.0 * einsum("Ppq,P->pq", Lh, J)
            - einsum("Ppk,Pkq->pq", Lh[:, :, :o], Lh[:, :o, :]))


def ladder_block(t2, vv, a0: int, a1: int, ein=None):
    """Rows a0 <= a < a1 of the ladder: (ac|bd) for that block of a, then
    sum_cd t[i,j,c,d] (ac|bd)."""
    if ein is None:
        W = einsum("Pac,Pbd->acbd", vv[:, a0:a1], vv)    # (ac|bd), a in block
        return einsum("ijcd,acbd->ijab", t2, W)
    W = ein("Pac,Pbd->acbd", vv[:, a0:a1], vv, ranges={"a": (a0, a1)})
    return ein("ijcd,acbd->ijab", t2, W, ranges={"a": (a0, a1)})


def ladder(t2, vv, ein=None):
    """sum_cd t[i,j,c,d] (ac|bd), (ac|bd) = sum_P vv[P,a,c] vv[P,b,d]."""
    v = vv.shape[1]
    if v == 0:
        return torch.zeros_like(t2)
    blk = max(1, min(v, int(2.0e7 // max(1, v ** 3))))
    if blk >= v:
        return ladder_block(t2, vv, 0, v, ein)
    parts = []
    for a0 in range(0, v, blk):
        a1 = min(v, a0 + blk)
        if torch.is_grad_enabled():
            parts.append(checkpoint(ladder_block, t2, vv, a0, a1, ein,
                                    use_reentrant=False))
        else:
            parts.append(ladder_block(t2, vv, a0, a1, ein))
    return torch.cat(parts, dim=2)


def residual(t1, t2, h, L, o, ein=None):
    """Closed-shell CCSD residuals and total energy.

    Returns (R1[i,a], R2[i,j,a,b], E) where E = <0|exp(-T) H exp(T)|0> is the
    total energy (reference + correlation).  t2 is symmetrised first, so the
    function is defined on the physical (symmetric) amplitude manifold.
    `ein` replaces torch.einsum in the contractions below (None: the dense
    einsum; oracle.blocked.irrep_einsum: the same products over the
    symmetry-allowed blocks only).
    """
    einsum = torch.einsum if ein is None else ein
    n = h.shape[0]
    t2 = sym2(t2)
    Lh, hh = dress(L, h, t1, o)
    F = dressed_fock(hh, Lh, o)
    oo, ov, vo, vv = Lh[:, :o, :o], Lh[:, :o, o:], Lh[:, o:, :o], Lh[:, o:, o:]
    Foo, Fov, Fvo, Fvv = F[:o, :o], F[:o, o:], F[o:, :o], F[o:, o:]

    g_ovov = einsum("Pia,Pjb->iajb", ov, ov)     # (ia|jb) (not dressed)
    g_vovo = einsum("Pai,Pbj->aibj", vo, vo)     # (ai|bj)
    g_oooo = einsum("Pki,Plj->kilj", oo, oo)     # (ki|lj)
    g_oovv = einsum("Pki,Pac->kiac", oo, vv)     # (ki|ac)
    g_exch = g_ovov.permute(0, 3, 2, 1)          # [l,d,k,c] -> (lc|kd)
    u = 2.0 * t2 - t2.permute(0, 1, 3, 2)        # u[i,j,a,b] = 2t_ij^ab - t_ij^ba

    # ---- singles
    R1 = Fvo.T.clone()                                            # F_ai
    Ykc = einsum("kicd,Pkc->Pid", u, ov)
    R1 = R1 + einsum("Pad,Pid->ia", vv, Ykc)                       # u (ad|kc)
    Zlc = einsum("klac,Plc->Pka", u, ov)
    R1 = R1 - einsum("Pki,Pka->ia", oo, Zlc)                       # u (ki|lc)
    R1 = R1 + einsum("ikac,kc->ia", u, Fov)                        # u F_kc

    # ---- doubles
    R2 = g_vovo.permute(1, 3, 0, 2)                                # (ai|bj)
    R2 = R2 + ladder(t2, vv, ein)                                  # PPL
    W = g_oooo + einsum("ijcd,kcld->kilj", t2, g_ovov)             # hole-hole
    R2 = R2 + einsum("klab,kilj->ijab", t2, W)
    # rings: the spin-orbital term P(ij)P(ab) sum_me t_im^ae W_mbej integrated
    # over spin; WA is the direct (same-pair) and WC the exchange pattern.
    g_ovvo = einsum("Pme,Pbj->mebj", ov, vo)                      # (me|bj)
    WA = (g_ovvo.permute(0, 2, 1, 3)
          + 0.5 * einsum("jnbf,menf->mbej", u, g_ovov)
          - 0.5 * einsum("jnbf,mfne->mbej", t2, g_ovov))
    WC = (-g_oovv.permute(0, 2, 3, 1)                              # -(mj|be)
          + 0.5 * einsum("jnfb,mfne->mbej", t2, g_ovov))
    ring = (einsum("mbej,imae->ijab", WA, u)
            + einsum("mbej,imae->ijab", WC, t2)
            + einsum("mbei,mjae->ijab", WC, t2))
    R2 = R2 + P_ij_ab(ring)
    Fvv2 = Fvv - einsum("klbd,ldkc->bc", u, g_ovov)
    Foo2 = Foo + einsum("ljcd,kdlc->kj", u, g_ovov)
    E1 = einsum("ijac,bc->ijab", t2, Fvv2) - einsum("ikab,kj->ijab", t2, Foo2)
    R2 = R2 + P_ij_ab(E1)
    R2 = sym2(R2)

    # ---- energy: <0|Hhat|0> + sum (2(ia|jb) - (ib|ja)) t_ij^ab
    E = (torch.trace(hh[:o, :o]) + torch.trace(F[:o, :o])
         + einsum("iajb,ijab->", 2.0 * g_ovov - g_exch, t2))
    return R1, R2, E


def denominators(f, o):
    d = torch.diagonal(f)
    Dia = d[:o, None] - d[None, o:]
    Dijab = (d[:o, None, None, None] + d[None, :o, None, None]
             - d[None, None, o:, None] - d[None, None, None, o:])
    return Dia, Dijab


class DIIS:
    """Pulay extrapolation on flattened vectors (Sec. 2.3 uses DIIS for the
    Lambda equations; the same scheme drives the amplitude equations)."""

    def __init__(self, nvec=8):
        self.nvec = nvec
        self.vecs, self.errs = [], []

    def push(self, vec, err):
        self.vecs.append(vec.clone())
        self.errs.append(err.clone())
        if len(self.vecs) > self.nvec:
            self.vecs.pop(0)
            self.errs.pop(0)

    def extrapolate(self):
        m = len(self.vecs)
        B = torch.empty((m + 1, m + 1), dtype=DT)
        for i in range(m):
            for j in range(i + 1):
                B[i, j] = B[j, i] = torch.dot(self.errs[i], self.errs[j])
        B[m, :m] = -1.0
        B[:m, m] = -1.0
        B[m, m] = 0.0
        rhs = torch.zeros(m + 1, dtype=DT)
        rhs[m] = -1.0
        # scale for conditioning
        s = torch.diagonal(B)[:m].max()
        if s > 0:
            B[:m, :m] /= s
        c = torch.linalg.solve(B, rhs)[:m]
        out = torch.zeros_like(self.vecs[0])
        for ci, vi in zip(c, self.vecs):
            out += ci * vi
        return out


def pack_amps(t1, t2):
    return torch.cat([t1.reshape(-1), t2.reshape(-1)])


def unpack_amps(vec, o, v):
    return vec[:o * v].reshape(o, v), vec[o * v:].reshape(o, o, v, v)


def solve_ccsd(h, L, o, tol=1e-10, e_tol=1e-12, maxiter=200, ndiis=8,
               diis_start=2, verbose=False):
    """Jacobi iterations with DIIS from t1 = 0, t2 = 0 (first step = MP2).

    Convergence: max |R/D| <= tol and |dE| <= e_tol.  Returns a dict with
    t1, t2, E (total), E_corr, iterations and the final max |R/D|.
    """
    n = h.shape[0]
    v = n - o
    f = fock(h, L, o)
    Dia, Dijab = denominators(f, o)
    eref = e_ref(h, L, o).item()
    t1 = torch.zeros((o, v), dtype=DT)
    t2 = torch.zeros((o, o, v, v), dtype=DT)
    diis = DIIS(ndiis)
    e_old = None
    hist = []
    with torch.no_grad():
        for it in range(1, maxiter + 1):
            R1, R2, E = residual(t1, t2, h, L, o)
            E = E.item()
            s1, s2 = R1 / Dia, R2 / Dijab
            rmax = max(s1.abs().max().item() if s1.numel() else 0.0,
                       s2.abs().max().item() if s2.numel() else 0.0)
            hist.append((it, E - eref, rmax))
            if verbose:
                print(f"ccsd it {it:3d} Ecorr {E - eref:.14f} rmax {rmax:.3e}")
            if (rmax <= tol and e_old is not None
                    and abs(E - e_old) <= e_tol):
                break
            e_old = E
            t1 = t1 + s1
            t2 = t2 + s2
            if ndiis and it >= diis_start:
                diis.push(pack_amps(t1, t2), pack_amps(s1, s2))
                if len(diis.vecs) >= 2:
                    t1, t2 = unpack_amps(diis.extrapolate(), o, v)
        else:
            raise RuntimeError(f"CCSD did not converge in {maxiter} iterations"
                               f" (rmax {rmax:.3e})")
    return dict(t1=t1, t2=sym2(t2), E=E, E_corr=E - eref, E_ref=eref,
                iterations=it, rmax=rmax, history=hist)


def energy_corr(t1, t2, h, L, o):
    """Correlation energy at given amplitudes: <0|Hbar|0> - E_ref."""
    with torch.no_grad():
        _, _, E = residual(t1, t2, h, L, o)
    return (E - e_ref(h, L, o)).item()
