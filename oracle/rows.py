"""CCSD energy and residual rows at given amplitudes (oracle, FP64, dense).

Test infrastructure, like the rest of `oracle/`.  The full residual in
`ccsd.residual` costs O(o^2 v^4) in its particle-particle ladder, which is
too slow on the CPU at the larger workloads.  The functions here evaluate
the SAME closed-shell CCSD equations (T1-dressed form; Sec. 2.3 for the
ladder built from L^P_ab) only where a check needs them:

  energy(t1, t2, h, L, o)
      <0| exp(-T) H exp(T) |0>: reference energy of the dressed Hamiltonian
      plus sum_ijab [2 (ia|jb) - (ib|ja)] t2[i,j,a,b].  No ladder.
  residual_rows(t1, t2, h, L, o, pairs)
      R1 (all of it) and R2[i, j, :, :] for the listed occupied pairs.  The
      ladder of one pair is sum_P Lhat^P_vv t2[i,j] (Lhat^P_vv)^T, i.e.
      sum_cd t2[i,j,c,d] (ac|bd) with (ac|bd) never formed.

Conventions are those of `ccsd.residual` (t2 is symmetrised first; R2 is the
alpha-beta projection; the ring term is the spin integration of the
spin-orbital P(ij)P(ab) t W term, direct part WA and exchange part WC).
Both functions are pinned directly against the brute-force determinant
projection (`brute.projections`) in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import torch

from .ccsd import sym2, dress, dressed_fock

einsum = torch.einsum


def _ovov_matrix(ov):
    """(ia|jb) as an (o*v) x (o*v) matrix, rows (i,a), columns (j,b)."""
    P, o, v = ov.shape
    X = ov.reshape(P, o * v)
    return X.T @ X


def energy(t1, t2, h, L, o):
    """Total energy <0|Hbar|0> at the given amplitudes (float)."""
    t2 = sym2(t2)
    Lh, hh = dress(L, h, t1, o)
    F = dressed_fock(hh, Lh, o)
    P = L.shape[0]
    v = h.shape[0] - o
    ov = Lh[:, :o, o:]                        # not changed by the dressing
    X = ov.reshape(P, o * v)
    # direct: sum (ia|jb) t2[i,j,a,b];  exchange: sum (ib|ja) t2[i,j,a,b]
    Md = t2.permute(0, 2, 1, 3).reshape(o * v, o * v)    # rows ia, cols jb
    Mx = t2.permute(0, 3, 1, 2).reshape(o * v, o * v)    # rows ib, cols ja
    direct = ((X @ Md) * X).sum()
    exch = ((X @ Mx) * X).sum()
    E = (torch.trace(hh[:o, :o]) + torch.trace(F[:o, :o])
         + 2.0 * direct - exch)
    return E.item()


def residual_rows(t1, t2, h, L, o, pairs):
    """(R1[i,a], {(i,j): R2[i,j,:,:]}) at the given amplitudes."""
    n = h.shape[0]
    v = n - o
    t2 = sym2(t2)
    Lh, hh = dress(L, h, t1, o)
    F = dressed_fock(hh, Lh, o)
    oo, ov, vo, vv = Lh[:, :o, :o], Lh[:, :o, o:], Lh[:, o:, :o], Lh[:, o:, o:]
    Foo, Fov, Fvo, Fvv = F[:o, :o], F[:o, o:], F[o:, :o], F[o:, o:]
    u = 2.0 * t2 - t2.permute(0, 1, 3, 2)

    # ---- singles (all of R1)
    R1 = Fvo.T.clone()
    Ykc = einsum("kicd,Pkc->Pid", u, ov)
    R1 = R1 + einsum("Pad,Pid->ia", vv, Ykc)
    Zlc = einsum("klac,Plc->Pka", u, ov)
    R1 = R1 - einsum("Pki,Pka->ia", oo, Zlc)
    R1 = R1 + einsum("ikac,kc->ia", u, Fov)

    # ---- intermediates shared by all rows
    G = _ovov_matrix(ov)                                 # (me|nf)
    g4 = G.reshape(o, v, o, v)
    Gx = g4.permute(0, 3, 2, 1).reshape(o * v, o * v)    # [m,e,n,f] -> (mf|ne)
    Fvv2 = Fvv - einsum("klbd,ldkc->bc", u, g4)
    Foo2 = Foo + einsum("ljcd,kdlc->kj", u, g4)

    def WA_col(j):
        """WA[m,b,e,j] for one j, as [m,b,e]."""
        direct = einsum("Pme,Pb->mbe", ov, vo[:, :, j])
        uj = u[j].permute(0, 2, 1).reshape(o * v, v)      # (n f) x b
        tj = t2[j].permute(0, 2, 1).reshape(o * v, v)
        x = (G @ uj - Gx @ tj).reshape(o, v, v)            # [m,e,b]
        return direct + 0.5 * x.permute(0, 2, 1)

    def WC_col(j):
        """WC[m,b,e,j] for one j, as [m,b,e]."""
        mjbe = einsum("Pm,Pbe->mbe", oo[:, :, j], vv)     # (mj|be)
        tj = t2[j].reshape(o * v, v)                      # [n,f,b] -> (n f) x b
        x = (Gx @ tj).reshape(o, v, v)                    # [m,e,b]
        return -mjbe + 0.5 * x.permute(0, 2, 1)

    cols = {}

    def col(j):
        if j not in cols:
            cols[j] = (WA_col(j), WC_col(j))
        return cols[j]

    def ring_row(i, j):
        """ring[i,j,a,b] of the spin-integrated ring term."""
        WAj, WCj = col(j)
        _, WCi = col(i)
        return (einsum("mbe,mae->ab", WAj, u[i])
                + einsum("mbe,mae->ab", WCj, t2[i])
                + einsum("mbe,mae->ab", WCi, t2[:, j]))

    def e1_row(i, j):
        return t2[i, j] @ Fvv2.T - einsum("kab,k->ab", t2[i], Foo2[:, j])

    def a_row(i, j):
        """(ai|bj) + ladder + hole-hole ladder at (i, j)."""
        x = vo[:, :, i].T @ vo[:, :, j]                   # (ai|bj)
        x = x + (torch.matmul(torch.matmul(vv, t2[i, j]),
                              vv.transpose(1, 2))).sum(0)  # PPL
        W = oo[:, :, i].T @ oo[:, :, j]                    # (ki|lj)
        W = W + einsum("cd,kcld->kl", t2[i, j], g4)
        return x + einsum("klab,kl->ab", t2, W)

    def x_row(i, j):
        """Unsymmetrised R2[i,j,:,:] (before the final (ia)<->(jb) average)."""
        return (a_row(i, j) + ring_row(i, j) + ring_row(j, i).T
                + e1_row(i, j) + e1_row(j, i).T)

    out = {}
    for (i, j) in pairs:
        xij = x_row(i, j)
        xji = xij if i == j else x_row(j, i)
        out[(i, j)] = 0.5 * (xij + xji.T)
    return R1, out
