"""Check of a gradient chain (t, lambda, Gamma^P) against the oracle's
Lagrangian at sizes where the dense oracle cannot solve the equations but
can still evaluate the Lagrangian once (Sec. 2.2):

    Lag(t, lambda; h, L) = E(t; h, L) + lambda1 . R1(t; h, L)
                                      + lambda2 . R2(t; h, L)

(oracle/lagrangian.py).  At a solution, Lag is stationary in t (the
amplitude and Lambda equations), and the gradient along a displacement D of
the Cholesky vectors at fixed h is dLag/dL . D = <Gamma^P, D>.  Both follow
from one central difference of Lag along the joint direction (dt, D):

    [Lag(t + e dt, L + e D) - Lag(t - e dt, L - e D)] / (2e)
        = dLag/dt . dt + dLag/dL . D + O(e^2 dt^3)

with dLag/dt . dt = 0 when lambda solves the Lambda equations, and no
truncation error in D (Lag is a quadratic polynomial in L at fixed t,
lambda and h).  A random dt makes a wrong lambda show up; comparing with
<Gamma^P, D> from the chain under test checks Gamma^P.  The Lagrangian is
evaluated with the symmetry-blocked einsum (oracle/blocked.py, pinned to
the dense one), which makes it affordable at c2.  Test helper only.
"""
import numpy as np
import torch

from synth import unpack_dense
from oracle import model, lagrangian, blocked


def allowed_doubles(s):
    """Symmetry pattern of t2[i,j,a,b]: irrep(i)^irrep(j) = irrep(a)^irrep(b)."""
    irr = np.asarray(s.orb_irrep)
    o = s.nocc
    io, iv = irr[:o], irr[o:]
    return ((io[:, None, None, None] ^ io[None, :, None, None]) ==
            (iv[None, None, :, None] ^ iv[None, None, None, :]))


def allowed_singles(s):
    irr = np.asarray(s.orb_irrep)
    o = s.nocc
    return irr[:o, None] == irr[None, o:]


def random_direction(s, t1, t2, seed=0):
    """Random amplitude direction with the symmetry pattern, scaled to the
    amplitudes' largest element, t2 part symmetric under (ia) <-> (jb)."""
    rng = np.random.default_rng(seed)
    d1 = rng.standard_normal(t1.shape) * allowed_singles(s)
    d2 = rng.standard_normal(t2.shape)
    d2 = 0.5 * (d2 + d2.transpose(1, 0, 3, 2)) * allowed_doubles(s)
    d1 *= np.abs(t1).max() / max(np.abs(d1).max(), 1e-300)
    d2 *= np.abs(t2).max() / max(np.abs(d2).max(), 1e-300)
    return d1, d2


def lagrangian_difference(s, t1, t2, l1, l2, dt1, dt2, D_packed, step):
    """Central difference of the oracle's Lagrangian along (dt, D) at fixed
    h = the model's core Hamiltonian of the undisplaced L."""
    T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa
    o = s.nocc
    L0 = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L0, o)
    D = T(unpack_dense(s, D_packed))
    ein = blocked.for_system(s)
    vals = []
    with torch.no_grad():
        for sg in (1.0, -1.0):
            vals.append(float(lagrangian.lagrangian(
                T(t1) + sg * step * T(dt1), T(t2) + sg * step * T(dt2),
                T(l1), T(l2), h, L0 + sg * step * D, o, ein)))
    return (vals[0] - vals[1]) / (2.0 * step)
