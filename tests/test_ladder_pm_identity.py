"""The symmetric/antisymmetric (+/-) packing of the particle-particle ladder
(Sec. 2.3) reproduces the plain ladder (CPU only).

The CUDA map (csrc/ladder_pm.cu) computes, over canonical pairs (p,q) of
each index pair (irrep(p) > irrep(q), or the same irrep and p >= q),
  A+-_{ij,cd} = (X_{ij,cd} + X_{ji,dc} +- (X_{ij,dc} + X_{ji,cd})) / 4
  W+-_{ab,cd} = (ac|bd) +- (ad|bc)   (c != d);  W+_{ab,cc} = (ac|bc), W- = 0
  S+- = A+- W+-^T
and every ordered element Y_{ij,ab} = S+ + s S- of its canonical
representative, s = -1 when exactly one of (ij), (ab) is swapped.  This test
writes those formulas out with loops over small symmetry-blocked arrays and
checks them against the plain contraction sum_cd X_{ij,cd} (ac|bd) for
pair-symmetric X, including the diagonal pairs (i = j, a = b, c = d) whose
weights a dropped factor would break, and checks that a planted sign error
is caught.  The partial form for O(o^3 v^3) products (only ij and cd
packed, the output pair unsymmetric) is pinned the same way.
"""
import numpy as np


def _system(seed, occ, vir, nq):
    rng = np.random.default_rng(seed)
    oi = np.repeat(np.arange(len(occ)), occ)
    vi = np.repeat(np.arange(len(vir)), vir)
    no, nv = len(oi), len(vi)
    # L^P_ac with irrep(P) = irrep(a) ^ irrep(c), symmetric in ac
    qi = np.repeat(np.arange(len(nq)), nq)
    L = rng.standard_normal((len(qi), nv, nv))
    L = 0.5 * (L + L.transpose(0, 2, 1))
    L *= (qi[:, None, None] == (vi[:, None] ^ vi[None, :])[None])
    V = np.einsum("Pac,Pbd->abcd", L, L)           # (ac|bd) at [a,b,c,d]
    # pair-symmetric amplitudes with the pair irrep rule
    X = rng.standard_normal((no, no, nv, nv))
    X = 0.5 * (X + X.transpose(1, 0, 3, 2))
    allowed = ((oi[:, None, None, None] ^ oi[None, :, None, None]) ==
               (vi[None, None, :, None] ^ vi[None, None, None, :]))
    return oi, vi, X * allowed, V


def _canonical(irr):
    n = len(irr)
    return [(p, q) for p in range(n) for q in range(n)
            if irr[p] > irr[q] or (irr[p] == irr[q] and p >= q)]


def _pm_ladder(oi, vi, X, V, sign=1.0):
    no, nv = len(oi), len(vi)
    Y = np.zeros_like(X)
    for G in range(max(oi.max(), vi.max()) + 1):
        R = [(i, j) for (i, j) in _canonical(oi) if oi[i] ^ oi[j] == G]
        C = [(c, d) for (c, d) in _canonical(vi) if vi[c] ^ vi[d] == G]
        if not R or not C:
            continue
        Ap = np.zeros((len(R), len(C)))
        Am = np.zeros_like(Ap)
        for r, (i, j) in enumerate(R):
            for u, (c, d) in enumerate(C):
                s_ = X[i, j, c, d] + X[j, i, d, c]
                t_ = X[i, j, d, c] + X[j, i, c, d]
                Ap[r, u] = 0.25 * (s_ + t_)
                Am[r, u] = 0.25 * (s_ - t_)
        Wp = np.zeros((len(C), len(C)))
        Wm = np.zeros_like(Wp)
        for v, (a, b) in enumerate(C):
            for u, (c, d) in enumerate(C):
                w1, w2 = V[a, b, c, d], V[a, b, d, c]
                if c == d:
                    Wp[v, u], Wm[v, u] = w1, 0.0
                else:
                    Wp[v, u], Wm[v, u] = w1 + w2, w1 - w2
        Sp, Sm = Ap @ Wp.T, sign * (Am @ Wm.T)
        for r, (i, j) in enumerate(R):
            for v, (a, b) in enumerate(C):
                p_, m_ = Sp[r, v], Sm[r, v]
                Y[i, j, a, b] += p_ + m_
                if a != b:
                    Y[i, j, b, a] += p_ - m_
                if i != j:
                    Y[j, i, a, b] += p_ - m_
                    if a != b:
                        Y[j, i, b, a] += p_ + m_
    return Y


def test_pm_packing_reproduces_the_ladder():
    for seed, occ, vir, nq in [(1, [2, 1], [3, 2], [4, 3]),
                               (2, [2, 1, 1, 1], [3, 2, 2, 1], [3, 2, 2, 2]),
                               (3, [3], [4], [5])]:
        oi, vi, X, V = _system(seed, occ, vir, nq)
        ref = np.einsum("ijcd,abcd->ijab", X, V)
        got = _pm_ladder(oi, vi, X, V)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), seed


def test_pm_flops_are_a_quarter():
    # canonical pairs per pair irrep: about half of all pairs
    oi = np.repeat(np.arange(8), 8)
    vi = np.repeat(np.arange(8), 60)
    full = sum(((oi[:, None] ^ oi[None, :]) == G).sum() *
               ((vi[:, None] ^ vi[None, :]) == G).sum() ** 2
               for G in range(8))
    co, cv = _canonical(oi), _canonical(vi)
    packed = 2 * sum(
        sum(1 for i, j in co if oi[i] ^ oi[j] == G) *
        sum(1 for c, d in cv if vi[c] ^ vi[d] == G) ** 2 for G in range(8))
    assert 0.25 <= packed / full <= 0.30


def test_planted_sign_error_is_caught():
    oi, vi, X, V = _system(2, [2, 1, 1, 1], [3, 2, 2, 1], [3, 2, 2, 2])
    ref = np.einsum("ijcd,abcd->ijab", X, V)
    bad = _pm_ladder(oi, vi, X, V, sign=-1.0)
    assert np.abs(bad - ref).max() > 1e-3 * np.abs(ref).max()


def _partial_pm(oi, vi, X, V):
    """Partial +/- form (Sec. 2.5) of Y_{ij,mb} = sum_cd X_{ij,cd} V_{mb,cd}
    for pair-symmetric X and a V without symmetry in (mb): canonical ij and
    cd only, Y_ij = S+ + S-, Y_ji = S+ - S-, two products at half the
    flops."""
    no, nv = len(oi), len(vi)
    Y = np.zeros((no, no) + V.shape[:2])
    R = _canonical(oi)
    C = _canonical(vi)
    for G in range(max(oi.max(), vi.max()) + 1):
        RG = [(i, j) for (i, j) in R if oi[i] ^ oi[j] == G]
        CG = [(c, d) for (c, d) in C if vi[c] ^ vi[d] == G]
        if not RG or not CG:
            continue
        Ap = np.array([[0.5 * (X[i, j, c, d] + X[i, j, d, c]) for c, d in CG]
                       for i, j in RG])
        Am = np.array([[0.5 * (X[i, j, c, d] - X[i, j, d, c]) for c, d in CG]
                       for i, j in RG])
        Wp = np.stack([V[:, :, c, d] + (V[:, :, d, c] if c != d else 0.0)
                       for c, d in CG], axis=-1)
        Wm = np.stack([V[:, :, c, d] - V[:, :, d, c] for c, d in CG],
                      axis=-1)
        Sp = np.einsum("ru,mbu->rmb", Ap, Wp)
        Sm = np.einsum("ru,mbu->rmb", Am, Wm)
        for r, (i, j) in enumerate(RG):
            Y[i, j] += Sp[r] + Sm[r]
            if i != j:
                Y[j, i] += Sp[r] - Sm[r]
    return Y


def test_partial_pm_packing_reproduces_the_product():
    # the O(o^3 v^3) product sum_cd tau_ij^cd (mc|bd) of the residual's
    # T1 terms, in the partial +/- form
    for seed, occ, vir, nq in [(1, [2, 1], [3, 2], [4, 3]),
                               (2, [2, 1, 1, 1], [3, 2, 2, 1], [3, 2, 2, 2])]:
        oi, vi, X, _ = _system(seed, occ, vir, nq)
        rng = np.random.default_rng(seed)
        # V[m,b,c,d] stands for (mc|bd); the identity uses only the pair
        # symmetry of X, so any V with a block pattern will do
        V = rng.standard_normal((len(oi), len(vi), len(vi), len(vi)))
        V *= ((oi[:, None, None, None] ^ vi[None, :, None, None]) ==
              (vi[None, None, :, None] ^ vi[None, None, None, :]))
        ref = np.einsum("ijcd,mbcd->ijmb", X, V)
        got = _partial_pm(oi, vi, X, V)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), seed
