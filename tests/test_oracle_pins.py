"""Pins of the FP64 oracle against what theory fixes (CPU only).

Each test ties the oracle to something other than itself:
  * brute-force projections <mu|exp(-T) H exp(T)|0> in a determinant basis,
  * exact two-electron FCI and Hellmann-Feynman derivatives (o = 1),
  * the closed-form MP2 energy,
  * central finite differences of the energy,
  * invariances (orbital rotations, Cholesky-vector rotations, symmetry),
  * Euler's theorem for the degree-2 homogeneity of the energy in L,
  * a pivoted Cholesky factorisation (LAPACK dpstrf) of the ERI matrix.
"""
import numpy as np
import pytest
import scipy.linalg
import torch

from synth import (random_system, unpack_dense, pack_dense, make_system,
                   make_displacements, make_displacement_nontotsym,
                   irrep_split, chol_split)
from oracle import brute, ccsd, model, lagrangian, fci2, mp2, rows

DT = torch.float64


def T(x):
    return torch.as_tensor(np.asarray(x), dtype=DT)


def _sys_dense(s):
    L = unpack_dense(s, s.L)
    h = model.core_from_eps(T(s.eps), T(L), s.nocc)
    return L, h


def _random_amps(rng, o, v, scale=0.1):
    t1 = rng.standard_normal((o, v)) * scale
    t2 = rng.standard_normal((o, o, v, v)) * scale
    return t1, 0.5 * (t2 + t2.transpose(1, 0, 3, 2))


# ---------------------------------------------------------------- generator
def test_generator_splits():
    assert irrep_split(60, 8, "even") == [8, 8, 8, 8, 7, 7, 7, 7]
    assert irrep_split(540, 8, "even") == [68] * 4 + [67] * 4
    assert irrep_split(40, 4, (0.4, 0.25, 0.2, 0.15)) == [16, 10, 8, 6]
    assert irrep_split(360, 4, (0.4, 0.25, 0.2, 0.15)) == [144, 90, 72, 54]
    assert chol_split(1600, 4, [160, 100, 80, 60]) == [456, 416, 376, 352]
    s = make_system(1)
    assert s.chol == [80] * 8 and s.occ == [2] * 8 and s.vir == [18] * 8


def test_pack_roundtrip_and_pattern():
    s = random_system([2, 1, 1, 0], [3, 2, 1, 2], [5, 3, 4, 2], seed=3)
    d = unpack_dense(s, s.L)
    assert np.array_equal(pack_dense(s, d), s.L)
    assert np.allclose(d, d.transpose(0, 2, 1))
    for P in range(s.nchol):
        for p in range(s.n):
            for q in range(s.n):
                if s.orb_irrep[p] ^ s.orb_irrep[q] != s.chol_irrep[P]:
                    assert d[P, p, q] == 0.0


# ---------------------------------------------------------------- Eq. 1
def test_cholesky_reconstructs_eri():
    s = random_system([1, 1], [2, 2], [4, 3], seed=11)
    L = unpack_dense(s, s.L)
    n = s.n
    g = model.eri(T(L)).numpy()
    M = g.reshape(n * n, n * n)
    assert np.allclose(M, M.T, atol=1e-14)
    # pivoted Cholesky of the ERI supermatrix: PSD, rank <= nL, exact
    c, piv, rank, info = scipy.linalg.lapack.dpstrf(M + 0.0, lower=1,
                                                    tol=1e-13)
    assert rank <= s.nchol
    Lc = np.tril(c)[:, :rank]
    Pm = np.eye(n * n)[:, piv - 1]
    assert np.abs(Pm @ Lc @ Lc.T @ Pm.T - M).max() < 1e-12
    # selection rule: (pq|rs) = 0 unless irrep(pq) == irrep(rs)
    ir = s.orb_irrep
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for t in range(n):
                    if ir[p] ^ ir[q] != ir[r] ^ ir[t]:
                        assert g[p, q, r, t] == 0.0


# ------------------------------------------------ amplitude equations (pin)
CASES = [((2,), (3,), (6,), 1), ((1, 1), (2, 1), (3, 3), 2),
         ((1,), (4,), (5,), 3), ((2, 1), (1, 1), (4, 2), 4)]


@pytest.mark.parametrize("occ,vir,chol,seed", CASES)
def test_residual_equals_determinant_projection(occ, vir, chol, seed):
    s = random_system(list(occ), list(vir), list(chol), seed=seed, scale=0.8)
    L = unpack_dense(s, s.L)
    rng = np.random.default_rng(seed)
    n, o, v = s.n, s.nocc, s.nvir
    h = rng.standard_normal((n, n)) * 0.3
    h = 0.5 * (h + h.T)                      # non-canonical, f_ia != 0
    t1, t2 = _random_amps(rng, o, v, 0.15)
    Eb, R1b, R2b = brute.projections(h, L, o, t1, t2)
    R1, R2, E = ccsd.residual(T(t1), T(t2), T(h), T(L), o)
    assert abs(E.item() - Eb) < 1e-12
    assert np.abs(R1.numpy() - R1b).max() < 1e-12
    assert np.abs(R2.numpy() - R2b).max() < 1e-12


def test_planted_mistake_is_caught(monkeypatch):
    """A 1% error in the ladder term must break the projection pin."""
    s = random_system([2], [3], [5], seed=9, scale=0.8)
    L = unpack_dense(s, s.L)
    rng = np.random.default_rng(9)
    h = np.diag(s.eps)
    t1, t2 = _random_amps(rng, 2, 3, 0.2)
    _, _, R2b = brute.projections(h, L, 2, t1, t2)
    good = ccsd.ladder
    monkeypatch.setattr(ccsd, "ladder",
                        lambda t, vv, *a: 0.99 * good(t, vv, *a))
    _, R2, _ = ccsd.residual(T(t1), T(t2), T(h), T(L), 2)
    assert np.abs(R2.numpy() - R2b).max() > 1e-5


def test_mp2_first_iteration():
    s = random_system([3], [7], [10], seed=3, scale=0.5)
    L, h = _sys_dense(s)
    o, v = 3, 7
    f = model.fock(h, T(L), o)
    Dia, Dijab = ccsd.denominators(f, o)
    z1, z2 = torch.zeros(o, v, dtype=DT), torch.zeros(o, o, v, v, dtype=DT)
    R1, R2, _ = ccsd.residual(z1, z2, h, T(L), o)
    assert (R1 / Dia).abs().max().item() < 1e-14      # f_ia = 0
    e = ccsd.energy_corr(z1, R2 / Dijab, h, T(L), o)
    assert abs(e - mp2.mp2_energy(s.eps, L, o)) < 1e-13


# ------------------------------------------------ two electrons: CCSD = FCI
@pytest.mark.parametrize("occ,vir,chol,seed", [((1,), (9,), (12,), 5),
                                               ((1, 0, 0, 0), (3, 2, 2, 1),
                                                (5, 3, 3, 3), 6)])
def test_ccsd_is_fci_for_two_electrons(occ, vir, chol, seed):
    s = random_system(list(occ), list(vir), list(chol), seed=seed, scale=0.6)
    L, h = _sys_dense(s)
    r = lagrangian.run_all(h, T(L), 1, tol=1e-12, e_tol=1e-13)
    E_fci, C = fci2.singlet_fci(h.numpy(), L)
    assert abs(r["cc"]["E"] - E_fci) < 1e-11
    # Hellmann-Feynman with h fixed: the Lambda gradient is exact
    dL = np.stack([unpack_dense(s, x) for x in make_displacements(s, 3)])
    g = lagrangian.gradient_from_density(r["G"], T(dL)).numpy()
    g_hf = fci2.hellmann_feynman(C, L, dL)
    assert np.abs(g - g_hf).max() < 1e-11


def test_two_electron_fci_matches_determinants():
    s = random_system([1], [3], [4], seed=21, scale=0.7)
    L, h = _sys_dense(s)
    E_fci, _ = fci2.singlet_fci(h.numpy(), L)
    assert abs(E_fci - brute.fci_ground_energy(h.numpy(), L, 1)) < 1e-12


# ------------------------------------------------ gradient vs finite diff.
def _fd_gradient(h, L, o, dL, steps=(1e-3, 5e-4)):
    def energy(x):
        return ccsd.solve_ccsd(h, T(L + x * dL), o, tol=1e-13,
                               e_tol=1e-14)["E"]
    fd = [(energy(s) - energy(-s)) / (2 * s) for s in steps]
    return (4.0 * fd[1] - fd[0]) / 3.0            # Richardson


@pytest.mark.parametrize("which", ["c0", "sym"])
def test_gradient_matches_finite_difference(which):
    if which == "c0":
        s = make_system(0)
        nx = 2
    else:
        s = random_system([2, 1, 1, 1], [4, 3, 3, 2], [8, 6, 6, 6], seed=13,
                          scale=0.35)
        nx = 2
    L, h = _sys_dense(s)
    o = s.nocc
    dL = np.stack([unpack_dense(s, x) for x in make_displacements(s, nx)])
    r = lagrangian.run_all(h, T(L), o, tol=1e-12, e_tol=1e-13)
    g = lagrangian.gradient_from_density(r["G"], T(dL)).numpy()
    for x in range(nx):
        assert abs(g[x] - _fd_gradient(h, L, o, dL[x])) < 1e-8


# ------------------------------------------------ symmetry
def test_non_totally_symmetric_displacement_gives_zero():
    s = random_system([1, 1, 1, 0], [3, 2, 2, 2], [6, 4, 4, 4], seed=17,
                      scale=0.5)
    L, h = _sys_dense(s)
    r = lagrangian.run_all(h, T(L), s.nocc, tol=1e-11)
    G = r["G"]
    for gx in (1, 2, 3):
        dL = unpack_dense(s, make_displacement_nontotsym(s, gx), gx=gx)
        assert np.abs(dL).max() > 0
        g = lagrangian.gradient_from_density(G, T(dL[None])).item()
        assert abs(g) < 1e-13
    # densities and amplitudes respect the selection rule
    ir, cir, o = s.orb_irrep, s.chol_irrep, s.nocc
    Gn = G.numpy()
    mask = (ir[None, :, None] ^ ir[None, None, :]) != cir[:, None, None]
    assert np.abs(Gn[mask]).max() < 1e-14
    t2 = r["cc"]["t2"].numpy()
    io, iv = ir[:o], ir[o:]
    m2 = (io[:, None, None, None] ^ io[None, :, None, None]
          ^ iv[None, None, :, None] ^ iv[None, None, None, :]) != 0
    assert np.abs(t2[m2]).max() < 1e-14


def test_lambda_is_symmetric():
    s = random_system([2], [4], [6], seed=31, scale=0.5)
    L, h = _sys_dense(s)
    r = lagrangian.run_all(h, T(L), 2, tol=1e-11)
    l2 = r["lam"]["l2"]
    assert (l2 - l2.permute(1, 0, 3, 2)).abs().max().item() < 1e-13


# ------------------------------------------------ invariances
def _rot(rng, k):
    q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return q


def test_orbital_rotation_invariance():
    s = random_system([3], [6], [9], seed=41, scale=0.5)
    L, h = _sys_dense(s)
    o, n = 3, s.n
    dL = unpack_dense(s, make_displacements(s, 1)[0])
    r0 = lagrangian.run_all(h, T(L), o, tol=1e-12, e_tol=1e-13)
    g0 = lagrangian.gradient_from_density(r0["G"], T(dL[None])).item()
    rng = np.random.default_rng(5)
    U = scipy.linalg.block_diag(_rot(rng, o), _rot(rng, n - o))
    Lr = np.einsum("pi,Ppq,qj->Pij", U, L, U)
    dLr = np.einsum("pi,Ppq,qj->Pij", U, dL, U)
    hr = T(U.T @ h.numpy() @ U)
    r1 = lagrangian.run_all(hr, T(Lr), o, tol=1e-12, e_tol=1e-13)
    g1 = lagrangian.gradient_from_density(r1["G"], T(dLr[None])).item()
    assert abs(r0["cc"]["E"] - r1["cc"]["E"]) < 1e-11
    assert abs(g0 - g1) < 1e-10


def test_cholesky_vector_rotation_invariance():
    """The CD is not unique (Sec. 2.1): any orthogonal mixing of the vectors
    leaves (pq|rs), hence E and the gradient, unchanged."""
    s = random_system([2], [5], [7], seed=43, scale=0.5)
    L, h = _sys_dense(s)
    dL = np.stack([unpack_dense(s, x) for x in make_displacements(s, 2)])
    O = _rot(np.random.default_rng(3), s.nchol)
    r0 = lagrangian.run_all(h, T(L), 2, tol=1e-12, e_tol=1e-13)
    r1 = lagrangian.run_all(h, T(np.einsum("PQ,Qpq->Ppq", O, L)), 2,
                            tol=1e-12, e_tol=1e-13)
    g0 = lagrangian.gradient_from_density(r0["G"], T(dL)).numpy()
    g1 = lagrangian.gradient_from_density(
        r1["G"], T(np.einsum("PQ,xQpq->xPpq", O, dL))).numpy()
    assert abs(r0["cc"]["E"] - r1["cc"]["E"]) < 1e-11
    assert np.abs(g0 - g1).max() < 1e-10


def test_euler_identity():
    """With the densities fixed, the energy is homogeneous of degree 2 in L:
    sum_P <Gamma^P, L^P> = 2 (E - sum_pq D_pq h_pq)."""
    s = random_system([2, 1], [4, 3], [6, 5], seed=47, scale=0.5)
    L, h = _sys_dense(s)
    r = lagrangian.run_all(h, T(L), s.nocc, tol=1e-12, e_tol=1e-13)
    lhs = float(np.sum(r["G"].numpy() * L))
    rhs = 2.0 * (r["cc"]["E"] - float(np.sum(r["D"].numpy() * h.numpy())))
    assert abs(lhs - rhs) < 1e-11
    # the 1-RDM traces to the electron count
    assert abs(np.trace(r["D"].numpy()) - 2 * s.nocc) < 1e-11


@pytest.mark.parametrize("occ,vir,chol,seed", CASES)
def test_rows_and_energy_equal_determinant_projection(occ, vir, chol, seed):
    """oracle.rows (residual rows and energy without the full ladder) against
    the brute-force projections, on unsymmetrised t2 and non-canonical h."""
    s = random_system(list(occ), list(vir), list(chol), seed=seed, scale=0.8)
    L = unpack_dense(s, s.L)
    rng = np.random.default_rng(seed + 50)
    n, o, v = s.n, s.nocc, s.nvir
    h = rng.standard_normal((n, n)) * 0.3
    h = 0.5 * (h + h.T)
    t1 = rng.standard_normal((o, v)) * 0.15
    t2 = rng.standard_normal((o, o, v, v)) * 0.15
    Eb, R1b, R2b = brute.projections(h, L, o, t1,
                                     0.5 * (t2 + t2.transpose(1, 0, 3, 2)))
    assert abs(rows.energy(T(t1), T(t2), T(h), T(L), o) - Eb) < 1e-12
    pairs = [(i, j) for i in range(o) for j in range(o)]
    R1, R2 = rows.residual_rows(T(t1), T(t2), T(h), T(L), o, pairs)
    assert np.abs(R1.numpy() - R1b).max() < 1e-12
    for p in pairs:
        assert np.abs(R2[p].numpy() - R2b[p]).max() < 1e-12


def test_rows_planted_mistake_is_caught(monkeypatch):
    """Dropping the ladder from the row evaluation breaks the projection pin."""
    s = random_system([2], [3], [5], seed=11, scale=0.8)
    L = unpack_dense(s, s.L)
    rng = np.random.default_rng(11)
    h = np.diag(s.eps)
    t1, t2 = _random_amps(rng, 2, 3, 0.2)
    _, _, R2b = brute.projections(h, L, 2, t1, t2)
    real = torch.matmul
    calls = {"n": 0}

    def no_ladder(a, b):                       # zero the PPL product
        calls["n"] += 1
        r = real(a, b)
        return r * 0.0 if a.dim() == 3 else r
    monkeypatch.setattr(rows.torch, "matmul", no_ladder)
    _, R2 = rows.residual_rows(T(t1), T(t2), T(h), T(L), 2, [(0, 1)])
    assert calls["n"] > 0
    assert np.abs(R2[(0, 1)].numpy() - R2b[0, 1]).max() > 1e-4


def test_raw_c0_diverges():
    """The literal distribution (s = 1) gives E_MP2 = -37 Eh for c0 and the
    CCSD iterations diverge (the reason for the energy scale s_cfg)."""
    s = make_system(0, scale=1.0)
    L, h = _sys_dense(s)
    assert mp2.mp2_energy(s.eps, L, s.nocc) < -30.0
    with pytest.raises(Exception):
        ccsd.solve_ccsd(T(h), T(L), s.nocc, tol=1e-10, maxiter=60, ndiis=0)


@pytest.mark.parametrize("which", ["c0", "sym"])
def test_frozen_fock_gradient_matches_finite_difference(which):
    """FROZEN_FOCK: f = diag(eps) at every displacement (h rebuilt from L)
    and E = E_corr; Gamma_FF . dL equals the central difference of E_corr."""
    if which == "c0":
        s = make_system(0)
    else:
        s = random_system([2, 1, 1, 1], [4, 3, 3, 2], [8, 6, 6, 6], seed=13,
                          scale=0.35)
    L, h = _sys_dense(s)
    o = s.nocc
    eps = T(s.eps)
    dL = np.stack([unpack_dense(s, x) for x in make_displacements(s, 2)])
    r = lagrangian.run_all(h, T(L), o, tol=1e-12, e_tol=1e-13)
    G = lagrangian.density_frozen_fock(r["cc"]["t1"], r["cc"]["t2"],
                                       r["lam"]["l1"], r["lam"]["l2"], eps,
                                       T(L), o)
    g = lagrangian.gradient_from_density(G, T(dL)).numpy()

    def ecorr(x, d):
        Lx = T(L + x * d)
        hx = model.core_from_eps(eps, Lx, o)
        return ccsd.solve_ccsd(hx, Lx, o, tol=1e-13, e_tol=1e-14)["E_corr"]

    for k in range(2):
        fd = [(ecorr(st, dL[k]) - ecorr(-st, dL[k])) / (2 * st)
              for st in (1e-3, 5e-4)]
        assert abs(g[k] - (4.0 * fd[1] - fd[0]) / 3.0) < 1e-8
    # and it differs from the default model's gradient (h fixed)
    g_fc = lagrangian.gradient_from_density(r["G"], T(dL)).numpy()
    assert np.abs(g - g_fc).max() > 1e-4


def test_rows_equal_full_residual_on_a_larger_symmetric_case():
    """Beyond brute-force sizes: oracle.rows reproduces every row of the
    (brute-force-pinned) full residual on a D2h case with ragged irreps."""
    s = random_system([2, 1, 1, 1, 1, 0, 1, 0], [5, 4, 3, 3, 2, 3, 2, 2],
                      [9, 7, 7, 6, 6, 6, 6, 5], seed=77, scale=0.4)
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, s.nocc)
    o, v = s.nocc, s.nvir
    rng = np.random.default_rng(77)
    t1 = T(rng.standard_normal((o, v)) * 0.05)
    t2 = T(rng.standard_normal((o, o, v, v)) * 0.05)
    R1f, R2f, Ef = ccsd.residual(t1, t2, h, L, o)
    assert abs(rows.energy(t1, t2, h, L, o) - Ef.item()) < 1e-12
    pairs = [(i, j) for i in range(o) for j in range(o)]
    R1, R2 = rows.residual_rows(t1, t2, h, L, o, pairs)
    assert (R1 - R1f).abs().max().item() < 1e-12
    for (i, j) in pairs:
        assert (R2[(i, j)] - R2f[i, j]).abs().max().item() < 1e-12


# ------------------------------------------- workload energy scales (s_cfg)
@pytest.mark.parametrize("occ,vir,chol,seed", [((3,), (9,), (14,), 21),
                                               ((2, 1, 2, 0), (4, 3, 3, 2),
                                                (6, 4, 5, 3), 22)])
def test_scale_calibration_mp2_equals_closed_form(occ, vir, chol, seed):
    # the calibration script's chunked MP2 over the packed L_ov block equals
    # the closed-form MP2 energy on the dense vectors (C1 and symmetric)
    from oracle import calibrate_scale
    s = random_system(list(occ), list(vir), list(chol), seed=seed, scale=0.7)
    L = unpack_dense(s, s.L)
    e_closed = mp2.mp2_energy(s.eps, L, s.nocc)
    Lov = calibrate_scale._ov_dense(s)
    assert np.array_equal(Lov, L[:, :s.nocc, s.nocc:])
    e_chunk = calibrate_scale.mp2_chunked(s.eps, Lov)
    assert abs(e_chunk - e_closed) <= 1e-12 * abs(e_closed)


def test_stored_scale_gives_target_mp2_energy():
    # E_MP2 is homogeneous of degree 4 in L, so the stored s_cfg of the
    # smallest workload must reproduce the target -0.04 Eh per occupied
    # orbital with the closed form on the scaled arrays
    s = make_system(0)
    L = unpack_dense(s, s.L)
    e = mp2.mp2_energy(s.eps, L, s.nocc)
    assert abs(e - (-0.04 * s.nocc)) < 1e-10


# ------------------------------------- DF / Cholesky three-term gradient
def _df_case(s, nx=2):
    from synth.df import make_df_inputs
    M, Kp, dB, dM = make_df_inputs(s, nx)
    L, h = _sys_dense(s)
    # three-index integrals of this workload: B = K L per irrep block, with
    # K the Cholesky factor of the metric (Eq. cv_2ndstep read backwards)
    B = np.zeros_like(L)
    P0, off = 0, 0
    for n in s.chol:
        K = np.linalg.cholesky(M[off:off + n * n].reshape(n, n))
        B[P0:P0 + n] = (K @ L[P0:P0 + n].reshape(n, -1)).reshape(n, *L.shape[1:])
        P0 += n
        off += n * n
    dBd = np.stack([unpack_dense(s, x) for x in dB])
    return L, h, M, dM, B, dBd


def _vectors_of(s, M, B):
    """L = K^{-1} B per irrep block (numpy, for the finite differences)."""
    L = np.zeros_like(B)
    P0, off = 0, 0
    for n in s.chol:
        K = np.linalg.cholesky(M[off:off + n * n].reshape(n, n))
        L[P0:P0 + n] = scipy.linalg.solve_triangular(
            K, B[P0:P0 + n].reshape(n, -1), lower=True).reshape(
                n, *B.shape[1:])
        P0 += n
        off += n * n
    return L


@pytest.mark.parametrize("occ,vir,chol,seed", [((3,), (7,), (12,), 61),
                                               ((2, 1, 1, 1), (4, 3, 3, 2),
                                                (8, 6, 6, 5), 62)])
def test_df_gradient_equals_differentiated_vector_form(occ, vir, chol, seed):
    from oracle import df
    s = random_system(list(occ), list(vir), list(chol), seed=seed, scale=0.4)
    L, h, M, dM, B, dB = _df_case(s)
    assert np.abs(_vectors_of(s, M, B) - L).max() < 1e-13
    r = lagrangian.run_all(h, T(L), s.nocc, tol=1e-12, e_tol=1e-13)
    g = df.df_gradient(r["G"], T(L), M, s.chol, T(dB), T(dM)).numpy()
    for x in range(2):
        # dL/dx of L(x) = chol(M + x dM)^{-1} (B + x dB), Richardson
        fd = []
        for step in (1e-3, 5e-4):
            Lp = _vectors_of(s, M + step * dM[x], B + step * dB[x])
            Lm = _vectors_of(s, M - step * dM[x], B - step * dB[x])
            fd.append((Lp - Lm) / (2 * step))
        dL = (4.0 * fd[1] - fd[0]) / 3.0
        ref = float(np.sum(r["G"].numpy() * dL))
        assert abs(g[x] - ref) < 1e-9, (x, g[x], ref)
    # a planted mistake in the metric term is caught
    g_bad = df.df_gradient(r["G"], T(L), M, s.chol, T(dB), T(2.0 * dM))
    assert np.abs(g_bad.numpy() - g).max() > 1e-4


def test_df_gradient_matches_energy_finite_difference():
    from oracle import df
    s = random_system([2, 1, 1, 1], [4, 3, 3, 2], [8, 6, 6, 5], seed=63,
                      scale=0.4)
    L, h, M, dM, B, dB = _df_case(s)
    o = s.nocc
    r = lagrangian.run_all(h, T(L), o, tol=1e-12, e_tol=1e-13)
    g = df.df_gradient(r["G"], T(L), M, s.chol, T(dB), T(dM)).numpy()

    def energy(x, k):
        Lx = _vectors_of(s, M + x * dM[k], B + x * dB[k])
        return ccsd.solve_ccsd(h, T(Lx), o, tol=1e-13, e_tol=1e-14)["E"]
    for k in range(2):
        fd = [(energy(st, k) - energy(-st, k)) / (2 * st)
              for st in (1e-3, 5e-4)]
        assert abs(g[k] - (4.0 * fd[1] - fd[0]) / 3.0) < 1e-8
