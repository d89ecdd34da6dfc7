"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path).  Both sides converge max|R/D| to 1e-12 here; the
amplitudes then agree to ~1e-11 and the energy (quadratic in the amplitude
error at a stationary Lagrangian, linear otherwise) to well below 1e-10 Eh.
  energy        |dE|        <= 1e-10 Eh
  gradient      |dg_x|      <= 1e-9  Eh per unit displacement
  t, lambda     max |d|     <= 1e-9
  Gamma^P       max |d|     <= 1e-9
"""
import json
import os

import numpy as np
import pytest
import torch

from synth import (make_system, random_system, make_displacements,
                   make_displacement_nontotsym, unpack_dense, pack_dense,
                   as_c1)
from oracle import model, lagrangian

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def oracle_run(s, tol=1e-12):
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
    r = lagrangian.run_all(h, L, s.nocc, tol=tol, e_tol=1e-13)
    return r


def gpu_run(cd, s, dL, tol=1e-12, **opt):
    o = cd.cdcc_default_options()
    o.conv_tol = tol
    o.energy_tol = 1e-13
    for k, v in opt.items():
        setattr(o, k, v)
    ctx = cd.init_from_system(s, options=o)
    e, it, res = cd.ccsd_solve(ctx)
    lit, lres = cd.lambda_solve(ctx)
    D1 = cd.build_density(ctx, s.n)
    g = cd.contract_dL(ctx, dL)
    out = dict(e=e, it=it, lit=lit, D1=D1, g=g,
               G=cd.cdcc_get_gamma(ctx),
               t1=cd.cdcc_get_amplitudes(ctx, 0, s.nocc, s.nvir),
               t2=cd.cdcc_get_amplitudes(ctx, 1, s.nocc, s.nvir),
               l1=cd.cdcc_get_amplitudes(ctx, 2, s.nocc, s.nvir),
               l2=cd.cdcc_get_amplitudes(ctx, 3, s.nocc, s.nvir),
               launches=cd.cdcc_kernel_launches(ctx))
    cd.cd_ccsd_free(ctx)
    return out


def compare(s, r, gg, dL):
    G_or = pack_dense(s, r["G"].numpy())
    g_or = dL @ G_or
    assert abs(gg["e"] - r["cc"]["E_corr"]) < 1e-10, (gg["e"], r["cc"]["E_corr"])
    assert np.abs(gg["t1"] - r["cc"]["t1"].numpy()).max() < 1e-9
    assert np.abs(gg["t2"] - r["cc"]["t2"].numpy()).max() < 1e-9
    assert np.abs(gg["l1"] - r["lam"]["l1"].numpy()).max() < 1e-9
    assert np.abs(gg["l2"] - r["lam"]["l2"].numpy()).max() < 1e-9
    assert np.abs(gg["G"] - G_or).max() < 1e-9
    assert np.abs(gg["g"] - g_or).max() < 1e-9
    assert np.abs(gg["D1"] - r["D"].numpy()).max() < 1e-9


def test_c0_matches_oracle(cd):
    s = make_system(0)
    dL = make_displacements(s)
    r = oracle_run(s)
    gg = gpu_run(cd, s, dL)
    compare(s, r, gg, dL)
    assert gg["launches"] > 0


@pytest.mark.parametrize("occ,vir,chol,seed", [
    ([2, 1, 1, 0], [5, 3, 4, 2], [9, 7, 6, 6], 101),   # empty occ irrep
    ([1, 1, 0, 0, 1, 0, 1, 0], [3, 2, 2, 3, 1, 2, 2, 1], [5, 3, 3, 3, 3, 3,
                                                          3, 2], 102),
    ([3, 2], [7, 5], [11, 9], 103),
])
def test_symmetric_ragged_matches_oracle(cd, occ, vir, chol, seed):
    s = random_system(occ, vir, chol, seed=seed, scale=0.45)
    dL = make_displacements(s, 3)
    r = oracle_run(s)
    gg = gpu_run(cd, s, dL)
    compare(s, r, gg, dL)


def test_two_electrons_tiny(cd):
    s = random_system([1], [1], [1], seed=7, scale=0.5)
    dL = make_displacements(s, 1)
    r = oracle_run(s)
    gg = gpu_run(cd, s, dL)
    compare(s, r, gg, dL)


def test_nontotally_symmetric_displacements_vanish(cd):
    s = random_system([1, 1, 1, 1], [3, 3, 2, 2], [6, 5, 5, 4], seed=5,
                      scale=0.4)
    d0 = make_displacements(s, 1)[0]
    d1 = make_displacement_nontotsym(s, 2)
    buf = np.concatenate([d0, d1, d0])
    ctx = cd.init_from_system(s)
    e, g = cd.gradient(ctx, buf, nx=3, x_irrep=[0, 2, 0])
    cd.cd_ccsd_free(ctx)
    assert g[1] == 0.0 and abs(g[0] - g[2]) < 1e-14 and g[0] != 0.0


def test_bounded_wait_gives_up_and_device_stays_usable(cd):
    """Failure detection without a GPU fault: a wait that nothing completes
    runs out, is reported as CDCC_ETIMEOUT, and work continues."""
    assert cd.cdcc_selftest_bounded_wait() == cd.CDCC_ETIMEOUT
    s = random_system([1], [2], [3], seed=19, scale=0.4)
    ctx = cd.init_from_system(s)
    e, g = cd.gradient(ctx, make_displacements(s, 1))
    cd.cd_ccsd_free(ctx)
    assert np.isfinite(e) and np.all(np.isfinite(g))


@pytest.mark.parametrize("which", ["c0", "ragged"])
def test_frozen_fock_matches_oracle(cd, which):
    """cdcc_options.fock_model = FROZEN_FOCK (Fock matrix kept at diag(eps)
    under a displacement, E = E_corr) against the oracle's Gamma_FF, which
    its own finite-difference pin fixes."""
    if which == "c0":
        s = make_system(0)
    else:
        s = random_system([3, 2], [7, 5], [11, 9], seed=103, scale=0.45)
    dL = make_displacements(s, 3)
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
    r = lagrangian.run_all(h, L, s.nocc, tol=1e-12, e_tol=1e-13)
    Gff = lagrangian.density_frozen_fock(r["cc"]["t1"], r["cc"]["t2"],
                                         r["lam"]["l1"], r["lam"]["l2"],
                                         s.eps, L, s.nocc)
    G_or = pack_dense(s, Gff.numpy())
    gg = gpu_run(cd, s, dL, fock_model=cd.FROZEN_FOCK)
    assert abs(gg["e"] - r["cc"]["E_corr"]) < 1e-10
    assert np.abs(gg["G"] - G_or).max() < 1e-9
    assert np.abs(gg["g"] - dL @ G_or).max() < 1e-9


def test_raw_c0_divergence_is_reported(cd):
    """c0 with the literal Cholesky distribution (s = 1, E_MP2 = -37 Eh) is
    the strong-correlation stress case: the oracle's CCSD diverges on it
    (plain Jacobi reaches NaN, DIIS turns singular).  The library must end
    with an error status, not hang or return a number, and stay usable."""
    s = make_system(0, scale=1.0)
    ctx = cd.init_from_system(s)
    with pytest.raises(cd.CdccError) as ei:
        cd.ccsd_solve(ctx)
    assert ei.value.status in (cd.CDCC_ENUMERIC, cd.CDCC_ENOCONV)
    cd.cd_ccsd_free(ctx)
    t = random_system([1], [2], [3], seed=23, scale=0.4)
    ctx = cd.init_from_system(t)
    e, g = cd.gradient(ctx, make_displacements(t, 1))
    cd.cd_ccsd_free(ctx)
    assert np.isfinite(e) and np.all(np.isfinite(g))


def test_call_order_enforced(cd):
    s = random_system([1], [2], [3], seed=9, scale=0.4)
    ctx = cd.init_from_system(s)
    with pytest.raises(cd.CdccError) as ei:
        cd.lambda_solve(ctx)
    assert ei.value.status == cd.CDCC_ESTATE
    with pytest.raises(cd.CdccError):
        cd.contract_dL(ctx, make_displacements(s, 1))
    cd.cd_ccsd_free(ctx)


def test_device_and_host_inputs_agree(cd):
    s = make_system(0)
    dL = make_displacements(s)
    ctx = cd.init_from_system(s)
    e1, g1 = cd.gradient(ctx, dL)
    g2 = cd.contract_dL(ctx, torch.as_tensor(dL, device="cuda"))
    cd.cd_ccsd_free(ctx)
    ctx = cd.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol, s.orb_irrep,
                          s.eps, s.chol_irrep,
                          torch.as_tensor(s.L, device="cuda"))
    e3, g3 = cd.gradient(ctx, dL)
    cd.cd_ccsd_free(ctx)
    assert np.array_equal(g1, g2)
    assert e1 == e3 and np.array_equal(g1, g3)


# ------------------------------------------------ full-size workload (c1)
def test_c1_symmetric_equals_c1_run_and_oracle(cd):
    s = make_system(1)
    dL = make_displacements(s)
    gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
    ctx = cd.init_from_system(s)
    e, it, res = cd.ccsd_solve(ctx)
    cd.lambda_solve(ctx)
    cd.build_density(ctx)
    g = cd.contract_dL(ctx, dL)
    G = cd.cdcc_get_gamma(ctx)
    t2 = cd.cdcc_get_amplitudes(ctx, 1, s.nocc, s.nvir).reshape(-1)
    l2 = cd.cdcc_get_amplitudes(ctx, 3, s.nocc, s.nvir).reshape(-1)
    cd.cd_ccsd_free(ctx)
    # against the stored FP64 oracle values (tests/golden/make_golden.py)
    assert abs(e - gold["e_corr"]) < 1e-9
    assert np.abs(g - np.array(gold["gradient"])).max() < 1e-8
    gi = np.array(gold["gamma_index"])
    assert np.abs(G[gi] - np.array(gold["gamma_value"])).max() < 1e-9
    ti = np.array(gold["t2_index"])
    assert np.abs(t2[ti] - np.array(gold["t2_value"])).max() < 1e-9
    assert np.abs(l2[ti] - np.array(gold["l2_value"])).max() < 1e-9
    # the same data with symmetry ignored (C1), on the GPU
    c1, (dL1,) = as_c1(s, [dL[0]])
    ctx = cd.init_from_system(c1)
    e1, g1 = cd.gradient(ctx, dL1[None])
    cd.cd_ccsd_free(ctx)
    assert abs(e1 - e) < 1e-10
    assert abs(g1[0] - g[0]) < 1e-9
