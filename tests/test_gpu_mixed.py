"""Tensor-core split-precision GEMM and the MIXED precision path (GPU).

Kernel level: cdcc_dgemm in every mode against an FP64 product computed
with numpy, error normalised by the magnitude bound |A||B| (so the bound is
independent of cancellation):
  mode 0 (FP64 DFMA)          <= 1e-14
  mode 1 (1 BF16 slice)       <= 1e-2     (8 significant bits)
  mode 2 (2 slices, 3 prods)  <= 2e-5     (~16 bits + FP32 accumulation)
  mode 3 (3 slices, 6 prods)  <= 2e-6     (FP32-class accumulation)
End to end: the MIXED schedule (tensor-core contractions, FP64 finish) must
meet the target accuracy against the FP64 oracle: |dE| <= 1e-8 Eh and
|dg_x| <= 1e-6 Eh per unit displacement.
"""
import json
import os

import numpy as np
import pytest
import torch

from synth import make_system, make_displacements, random_system, pack_dense
from synth import unpack_dense

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = {0: 1e-14, 1: 1e-2, 2: 2e-5, 3: 2e-6}


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    cbuild.build()
    return cdcc


SHAPES = [(1, 1, 1), (5, 3, 7), (128, 128, 64), (200, 37, 300),
          (32, 700, 650), (300, 290, 5000), (129, 257, 77), (64, 32, 1000),
          (1, 1, 5000), (7, 9, 9000),
          # one output side <= 16 (the narrow FP64 kernel): large M or large
          # N, short K, long K split over CTAs, small sides 4, 8 and 16
          (3000, 8, 8), (8, 3000, 68), (68, 8, 30000), (16, 700, 40),
          (2000, 4, 100), (7, 1000, 20000), (300, 16, 1500),
          # both sides <= 16 with the smaller one first, short K
          (3, 10, 50), (10, 3, 50), (12, 16, 700),
          # small output, long K: the exact-slice kernel splits K over the
          # SMs (fixed-order reduction of the parts)
          (67, 67, 60000)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_dgemm_all_modes(cd, M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7 + N * 3 + K + 10 * ta + tb)
    A = rng.standard_normal((K, M) if ta else (M, K)) * \
        np.exp(rng.uniform(-3, 0, (K, M) if ta else (M, K)))
    B = rng.standard_normal((N, K) if tb else (K, N))
    C0 = rng.standard_normal((M, N))
    opA = A.T if ta else A
    opB = B.T if tb else B
    ref = 0.5 * C0 + 1.5 * (opA @ opB)
    bound = 1.5 * (np.abs(opA) @ np.abs(opB)).max() + 1e-300
    dA = torch.as_tensor(A, device="cuda")
    dB = torch.as_tensor(B, device="cuda")
    for mode in (0, 1, 2, 3):
        dC = torch.as_tensor(C0, device="cuda")
        cd.cdcc_dgemm(ta, tb, M, N, K, 1.5, dA, A.shape[1], dB, B.shape[1],
                      0.5, dC, N, mode=mode)
        torch.cuda.synchronize()
        err = np.abs(dC.cpu().numpy() - ref).max() / bound
        assert err <= BOUND[mode], (mode, err)
    # exact-slice modes: per element, relative to K * rowmax(A) * colmax(B)
    scale = 1.5 * K * np.abs(opA).max(axis=1)[:, None] * \
        np.abs(opB).max(axis=0)[None, :] + 1e-300
    for mode, bits in ((12, 15), (13, 22), (14, 29)):
        dC = torch.as_tensor(C0, device="cuda")
        cd.cdcc_dgemm(ta, tb, M, N, K, 1.5, dA, A.shape[1], dB, B.shape[1],
                      0.5, dC, N, mode=mode)
        torch.cuda.synchronize()
        err = (np.abs(dC.cpu().numpy() - ref) / scale).max()
        assert err <= 2.0 ** (1 - bits), (mode, err)


def _oracle_values(s, dL):
    from oracle import model, lagrangian
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
    r = lagrangian.run_all(h, L, s.nocc, tol=1e-11, e_tol=1e-13)
    return r["cc"]["E_corr"], dL @ pack_dense(s, r["G"].numpy())


def _mixed(cd, s, dL, prec=None):
    o = cd.cdcc_default_options()
    o.precision = cd.PREC_MIXED if prec is None else prec
    o.conv_tol = 1e-10
    ctx = cd.init_from_system(s, options=o)
    ctx_e, g = cd.gradient(ctx, dL)
    info = cd.cdcc_solver_info(ctx)
    tc = cd.cdcc_kernel_stats(ctx, 5) if False else None
    cd.cd_ccsd_free(ctx)
    return ctx_e, g, info


def test_mixed_c0_meets_target(cd):
    s = make_system(0)
    dL = make_displacements(s)
    e_or, g_or = _oracle_values(s, dL)
    e, g, info = _mixed(cd, s, dL)
    assert abs(e - e_or) <= 1e-8
    assert np.abs(g - g_or).max() <= 1e-6
    assert info[0] >= 1 and info[2] >= 1       # mixed iterations happened


def test_mixed_ragged_symmetric_meets_target(cd):
    s = random_system([3, 2, 2, 1], [30, 22, 18, 14], [70, 60, 56, 50],
                      seed=303, scale=0.3)
    dL = make_displacements(s, 4)
    e_or, g_or = _oracle_values(s, dL)
    e, g, info = _mixed(cd, s, dL)
    assert abs(e - e_or) <= 1e-8
    assert np.abs(g - g_or).max() <= 1e-6


def test_mixed_c1_meets_target(cd):
    s = make_system(1)
    dL = make_displacements(s)
    gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
    e, g, info = _mixed(cd, s, dL)
    assert abs(e - gold["e_corr"]) <= 1e-8
    assert np.abs(g - np.array(gold["gradient"])).max() <= 1e-6


@pytest.mark.parametrize("which", ["c0", "ragged", "c1"])
def test_tensor_core_finish_meets_target(cd, which):
    """CDCC_PREC_TC: every large contraction on the tensor cores (2-slice
    early iterations, exact-slice finish, prepare and density)."""
    if which == "c0":
        s = make_system(0)
        dL = make_displacements(s)
        e_ref, g_ref = _oracle_values(s, dL)
    elif which == "ragged":
        s = random_system([3, 2, 2, 1], [30, 22, 18, 14], [70, 60, 56, 50],
                          seed=303, scale=0.3)
        dL = make_displacements(s, 4)
        e_ref, g_ref = _oracle_values(s, dL)
    else:
        s = make_system(1)
        dL = make_displacements(s)
        gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
        e_ref, g_ref = gold["e_corr"], np.array(gold["gradient"])
    e, g, info = _mixed(cd, s, dL, prec=cd.PREC_TC)
    assert abs(e - e_ref) <= 1e-8, abs(e - e_ref)
    assert np.abs(g - g_ref).max() <= 1e-6


def test_fp64_gemm_tuned_shape_is_deterministic(cd):
    """The first call of a block shape times every tile shape; the choice
    must not change any bit of the result (split-K from a fixed tiling)."""
    torch.manual_seed(5)
    for (M, N, K) in [(32, 2592, 2592), (45, 70, 3000), (130, 40, 900)]:
        A = torch.randn(M, K, dtype=torch.float64, device="cuda")
        B = torch.randn(N, K, dtype=torch.float64, device="cuda")
        outs = []
        for _ in range(3):
            C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
            cd.cdcc_dgemm(0, 1, M, N, K, 1.0, A, K, B, K, 0.0, C, N, mode=0)
            outs.append(C.cpu())
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
        ref = (A.cpu() @ B.cpu().T)
        assert (outs[0] - ref).abs().max().item() < 1e-10 * K ** 0.5


@pytest.mark.parametrize("prec", ["fp64", "mixed", "tc"])
def test_error_estimate_brackets_the_measured_error(cd, prec):
    """cdcc_error_estimate against the error actually measured on c1 (the
    same gradient with the FP64 schedule): the estimate is of the right
    size (a first-order quantity: within a factor 10 of the measured energy
    error above the 1e-11 convergence noise), below the 1e-8 Eh / 1e-6
    targets, and it leaves Gamma and g unchanged."""
    s = make_system(1)
    dL = make_displacements(s, 4)
    ref = cd.init_from_system(s)
    e64, g64 = cd.gradient(ref, dL)
    cd.cd_ccsd_free(ref)
    o = cd.cdcc_default_options()
    o.precision = {"fp64": cd.PREC_FP64, "mixed": cd.PREC_MIXED,
                   "tc": cd.PREC_TC}[prec]
    ctx = cd.init_from_system(s, options=o)
    e, g = cd.gradient(ctx, dL)
    G = cd.cdcc_get_gamma(ctx)
    dE, dg = cd.cdcc_error_estimate(ctx, dL)
    assert np.array_equal(cd.cdcc_get_gamma(ctx), G)
    assert np.array_equal(cd.contract_dL(ctx, dL), g)
    cd.cd_ccsd_free(ctx)
    err = abs(e - e64)
    assert np.isfinite(dE) and dE >= 0 and np.all(dg >= 0)
    assert dE <= 1e-8 and np.abs(dg).max() <= 1e-6
    if prec == "fp64":
        assert dE < 1e-11 and np.abs(dg).max() < 1e-12
    else:
        # not an underestimate beyond the convergence noise, and not an
        # overestimate by more than 10x once the error is above that noise
        assert err <= 10 * dE + 1e-11, (err, dE)
        if err > 1e-11:
            assert dE <= 10 * err, (err, dE)
