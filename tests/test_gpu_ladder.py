"""The particle-particle ladder assembled on the fly from L^P_ab (no stored
(ab|cd) integrals) against the FP64 oracle and against the stored ladder.

Batch sizes are forced small so that the row batches are ragged (one a per
batch, and a few a per batch with a short tail), and one system has an
irrep without Cholesky vectors (its (ac|bd) blocks vanish).  Tolerances as
in test_gpu_parity.py (FP64) and test_gpu_mixed.py (tensor-core schedules).
"""
import json
import os

import numpy as np
import pytest
import torch

from synth import make_system, random_system, make_displacements, pack_dense
from oracle import model, lagrangian
from synth import unpack_dense

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def oracle_run(s):
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
    return lagrangian.run_all(h, L, s.nocc, tol=1e-12, e_tol=1e-13)


def run(cd, s, dL, **opt):
    o = cd.cdcc_default_options()
    o.conv_tol = 1e-12
    o.energy_tol = 1e-13
    for k, v in opt.items():
        setattr(o, k, v)
    ctx = cd.init_from_system(s, options=o)
    mode = cd.cdcc_ladder_mode(ctx)
    e, it, res = cd.ccsd_solve(ctx)
    cd.lambda_solve(ctx)
    D1 = cd.build_density(ctx, s.n)
    g = cd.contract_dL(ctx, dL)
    G = cd.cdcc_get_gamma(ctx)
    cd.cd_ccsd_free(ctx)
    return dict(e=e, g=g, G=G, D1=D1, mode=mode)


CASES = {
    "c0": lambda: make_system(0),
    "ragged": lambda: random_system([3, 2, 2, 1], [7, 5, 4, 3],
                                    [12, 10, 9, 8], seed=211, scale=0.4),
    "no_chol_irrep": lambda: random_system([2, 1, 1, 1], [4, 3, 3, 2],
                                           [7, 0, 6, 5], seed=212, scale=0.4),
    "d2h_empty_vir": lambda: random_system([1, 1, 0, 1, 0, 0, 1, 0],
                                           [3, 2, 2, 0, 1, 2, 2, 1],
                                           [5, 3, 3, 3, 3, 3, 3, 2],
                                           seed=213, scale=0.45),
}


@pytest.mark.parametrize("pm", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("batch_gb", [1e-9, 2.5e-6, 2.0])
def test_on_the_fly_ladder_matches_oracle(cd, name, batch_gb, pm):
    # pm = 1: the +/- packed map (canonical pairs, two products)
    s = CASES[name]()
    dL = make_displacements(s, 3)
    r = oracle_run(s)
    gg = run(cd, s, dL, ladder=cd.LADDER_OTF, ladder_batch_gb=batch_gb,
             ladder_pm=pm)
    assert gg["mode"] == cd.LADDER_OTF
    G_or = pack_dense(s, r["G"].numpy())
    assert abs(gg["e"] - r["cc"]["E_corr"]) < 1e-10
    assert np.abs(gg["G"] - G_or).max() < 1e-9
    assert np.abs(gg["g"] - dL @ G_or).max() < 1e-9
    assert np.abs(gg["D1"] - r["D"].numpy()).max() < 1e-9


@pytest.mark.parametrize("pm", [0, 1])
def test_stored_and_on_the_fly_agree_c1(cd, pm):
    s = make_system(1)
    dL = make_displacements(s)
    gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
    a = run(cd, s, dL, ladder=cd.LADDER_STORED)
    b = run(cd, s, dL, ladder=cd.LADDER_OTF, ladder_batch_gb=0.01,
            ladder_pm=pm)
    assert a["mode"] == cd.LADDER_STORED and b["mode"] == cd.LADDER_OTF
    assert abs(a["e"] - b["e"]) < 1e-11
    assert np.abs(a["g"] - b["g"]).max() < 1e-10
    assert abs(b["e"] - gold["e_corr"]) < 1e-9
    assert np.abs(b["g"] - np.array(gold["gradient"])).max() < 1e-8


@pytest.mark.parametrize("pm", [0, 1])
@pytest.mark.parametrize("prec", ["mixed", "tc"])
def test_on_the_fly_ladder_tensor_core_schedules_c1(cd, prec, pm):
    s = make_system(1)
    dL = make_displacements(s)
    gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
    p = cd.PREC_TC if prec == "tc" else cd.PREC_MIXED
    o = cd.cdcc_default_options()
    o.precision = p
    o.ladder = cd.LADDER_OTF
    o.ladder_batch_gb = 0.05
    o.ladder_pm = pm
    ctx = cd.init_from_system(s, options=o)
    e, g = cd.gradient(ctx, dL)
    cd.cd_ccsd_free(ctx)
    assert abs(e - gold["e_corr"]) <= 1e-8
    assert np.abs(g - np.array(gold["gradient"])).max() <= 1e-6


def test_fused_float_slice_ladder_with_empty_cholesky_irrep(cd):
    # blocks large enough for the tensor-core route (the float-slice ladder
    # builds its (ab|cd) batch rows straight into BF16 slices), an irrep
    # without Cholesky vectors (zero integral blocks inside a batch) and
    # small ragged row batches, in the tensor-core schedule against the
    # FP64 oracle at the schedule's tolerance
    s = random_system([5, 4, 4, 3], [24, 20, 20, 16], [40, 0, 34, 30],
                      seed=214, scale=0.15)
    dL = make_displacements(s, 3)
    r = oracle_run(s)
    G_or = pack_dense(s, r["G"].numpy())
    for batch_gb, pm in ((0.0013, 0), (2.0, 0), (0.0013, 1), (2.0, 1)):
        gg = run(cd, s, dL, ladder=cd.LADDER_OTF, ladder_batch_gb=batch_gb,
                 precision=cd.PREC_TC, conv_tol=1e-10, energy_tol=1e-12,
                 ladder_pm=pm)
        assert gg["mode"] == cd.LADDER_OTF
        assert abs(gg["e"] - r["cc"]["E_corr"]) <= 1e-8
        assert np.abs(gg["g"] - dL @ G_or).max() <= 1e-6


@pytest.mark.parametrize("pm", [0, 1])
def test_float_slice_ladder_without_kept_slices(cd, pm):
    # the float-slice ladder when no batch slices may be kept
    # (ladder_slices_gb = 0): the plain map builds each batch into the batch
    # buffer, the +/- map multiplies its FP64 W+- through the generic
    # tensor-core route; same oracle and tolerances as above
    s = random_system([5, 4, 4, 3], [24, 20, 20, 16], [40, 0, 34, 30],
                      seed=214, scale=0.15)
    dL = make_displacements(s, 3)
    r = oracle_run(s)
    G_or = pack_dense(s, r["G"].numpy())
    gg = run(cd, s, dL, ladder=cd.LADDER_OTF, ladder_batch_gb=0.0013,
             precision=cd.PREC_TC, conv_tol=1e-10, energy_tol=1e-12,
             ladder_pm=pm, ladder_slices_gb=0.0)
    assert gg["mode"] == cd.LADDER_OTF
    assert abs(gg["e"] - r["cc"]["E_corr"]) <= 1e-8
    assert np.abs(gg["g"] - dL @ G_or).max() <= 1e-6
