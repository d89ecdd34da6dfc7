"""The allocation-free contract_dL entry point (cdcc_contract_dL_noalloc).

It serves callers that cannot allocate device memory (code inside a host
framework that owns the device memory, serving loops that must not call
cudaMalloc).  This file is collected last so that a run stopping at the
first failure has already run every other test.  The tests call the entry
point through the C ABI on caller-owned device tensors and check it against
the existing contract_dL, against the stored FP64 oracle gradient of the
D2h o=16 v=144 nL=640 workload, and against an FP64 matrix-vector product
on a tensor large enough to fill every block of the fixed scratch array;
each case makes two calls in a row (the shared device scratch keeps the
previous call's contents).
"""
import json
import os

import numpy as np
import pytest
import torch

from synth import make_system, random_system, make_displacements

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-9   # the absolute gradient tolerance of the FP64 parity tests


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    cbuild.build()
    cdcc.load()
    return cdcc


def _gamma_and_reference(cd, s, dL):
    ctx = cd.init_from_system(s)
    _, g_ref = cd.gradient(ctx, dL)
    gamma = cd.cdcc_get_gamma(ctx)
    cd.cd_ccsd_free(ctx)
    return gamma, g_ref


def _twice(cd, G, D, nx, nnz):
    out = []
    for _ in range(2):       # two calls in a row share the scratch
        g = torch.full((nx,), float("nan"), dtype=torch.float64,
                       device="cuda")
        cd.cdcc_contract_dL_noalloc(G, D, nx, nnz, g)
        torch.cuda.synchronize()
        out.append(g.cpu().numpy())
    return out


def test_noalloc_matches_contract_dL_twice(cd):
    cases = [make_system(0),
             random_system([2, 1, 1, 0], [5, 3, 4, 2], [9, 7, 6, 6], seed=77,
                           scale=0.45)]
    nxs = [6, 11]
    for s, nx in zip(cases, nxs):
        dL = make_displacements(s, nx)
        gamma, g_ref = _gamma_and_reference(cd, s, dL)
        G = torch.as_tensor(gamma, device="cuda")
        D = torch.as_tensor(dL, device="cuda")
        for g in _twice(cd, G, D, nx, gamma.size):
            assert np.abs(g - g_ref).max() < TOL


def test_noalloc_maximum_nx_matches_contract_dL(cd):
    # nx = CDCC_NOALLOC_MAX_NX = 64: every slot of the scratch array's
    # displacement dimension is used (8 passes of 8 displacements)
    s = random_system([2, 1, 1, 0], [5, 3, 4, 2], [9, 7, 6, 6], seed=78,
                      scale=0.45)
    dL = make_displacements(s, 64)
    gamma, g_ref = _gamma_and_reference(cd, s, dL)
    G = torch.as_tensor(gamma, device="cuda")
    D = torch.as_tensor(dL, device="cuda")
    for g in _twice(cd, G, D, 64, gamma.size):
        assert np.abs(g - g_ref).max() < TOL


def test_noalloc_d2h_workload_against_oracle_gradient(cd):
    # Gamma of the D2h o=16 v=144 nL=640 workload (FP64 schedule), contracted
    # with its 18 displacements, against the stored FP64 oracle gradient
    gold = json.load(open(os.path.join(HERE, "golden", "c1.json")))
    s = make_system(1)
    dL = make_displacements(s)
    gamma, g_ref = _gamma_and_reference(cd, s, dL)
    G = torch.as_tensor(gamma, device="cuda")
    D = torch.as_tensor(dL, device="cuda")
    for g in _twice(cd, G, D, dL.shape[0], gamma.size):
        assert np.abs(g - g_ref).max() < TOL
        assert np.abs(g - np.array(gold["gradient"])).max() < 1e-8


def test_noalloc_fills_every_block(cd):
    # nnz above (8 x SM count) x 4096 elements: the grid is clamped and every
    # block sums more than 4096 elements; nx = 9 spans two passes
    nnz, nx = 6_000_001, 9
    gen = torch.Generator(device="cpu").manual_seed(909)
    Gh = torch.randn(nnz, dtype=torch.float64, generator=gen)
    Dh = torch.randn(nx, nnz, dtype=torch.float64, generator=gen)
    ref = (Dh @ Gh).numpy()
    # rounding bound of two FP64 summation orders whose trees are at most a
    # few hundred additions deep: 1e-13 * sum |G_e dL_xe|
    bound = 1e-13 * (Dh.abs() @ Gh.abs()).numpy()
    G = Gh.cuda()
    D = Dh.cuda().contiguous()
    for g in _twice(cd, G, D, nx, nnz):
        assert np.all(np.abs(g - ref) < bound)


def test_noalloc_rejects_bad_sizes_and_foreign_memory(cd):
    G = torch.zeros(16, dtype=torch.float64, device="cuda")
    D = torch.zeros(16 * 65, dtype=torch.float64, device="cuda")
    g = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(cd.CdccError) as ei:
        cd.cdcc_contract_dL_noalloc(G, D, 65, 16, g)       # nx > maximum
    assert ei.value.status == cd.CDCC_EINVAL
    with pytest.raises(cd.CdccError):
        cd.cdcc_contract_dL_noalloc(G, D, 0, 16, g)
    # host memory is refused before anything is launched
    with pytest.raises(cd.CdccError) as ei:
        cd.cdcc_contract_dL_noalloc(G.cpu(), D, 1, 16, g)
    assert ei.value.status == cd.CDCC_EINVAL
    if torch.cuda.device_count() > 1:
        # memory of another GPU is refused as well (no launch happens)
        G1 = torch.zeros(16, dtype=torch.float64, device="cuda:1")
        with pytest.raises(cd.CdccError) as ei:
            cd.cdcc_contract_dL_noalloc(G1, D, 1, 16, g)
        assert ei.value.status == cd.CDCC_EINVAL
