"""The allocation-free contract_dL entry point (cdcc_contract_dL_noalloc).

It serves callers that cannot allocate device memory (code inside a host
framework that owns the device memory, serving loops that must not call
cudaMalloc).  This file is collected last so that a run stopping at the
first failure has already run every other test.  The test calls the new
entry point through the C ABI on caller-owned device tensors and checks it
against the existing contract_dL, within the parity-test tolerance, on two
calls in a row (the shared device scratch keeps the previous call's
contents).
"""
import numpy as np
import pytest
import torch

from synth import make_system, random_system, make_displacements

pytestmark = pytest.mark.gpu

TOL = 1e-9   # the absolute gradient tolerance of the FP64 parity tests


def _gamma_and_reference(cd, s, dL):
    ctx = cd.init_from_system(s)
    _, g_ref = cd.gradient(ctx, dL)
    gamma = cd.cdcc_get_gamma(ctx)
    cd.cd_ccsd_free(ctx)
    return gamma, g_ref


def test_noalloc_matches_contract_dL_twice():
    from paper_2512_21909_gb300 import build as cbuild, cdcc as cd
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    cbuild.build()
    cases = [make_system(0),
             random_system([2, 1, 1, 0], [5, 3, 4, 2], [9, 7, 6, 6], seed=77,
                           scale=0.45)]
    nxs = [6, 11]
    for s, nx in zip(cases, nxs):
        dL = make_displacements(s, nx)
        gamma, g_ref = _gamma_and_reference(cd, s, dL)
        G = torch.as_tensor(gamma, device="cuda")
        D = torch.as_tensor(dL, device="cuda")
        for _ in range(2):       # two calls in a row share the scratch
            g = torch.full((nx,), float("nan"), dtype=torch.float64,
                           device="cuda")
            cd.cdcc_contract_dL_noalloc(G, D, nx, gamma.size, g)
            torch.cuda.synchronize()
            assert np.abs(g.cpu().numpy() - g_ref).max() < TOL


def test_noalloc_rejects_bad_sizes():
    from paper_2512_21909_gb300 import build as cbuild, cdcc as cd
    cbuild.build()
    G = torch.zeros(16, dtype=torch.float64, device="cuda")
    D = torch.zeros(16 * 65, dtype=torch.float64, device="cuda")
    g = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(cd.CdccError) as ei:
        cd.cdcc_contract_dL_noalloc(G, D, 65, 16, g)       # nx > maximum
    assert ei.value.status == cd.CDCC_EINVAL
    with pytest.raises(cd.CdccError):
        cd.cdcc_contract_dL_noalloc(G, D, 0, 16, g)
