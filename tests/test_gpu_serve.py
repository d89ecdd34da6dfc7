"""Serving on the GPU: requests of the serving workload (mixed sizes and
point groups, including D2h requests with empty irreps) run together through
the server (several in flight on their own streams) and each alone; every
request gives the same energy and gradient in both, and the smallest agree
with the FP64 oracle (|dE| <= 1e-8 Eh, |dg| <= 1e-6, tensor-core schedule).
"""
import numpy as np
import pytest
import torch

from synth import make_displacements, unpack_dense, pack_dense
from synth.serving import serving_jobs, job_system
from oracle import model, lagrangian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cd():
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    cbuild.build()
    return cdcc


def _requests(specs):
    from paper_2512_21909_gb300.serve import Request
    out = []
    for k, sp in enumerate(specs):
        s = job_system(sp)
        out.append(Request.from_system(sp.index, 0.0, s,
                                       make_displacements(s, 2)))
        out[-1].extra["system"] = s
    return out


def test_requests_alone_and_in_the_mix_agree(cd):
    from paper_2512_21909_gb300.serve import GradientServer, latency_stats
    specs = sorted(serving_jobs(), key=lambda j: j.o)[:10]
    mix = _requests(specs)
    srv = GradientServer(precision=cd.PREC_TC, max_active=4)
    srv.run(mix, realtime=False)
    assert all(r.status == "done" for r in mix), [r.status for r in mix]
    assert srv.max_seen_active >= 2
    st = latency_stats(mix, srv.wall)
    assert st["done"] == len(mix)
    alone = _requests(specs)
    solo = GradientServer(precision=cd.PREC_TC, max_active=1)
    solo.run(alone, realtime=False)
    for a, b in zip(mix, alone):
        assert b.status == "done"
        assert abs(a.e - b.e) <= 1e-12, (a.index, a.e, b.e)
        assert np.abs(a.g - b.g).max() <= 1e-12
    # the two smallest against the FP64 oracle
    for r in mix[:2]:
        s = r.extra["system"]
        L = torch.as_tensor(unpack_dense(s, s.L))
        h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
        o = lagrangian.run_all(h, L, s.nocc, tol=1e-11, e_tol=1e-12)
        g_or = r.dL @ pack_dense(s, o["G"].numpy())
        assert abs(r.e - o["cc"]["E_corr"]) <= 1e-8
        assert np.abs(r.g - g_or).max() <= 1e-6


def test_small_requests_against_stored_oracle_values(cd):
    # every request of the serving workload with o <= 16 (C1, C2v and D2h,
    # some with empty irreps), served together in the tensor-core schedule,
    # against the FP64 oracle values of tests/golden/serving.json; every
    # result carries its energy error report
    import json
    import os
    from paper_2512_21909_gb300.serve import GradientServer
    gold = json.load(open(os.path.join(os.path.dirname(
        os.path.abspath(__file__)), "golden", "serving.json")))["requests"]
    specs = [sp for sp in serving_jobs() if str(sp.index) in gold]
    assert len(specs) == len(gold) and len(specs) >= 15
    reqs = _requests(specs)
    srv = GradientServer(precision=cd.PREC_TC, max_active=4)
    srv.run(reqs, realtime=False)
    for r in reqs:
        ref = gold[str(r.index)]
        assert r.status == "done", (r.index, r.status)
        assert abs(r.e - ref["e_corr"]) <= 1e-8, (r.index, r.e, ref["e_corr"])
        assert np.abs(r.g - np.array(ref["gradient"])).max() <= 1e-6
        assert np.isfinite(r.err_dE) and 0.0 <= r.err_dE <= 1e-8, r.err_dE


def test_largest_requests_against_oracle_rows(cd):
    # the four largest requests (o = 40, v = 360, too large for the dense
    # oracle): the server's energy and gradient equal those of the same
    # request run alone through the context API, and the oracle's energy
    # functional and residual rows at that run's amplitudes confirm it
    from oracle import rows
    from paper_2512_21909_gb300.serve import GradientServer
    specs = sorted(serving_jobs(), key=lambda j: (-j.o, j.index))[:4]
    mix = _requests(specs)
    srv = GradientServer(precision=cd.PREC_TC, max_active=2)
    srv.run(mix, realtime=False)
    for r in mix:
        assert r.status == "done", (r.index, r.status)
        s = r.extra["system"]
        o, v = s.nocc, s.nvir
        opt = cd.cdcc_default_options()
        opt.precision = cd.PREC_TC
        opt.ladder = r.ladder
        ctx = cd.init_from_system(s, options=opt)
        e, _, _ = cd.ccsd_solve(ctx)
        t1 = cd.cdcc_get_amplitudes(ctx, 0, o, v)
        t2 = cd.cdcc_get_amplitudes(ctx, 1, o, v)
        cd.lambda_solve(ctx)
        cd.build_density(ctx)
        g = cd.contract_dL(ctx, r.dL)
        cd.cd_ccsd_free(ctx)
        assert abs(e - r.e) <= 1e-12 and np.abs(g - r.g).max() <= 1e-12
        L = torch.as_tensor(unpack_dense(s, s.L))
        h = model.core_from_eps(torch.as_tensor(s.eps), L, o)
        eref = model.e_ref(h, L, o).item()
        t1t, t2t = torch.as_tensor(t1), torch.as_tensor(t2)
        e_or = rows.energy(t1t, t2t, h, L, o) - eref
        assert abs(e - e_or) <= 1e-9, (r.index, e, e_or)
        R1, R2 = rows.residual_rows(t1t, t2t, h, L, o, [(0, o - 1)])
        D1 = s.eps[:o, None] - s.eps[None, o:]
        assert np.abs(R1.numpy() / D1).max() <= 1e-8
        Dij = s.eps[0] + s.eps[o - 1] - s.eps[o:, None] - s.eps[None, o:]
        assert np.abs(R2[(0, o - 1)].numpy() / Dij).max() <= 1e-8
