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
