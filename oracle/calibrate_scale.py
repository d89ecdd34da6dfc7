"""Compute the per-workload scale s_cfg stored in synth/gen.py (SCALES).

The literal distribution of the Cholesky vectors makes |E_MP2| grow like
o^2 v^2 nL; s_cfg rescales L (and dL) so that E_MP2 is about -0.04 Eh per
occupied orbital.  E_MP2 is homogeneous of degree 4 in L, hence
    s_cfg = min(1, (0.04 o / |E_MP2(s=1)|)^(1/4)).
Run:  python -m oracle.calibrate_scale   (prints the table)
      python -m oracle.calibrate_scale --serving   (writes
      synth/serving_scales.json, the per-request scales of the serving workload)
"""
from __future__ import annotations

import numpy as np

from synth import make_system, CONFIGS
from synth.gen import _irrep_members


def _ov_dense(sysm):
    """Dense L^P_ia block (nchol, o, v) from the packed pattern."""
    h = sysm.nirrep
    mem = _irrep_members(sysm.orb_irrep, h)
    o = sysm.nocc
    out = np.zeros((sysm.nchol, o, sysm.nvir))
    pos, P0 = 0, 0
    for gP in range(h):
        for k in range(sysm.chol[gP]):
            for gp in range(h):
                gq = gp ^ gP
                rp, rq = mem[gp], mem[gq]
                blk = sysm.L[pos:pos + len(rp) * len(rq)].reshape(len(rp),
                                                                   len(rq))
                pos += len(rp) * len(rq)
                ip = rp < o
                aq = rq >= o
                out[P0 + k][np.ix_(rp[ip], rq[aq] - o)] = blk[np.ix_(ip, aq)]
        P0 += sysm.chol[gP]
    return out


def mp2_chunked(eps, Lov):
    """E_MP2 (oracle/mp2.py formula), one occupied index i at a time."""
    nP, o, v = Lov.shape
    e_o, e_v = eps[:o], eps[o:]
    flat = Lov.reshape(nP, o * v)
    tot = 0.0
    for i in range(o):
        g = (Lov[:, i].T @ flat).reshape(v, o, v)              # (ia|jb)[a,j,b]
        gx = g.transpose(2, 1, 0)                              # (ib|ja)[a,j,b]
        D = e_o[i] - e_v[:, None, None] + e_o[None, :, None] - e_v[None, None, :]
        tot += float(np.sum(g * (2.0 * g - gx) / D))
    return tot


def calibrate(idx: int) -> float:
    s1 = make_system(idx, scale=1.0)
    e = mp2_chunked(s1.eps, _ov_dense(s1))
    return min(1.0, (0.04 * s1.nocc / abs(e)) ** 0.25), e


def calibrate_serving(path=None):
    """Per-request scales of the serving workload -> synth/serving_scales.json
    (same rule as the fixed workloads, E_MP2 from the arrays at s = 1)."""
    import json
    from synth.serving import serving_jobs, job_system, SCALES_FILE
    out = {}
    for spec in serving_jobs():
        s1 = job_system(spec, scale=1.0)
        e = mp2_chunked(s1.eps, _ov_dense(s1))
        out[str(spec.index)] = min(1.0, (0.04 * s1.nocc / abs(e)) ** 0.25)
        print(spec.index, spec.group, spec.o, out[str(spec.index)], flush=True)
    with open(path or SCALES_FILE, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    import sys
    if "--serving" in sys.argv:
        calibrate_serving()
    else:
        for idx in sorted(CONFIGS):
            s, e = calibrate(idx)
            print(f"{idx}: s_cfg = {s!r}   (E_MP2 at s=1: {e:.6e})")
