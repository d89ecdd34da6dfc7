"""Write oracle reference values for the full-size parity tests.

Calls only `oracle/` (and the seeded generators in `synth/`).  For each
workload it stores the FP64 oracle's correlation energy, iteration counts,
the gradient g_x for every displacement and a seeded sample of Gamma^P,
t2 and lambda2 elements (packed / dense indices with values).

    python tests/golden/make_golden.py 1        # writes tests/golden/c1.json
    python tests/golden/make_golden.py serving  # writes tests/golden/serving.json
    python tests/golden/make_golden.py relaxed1 # writes c1_relaxed.json
(relaxed: the gradient of the orbital-relaxed model, oracle/zvector.py.)
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth import make_system, make_displacements, unpack_dense, pack_dense  # noqa
from oracle import model, lagrangian  # noqa


def golden(idx: int, nsample: int = 64):
    s = make_system(idx)
    o = s.nocc
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, o)
    t0 = time.time()
    r = lagrangian.run_all(h, L, o, tol=1e-11, e_tol=1e-13, verbose=True)
    secs = time.time() - t0
    dL = make_displacements(s)
    G = pack_dense(s, r["G"].numpy())
    g = dL @ G
    rng = np.random.default_rng(1234 + idx)
    gi = rng.choice(G.size, nsample, replace=False)
    t2 = r["cc"]["t2"].numpy()
    l2 = r["lam"]["l2"].numpy()
    big = np.argsort(-np.abs(t2).reshape(-1))[:nsample]
    return dict(
        workload=s.name, cfg_index=idx, scale=s.scale, tol=1e-11,
        e_corr=r["cc"]["E_corr"], e_ref=r["cc"]["E_ref"],
        ccsd_iterations=r["cc"]["iterations"],
        lambda_iterations=r["lam"]["iterations"], oracle_seconds=secs,
        gradient=g.tolist(),
        gamma_index=gi.tolist(), gamma_value=G[gi].tolist(),
        t2_index=big.tolist(), t2_value=t2.reshape(-1)[big].tolist(),
        l2_value=l2.reshape(-1)[big].tolist(),
        D1_trace=float(np.trace(r["D"].numpy())),
    )


def golden_relaxed(idx: int):
    """Relaxed gradient (Sec. 2.5, Eq. z_vector) of the orbital-relaxed
    model on workload idx: every displacement, the Z-vector norm and its
    largest elements."""
    from oracle import zvector
    s = make_system(idx)
    o = s.nocc
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, o)
    t0 = time.time()
    r = lagrangian.run_all(h, L, o, tol=1e-11, e_tol=1e-13)
    dL = make_displacements(s)
    dLd = torch.as_tensor(np.stack([unpack_dense(s, x) for x in dL]))
    g, Z, _ = zvector.relaxed_gradient(r, h, L, o, dLd)
    secs = time.time() - t0
    Zf = Z.numpy().reshape(-1)
    big = np.argsort(-np.abs(Zf))[:32]
    return dict(
        workload=s.name, cfg_index=idx, tol=1e-11, model="relaxed",
        e_corr=r["cc"]["E_corr"], gradient=g.numpy().tolist(),
        gradient_unrelaxed=(dL @ pack_dense(s, r["G"].numpy())).tolist(),
        z_norm=float(np.linalg.norm(Zf)), z_index=big.tolist(),
        z_value=Zf[big].tolist(), oracle_seconds=secs)


def golden_serving(omax: int = 16, nx: int = 2):
    """FP64 oracle energy and gradient of every serving request with
    o <= omax (the first 64 requests of the serving workload)."""
    from synth.serving import serving_jobs, job_system
    out = {}
    for sp in serving_jobs():
        if sp.o > omax:
            continue
        s = job_system(sp)
        L = torch.as_tensor(unpack_dense(s, s.L))
        h = model.core_from_eps(torch.as_tensor(s.eps), L, s.nocc)
        t0 = time.time()
        r = lagrangian.run_all(h, L, s.nocc, tol=1e-11, e_tol=1e-13)
        dL = make_displacements(s, nx)
        g = dL @ pack_dense(s, r["G"].numpy())
        out[str(sp.index)] = dict(o=sp.o, group=sp.group, scale=s.scale,
                                  e_corr=r["cc"]["E_corr"],
                                  gradient=g.tolist(),
                                  oracle_seconds=time.time() - t0)
        print(sp.index, sp.o, sp.group, r["cc"]["E_corr"], flush=True)
    return dict(workload="serving requests with o <= %d" % omax, tol=1e-11,
                nx=nx, requests=out)


if __name__ == "__main__":
    for a in sys.argv[1:]:
        if a == "serving":
            out = golden_serving()
            path = os.path.join(HERE, "serving.json")
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
            print("wrote", path)
            continue
        if a.startswith("relaxed"):
            idx = int(a[len("relaxed"):])
            out = golden_relaxed(idx)
            path = os.path.join(HERE, f"c{idx}_relaxed.json")
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
            print("wrote", path)
            continue
        idx = int(a)
        out = golden(idx)
        path = os.path.join(HERE, f"c{idx}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print("wrote", path, "E_corr", out["e_corr"])
