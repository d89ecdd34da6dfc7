"""C-ABI library: it loads, exports every declared symbol, and its host-side
input validation rejects bad inputs before touching a GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2512_21909_gb300 import build as cbuild
from paper_2512_21909_gb300 import cdcc
from synth import random_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cbuild.build()
    return cdcc.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;",
                             src, flags=re.M):
            if not m.group(0).lstrip().startswith("typedef"):
                names.append(m.group(1))
    return sorted(set(names))


def test_all_declared_symbols_exported(lib):
    names = declared_functions()
    assert "cd_ccsd_init" in names and "contract_dL" in names
    # serving, error report and three-term gradient entry points
    for n in ("cdcc_server_create", "cdcc_submit", "cdcc_poll", "cdcc_wait",
              "cdcc_server_destroy", "cdcc_job_footprint",
              "cdcc_energy_error", "contract_df", "cdcc_metric_size",
              "cdcc_contract_dL_noalloc", "cdcc_cd_two_step"):
        assert n in names, n
    for n in names:
        assert hasattr(lib, n), n


def test_default_options(lib):
    o = cdcc.cdcc_default_options()
    assert o.conv_tol == 1e-10 and o.max_iter == 100 and o.diis_dim == 8
    assert o.precision == cdcc.PREC_FP64


def _init(s, **kw):
    args = dict(nirrep=s.nirrep, nocc=s.nocc, nvir=s.nvir, nchol=s.nchol,
                orb_irrep=s.orb_irrep, eps=s.eps, chol_irrep=s.chol_irrep,
                L=s.L)
    args.update(kw)
    return cdcc.cd_ccsd_init(**args, use_torch_memory=False)


@pytest.mark.parametrize("bad", [
    dict(nirrep=3),
    dict(nocc=0),
    dict(orb_irrep="unsorted"),
    dict(chol_irrep="out_of_range"),
    dict(eps="overlap"),
])
def test_invalid_inputs_rejected_on_host(lib, bad):
    s = random_system([1, 1], [2, 2], [3, 3], seed=1)
    kw = {}
    for k, v in bad.items():
        if v == "unsorted":
            oi = s.orb_irrep.copy()
            oi[s.nocc:] = oi[s.nocc:][::-1]
            kw[k] = oi
        elif v == "out_of_range":
            ci = s.chol_irrep.copy()
            ci[-1] = 7
            kw[k] = ci
        elif v == "overlap":
            e = s.eps.copy()
            e[0] = 5.0
            kw[k] = e
        else:
            kw[k] = v
    with pytest.raises(cdcc.CdccError) as ei:
        _init(s, **kw)
    assert ei.value.status == cdcc.CDCC_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises; there is no CPU path."""
    from paper_2512_21909_gb300 import cdcc
    monkeypatch.setattr(cdcc, "_lib", None)
    monkeypatch.setattr(cdcc, "LIB", str(tmp_path / "absent" / "libcdcc.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        cdcc.load()
    with pytest.raises(RuntimeError):
        cdcc.cdcc_default_options()


@pytest.mark.parametrize("kw", [dict(tau=0.0), dict(tau=float("nan")),
                                dict(sigma=0.0), dict(sigma=1.5),
                                dict(qmax=0), dict(nirrep=9),
                                dict(npair=-1)])
def test_two_step_cd_rejects_bad_arguments(lib, kw):
    # checked before any device call: no GPU needed
    nirrep = kw.get("nirrep", 1)
    npair = [kw.get("npair", 3)] * nirrep
    naux = [2] * nirrep
    B = np.ones(max(sum(max(n, 0) * k for n, k in zip(npair, naux)), 1))
    with pytest.raises(cdcc.CdccError) as e:
        cdcc.cd_two_step(npair, naux, B, kw.get("tau", 1e-6),
                         sigma=kw.get("sigma", 1e-2), qmax=kw.get("qmax", 10))
    assert e.value.status == cdcc.CDCC_EINVAL


@pytest.mark.parametrize("relaxed,frozen", [(2, False), (1, True)])
def test_relaxed_option_rejected_on_host(lib, relaxed, frozen):
    # orbital relaxation is defined for the fixed-core model only
    s = random_system([1, 1], [2, 2], [3, 3], seed=1)
    o = cdcc.cdcc_default_options()
    assert o.relaxed == 0
    o.relaxed = relaxed
    if frozen:
        o.fock_model = cdcc.FROZEN_FOCK
    with pytest.raises(cdcc.CdccError) as ei:
        _init(s, options=o)
    assert ei.value.status == cdcc.CDCC_EINVAL
