"""Thin ctypes binding of include/cdcc.h (argument marshalling only).

Every compute step runs inside libcdcc.so.  Inputs may be numpy arrays (host)
or CUDA torch tensors (device); outputs are numpy arrays.  Device memory of
a context comes from PyTorch's caching allocator and work runs on the
current torch stream unless options say otherwise.  There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

_lib = None

CDCC_OK, CDCC_EINVAL, CDCC_ENOMEM, CDCC_ENOCONV, CDCC_ENUMERIC, CDCC_ECUDA, \
    CDCC_ESTATE, CDCC_ETIMEOUT = range(8)
STATUS = {0: "CDCC_OK", 1: "CDCC_EINVAL", 2: "CDCC_ENOMEM", 3: "CDCC_ENOCONV",
          4: "CDCC_ENUMERIC", 5: "CDCC_ECUDA", 6: "CDCC_ESTATE",
          7: "CDCC_ETIMEOUT"}
PREC_FP64, PREC_MIXED, PREC_TC = 0, 1, 2
LADDER_AUTO, LADDER_STORED, LADDER_OTF = 0, 1, 2
FIXED_CORE, FROZEN_FOCK = 0, 1

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t,
                           ctypes.c_void_p, ctypes.c_void_p)


class cdcc_options(ctypes.Structure):
    _fields_ = [("conv_tol", ctypes.c_double), ("energy_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("diis_dim", ctypes.c_int),
                ("precision", ctypes.c_int), ("switch_tol", ctypes.c_double),
                ("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_user", ctypes.c_void_p), ("ladder", ctypes.c_int),
                ("ladder_batch_gb", ctypes.c_double),
                ("fock_model", ctypes.c_int),
                ("ladder_linearize", ctypes.c_int),
                ("perm_cache_gb", ctypes.c_double),
                ("ladder_slices_gb", ctypes.c_double),
                ("ladder_pm", ctypes.c_int),
                ("relaxed", ctypes.c_int)]


class CdccError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return LIB


def load():
    """Load libcdcc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(
            f"libcdcc.so not found at {LIB}: build it with "
            "`python -m paper_2512_21909_gb300.build` (no CPU fallback)")
    L = ctypes.CDLL(LIB)
    P = ctypes.POINTER
    vp, i32p, dp = ctypes.c_void_p, P(ctypes.c_int32), ctypes.c_void_p
    L.cdcc_default_options.argtypes = [P(cdcc_options)]
    L.cd_ccsd_init.argtypes = [P(vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, vp, vp, vp, vp, P(cdcc_options)]
    L.cdcc_packed_size.argtypes = [vp, ctypes.c_int]
    L.cdcc_packed_size.restype = ctypes.c_size_t
    L.ccsd_solve.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int),
                             P(ctypes.c_double)]
    L.lambda_solve.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_double)]
    L.build_density.argtypes = [vp, vp]
    L.cdcc_get_gamma.argtypes = [vp, vp]
    L.contract_dL.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.gradient.argtypes = [vp, ctypes.c_int, vp, vp, P(ctypes.c_double), vp]
    L.cdcc_get_amplitudes.argtypes = [vp, ctypes.c_int, vp]
    L.cdcc_phase_times.argtypes = [vp, vp]
    L.cdcc_profile.argtypes = [vp, ctypes.c_int]
    L.cdcc_profile.restype = ctypes.c_int
    L.cdcc_kernel_stats.argtypes = [vp, ctypes.c_int, P(ctypes.c_double),
                                    P(ctypes.c_longlong), P(ctypes.c_double)]
    L.cdcc_kernel_stats.restype = ctypes.c_int
    L.cdcc_kernel_launches.argtypes = [vp]
    L.cdcc_kernel_launches.restype = ctypes.c_longlong
    L.cdcc_last_error.argtypes = [vp]
    L.cdcc_last_error.restype = ctypes.c_char_p
    L.cd_ccsd_free.argtypes = [vp]
    L.cd_ccsd_free.restype = None
    for name in ("cd_ccsd_init", "ccsd_solve", "lambda_solve",
                 "build_density", "cdcc_get_gamma", "contract_dL", "gradient",
                 "cdcc_get_amplitudes", "cdcc_phase_times"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


# ------------------------------------------------------------------ helpers
def _ptr(x):
    """(pointer, keepalive) for a numpy array or a torch tensor."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    return ctypes.c_void_p(x.ctypes.data), x


def _f64(x):
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64:
            raise ValueError("expected float64")
        return x
    return np.ascontiguousarray(x, dtype=np.float64)


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


_KEEP = {}


def _torch_allocator(device):
    import torch

    def alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device,
                                                      stream or 0)
        except Exception:
            return None

    def free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


class Context:
    """Owns a cdcc_ctx*; freed on close() / garbage collection."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    @property
    def value(self):
        return self.handle.value

    def close(self):
        if self.handle is not None and self.handle.value:
            load().cd_ccsd_free(self.handle)
            _KEEP.pop(id(self), None)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(ctx, status):
    if status != CDCC_OK:
        msg = load().cdcc_last_error(ctx.handle if ctx else None)
        raise CdccError(status, msg.decode() if msg else "")


# ------------------------------------------------------------ the C ABI
def cdcc_default_options() -> cdcc_options:
    o = cdcc_options()
    load().cdcc_default_options(ctypes.byref(o))
    return o


def cd_ccsd_init(nirrep, nocc, nvir, nchol, orb_irrep, eps, chol_irrep, L,
                 options: cdcc_options | None = None, use_torch_memory=True,
                 stream=None) -> Context:
    lib = load()
    opt = options if options is not None else cdcc_default_options()
    keep = []
    if use_torch_memory:
        import torch
        dev = opt.device
        fa, ff = _torch_allocator(dev)
        opt.dev_alloc, opt.dev_free = fa, ff
        keep += [fa, ff]
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
    if stream is not None:
        opt.stream = ctypes.c_void_p(int(stream))
    oi, ci = _i32(orb_irrep), _i32(chol_irrep)
    e = _f64(eps)
    Lp, Lk = _ptr(_f64(L))
    keep += [opt]
    h = ctypes.c_void_p()
    st = lib.cd_ccsd_init(ctypes.byref(h), int(nirrep), int(nocc), int(nvir),
                          int(nchol), oi.ctypes.data_as(ctypes.c_void_p),
                          e.ctypes.data_as(ctypes.c_void_p),
                          ci.ctypes.data_as(ctypes.c_void_p), Lp,
                          ctypes.byref(opt))
    ctx = Context(h, keep)
    _KEEP[id(ctx)] = keep
    if st != CDCC_OK:
        msg = lib.cdcc_last_error(h).decode()
        ctx.close()
        raise CdccError(st, msg)
    return ctx


def cdcc_packed_size(ctx, gx=0) -> int:
    return int(load().cdcc_packed_size(ctx.handle, int(gx)))


def ccsd_solve(ctx):
    e, it, r = ctypes.c_double(), ctypes.c_int(), ctypes.c_double()
    _check(ctx, load().ccsd_solve(ctx.handle, ctypes.byref(e), ctypes.byref(it),
                                  ctypes.byref(r)))
    return e.value, it.value, r.value


def lambda_solve(ctx):
    it, r = ctypes.c_int(), ctypes.c_double()
    _check(ctx, load().lambda_solve(ctx.handle, ctypes.byref(it),
                                    ctypes.byref(r)))
    return it.value, r.value


def build_density(ctx, n=None):
    D1 = None if n is None else np.zeros((n, n))
    _check(ctx, load().build_density(
        ctx.handle, None if D1 is None else D1.ctypes.data_as(ctypes.c_void_p)))
    return D1


def cdcc_get_gamma(ctx):
    out = np.empty(cdcc_packed_size(ctx, 0))
    _check(ctx, load().cdcc_get_gamma(ctx.handle,
                                      out.ctypes.data_as(ctypes.c_void_p)))
    return out


def _displacements(dL, x_irrep, nx):
    if x_irrep is None:
        xi = None
        xp = None
    else:
        xi = _i32(x_irrep)
        xp = xi.ctypes.data_as(ctypes.c_void_p)
    d = _f64(dL)
    dp, _ = _ptr(d)
    return xi, xp, d, dp


def contract_dL(ctx, dL, nx=None, x_irrep=None):
    if nx is None:
        nx = dL.shape[0] if getattr(dL, "ndim", 1) > 1 else 1
    xi, xp, d, dp = _displacements(dL, x_irrep, nx)
    g = np.zeros(nx)
    _check(ctx, load().contract_dL(ctx.handle, int(nx), xp, dp,
                                   g.ctypes.data_as(ctypes.c_void_p)))
    return g


def cdcc_metric_size(ctx) -> int:
    lib = load()
    lib.cdcc_metric_size.argtypes = [ctypes.c_void_p]
    lib.cdcc_metric_size.restype = ctypes.c_size_t
    return int(lib.cdcc_metric_size(ctx.handle))


def contract_df(ctx, metric, dB, dM):
    """Three-term DF/CD gradient (see include/cdcc.h): metric packed,
    dB (nx, packed), dM (nx, metric size); host or device arrays."""
    lib = load()
    lib.contract_df.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + \
        [ctypes.c_void_p] * 3
    lib.contract_df.restype = ctypes.c_int
    Mp, Mk = _ptr(_f64(metric))
    dBp, dBk = _ptr(_f64(dB))
    dMp, dMk = _ptr(_f64(dM))
    nx = int(dB.shape[0])
    g = np.zeros(max(nx, 1))
    _check(ctx, lib.contract_df(ctx.handle, Mp, nx, dBp, dMp,
                                g.ctypes.data_as(ctypes.c_void_p)))
    return g[:nx]


def cd_two_step(npair, naux, B, tau, sigma=1e-2, qmax=1000, device=0,
                max_vectors=None):
    """Symmetry-adapted two-step Cholesky decomposition (see
    include/cdcc.h, cdcc_cd_two_step): npair, naux per irrep; B the packed
    factor blocks (host or device array).  Returns (pivots, vectors, stats):
    pivots[G] (pair indices in the order taken), vectors[G]
    (ncv x npair numpy arrays), stats [macro, micro, first s, second s]."""
    lib = load()
    lib.cdcc_cd_two_step.argtypes = (
        [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
         ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
         ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_char_p,
         ctypes.c_int])
    lib.cdcc_cd_two_step.restype = ctypes.c_int
    h = len(npair)
    npa = np.ascontiguousarray(npair, dtype=np.int32)
    nax = np.ascontiguousarray(naux, dtype=np.int32)
    Bp, Bk = _ptr(_f64(B))
    ncv = np.zeros(h, np.int32)
    stats = np.zeros(4)
    msg = ctypes.create_string_buffer(256)
    # outputs sized for the factor's rank (plus a margin); if that is too
    # small the call reports the counts and is repeated with exact sizes
    per = [min(int(n), int(k) + 64) for n, k in zip(npair, naux)]
    if max_vectors is not None:
        per = [min(int(n), int(max_vectors)) for n in npair]
    for _ in range(2):
        piv = np.zeros(max(sum(per), 1), np.int32)
        L = np.zeros(max(sum(c * int(n) for c, n in zip(per, npair)), 1))
        st = lib.cdcc_cd_two_step(
            h, npa.ctypes.data_as(ctypes.c_void_p),
            nax.ctypes.data_as(ctypes.c_void_p), Bp, float(tau),
            float(sigma), int(qmax), int(device), None,
            ncv.ctypes.data_as(ctypes.c_void_p),
            piv.ctypes.data_as(ctypes.c_void_p), int(piv.size),
            L.ctypes.data_as(ctypes.c_void_p), int(L.size),
            stats.ctypes.data_as(ctypes.c_void_p), msg, 256)
        if st == CDCC_ENOMEM and int(ncv.sum()) > 0 and \
                any(int(c) > p for c, p in zip(ncv, per)):
            per = [int(c) for c in ncv]
            continue
        break
    if st != CDCC_OK:
        raise CdccError(st, msg.value.decode(errors="replace"))
    pivots, vectors, po, lo = [], [], 0, 0
    for g in range(h):
        k, n = int(ncv[g]), int(npair[g])
        pivots.append(piv[po:po + k].tolist())
        vectors.append(L[lo:lo + k * n].reshape(k, n).copy())
        po += k
        lo += k * n
    return pivots, vectors, stats


def ladder_pm_tables(nocc_irrep, nvir_irrep, batch_gb=2.0):
    """Index tables of the +/- packed ladder (include/cdcc.h,
    cdcc_ladder_pm_tables; host only).  Returns {G: dict(uo, uv, nrow, ncol,
    r1, r2, c1, c2, batches=[dict(ga, a0, a1, lr, y1, y2)])}."""
    lib = load()
    lib.cdcc_ladder_pm_tables.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
        ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.cdcc_ladder_pm_tables.restype = ctypes.c_int
    h = len(nocc_irrep)
    no = np.ascontiguousarray(nocc_irrep, dtype=np.int32)
    nv = np.ascontiguousarray(nvir_irrep, dtype=np.int32)
    n = ctypes.c_int64(0)
    args = (h, no.ctypes.data_as(ctypes.c_void_p),
            nv.ctypes.data_as(ctypes.c_void_p), float(batch_gb))
    st = lib.cdcc_ladder_pm_tables(*args, None, 0, ctypes.byref(n))
    if st != CDCC_OK:
        raise CdccError(st, "cdcc_ladder_pm_tables")
    out = np.zeros(max(1, n.value), np.int32)
    st = lib.cdcc_ladder_pm_tables(*args, out.ctypes.data_as(ctypes.c_void_p),
                                   int(out.size), ctypes.byref(n))
    if st != CDCC_OK:
        raise CdccError(st, "cdcc_ladder_pm_tables")
    res, k = {}, 0
    while k < n.value:
        G, uo, uv, nb, nrow, ncol = (int(x) for x in out[k:k + 6])
        k += 6
        e = dict(uo=uo, uv=uv, nrow=nrow, ncol=ncol,
                 r1=out[k:k + uo], r2=out[k + uo:k + 2 * uo])
        k += 2 * uo
        e["c1"], e["c2"] = out[k:k + uv], out[k + uv:k + 2 * uv]
        k += 2 * uv
        e["batches"] = []
        for _ in range(nb):
            ga, a0, a1, m = (int(x) for x in out[k:k + 4])
            k += 4
            e["batches"].append(dict(ga=ga, a0=a0, a1=a1,
                                     lr=out[k:k + m], y1=out[k + m:k + 2 * m],
                                     y2=out[k + 2 * m:k + 3 * m]))
            k += 3 * m
        res[G] = e
    return res


def cdcc_error_estimate(ctx, dL=None, nx=None, x_irrep=None):
    """(dE, dg[nx]): change of E and g caused by the schedule's reduced
    precision, measured against FP64 at the converged t and lambda."""
    lib = load()
    lib.cdcc_error_estimate.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
    lib.cdcc_error_estimate.restype = ctypes.c_int
    dE = ctypes.c_double()
    if dL is None:
        _check(ctx, lib.cdcc_error_estimate(ctx.handle, 0, None, None,
                                            ctypes.byref(dE), None))
        return dE.value, np.zeros(0)
    if nx is None:
        nx = dL.shape[0] if getattr(dL, "ndim", 1) > 1 else 1
    xi, xp, d, dp = _displacements(dL, x_irrep, nx)
    dg = np.zeros(nx)
    _check(ctx, lib.cdcc_error_estimate(
        ctx.handle, int(nx), xp, dp, ctypes.byref(dE),
        dg.ctypes.data_as(ctypes.c_void_p)))
    return dE.value, dg


def gradient(ctx, dL, nx=None, x_irrep=None):
    if nx is None:
        nx = dL.shape[0] if getattr(dL, "ndim", 1) > 1 else 1
    xi, xp, d, dp = _displacements(dL, x_irrep, nx)
    g = np.zeros(nx)
    e = ctypes.c_double()
    _check(ctx, load().gradient(ctx.handle, int(nx), xp, dp, ctypes.byref(e),
                                g.ctypes.data_as(ctypes.c_void_p)))
    return e.value, g


def cdcc_get_amplitudes(ctx, which, nocc, nvir):
    shape = (nocc, nvir) if which % 2 == 0 else (nocc, nocc, nvir, nvir)
    out = np.zeros(shape)
    _check(ctx, load().cdcc_get_amplitudes(ctx.handle, int(which),
                                           out.ctypes.data_as(ctypes.c_void_p)))
    return out


def cdcc_phase_times(ctx):
    t = np.zeros(4)
    _check(ctx, load().cdcc_phase_times(ctx.handle,
                                        t.ctypes.data_as(ctypes.c_void_p)))
    return t


KERNEL_CLASSES = ("gemm64", "permute", "update", "contract_dL", "other",
                  "tc_float_slices", "tc_exact_slices")


def cdcc_solver_info(ctx):
    """(ccsd mixed, ccsd fp64, lambda mixed, lambda fp64) iterations."""
    lib = load()
    lib.cdcc_solver_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.cdcc_solver_info.restype = ctypes.c_int
    info = np.zeros(4, dtype=np.int32)
    _check(ctx, lib.cdcc_solver_info(ctx.handle,
                                     info.ctypes.data_as(ctypes.c_void_p)))
    return tuple(int(x) for x in info)


def cdcc_ladder_stats(ctx):
    """(seconds, algorithmic flops, calls) of the ladder contractions while
    profiling was on."""
    lib = load()
    lib.cdcc_ladder_stats.argtypes = [ctypes.c_void_p] * 4
    lib.cdcc_ladder_stats.restype = ctypes.c_int
    sec, fl, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_longlong()
    _check(ctx, lib.cdcc_ladder_stats(ctx.handle, ctypes.byref(sec),
                                      ctypes.byref(fl), ctypes.byref(n)))
    return sec.value, fl.value, n.value


def cdcc_ladder_mode(ctx) -> int:
    """LADDER_STORED or LADDER_OTF, as chosen by the context."""
    lib = load()
    lib.cdcc_ladder_mode.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.cdcc_ladder_mode.restype = ctypes.c_int
    m = ctypes.c_int(0)
    _check(ctx, lib.cdcc_ladder_mode(ctx.handle, ctypes.byref(m)))
    return m.value


def cdcc_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
               mode=0, stream=None):
    """C = beta C + alpha op(A) op(B) on CUDA tensors (row-major)."""
    lib = load()
    lib.cdcc_dgemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_int, ctypes.c_double,
                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    lib.cdcc_dgemm.restype = ctypes.c_int
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.cdcc_dgemm(int(transA), int(transB), int(M), int(N), int(K),
                        float(alpha), ctypes.c_void_p(A.data_ptr()), int(lda),
                        ctypes.c_void_p(B.data_ptr()), int(ldb), float(beta),
                        ctypes.c_void_p(C.data_ptr()), int(ldc), int(mode),
                        ctypes.c_void_p(int(stream)))
    if st != CDCC_OK:
        raise CdccError(st, "cdcc_dgemm failed")


def cdcc_profile(ctx, enable=True):
    _check(ctx, load().cdcc_profile(ctx.handle, int(bool(enable))))


def cdcc_kernel_stats(ctx, kind):
    """(device seconds, launches, algorithmic work) of a kernel class."""
    sec, n, w = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, load().cdcc_kernel_stats(ctx.handle, int(kind),
                                         ctypes.byref(sec), ctypes.byref(n),
                                         ctypes.byref(w)))
    return sec.value, n.value, w.value


def cdcc_kernel_launches(ctx) -> int:
    return int(load().cdcc_kernel_launches(ctx.handle))


def cdcc_last_error(ctx) -> str:
    return load().cdcc_last_error(ctx.handle).decode()


def cd_ccsd_free(ctx):
    ctx.close()


def cdcc_contract_dL_noalloc(gamma, dL, nx, nnz, g, stream=None):
    """Allocation-free contract_dL on caller-owned CUDA tensors (gamma: packed
    Gamma, dL: nx packed tensors, g: nx outputs); enqueues on `stream`
    (default: the current torch stream) and returns without waiting."""
    lib = load()
    if not hasattr(lib, "_noalloc_typed"):
        lib.cdcc_contract_dL_noalloc.argtypes = [
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t,
            ctypes.c_void_p, ctypes.c_void_p]
        lib.cdcc_contract_dL_noalloc.restype = ctypes.c_int
        lib._noalloc_typed = True
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    st = lib.cdcc_contract_dL_noalloc(
        ctypes.c_void_p(gamma.data_ptr()), ctypes.c_void_p(dL.data_ptr()),
        int(nx), int(nnz), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(int(stream)))
    if st != CDCC_OK:
        raise CdccError(st, "cdcc_contract_dL_noalloc failed")


def cdcc_selftest_bounded_wait(stream=None) -> int:
    """Run the bounded-wait self-test; returns the cdcc_status code
    (CDCC_ETIMEOUT means the give-up path works)."""
    lib = load()
    lib.cdcc_selftest_bounded_wait.argtypes = [ctypes.c_void_p]
    lib.cdcc_selftest_bounded_wait.restype = ctypes.c_int
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    return int(lib.cdcc_selftest_bounded_wait(ctypes.c_void_p(int(stream))))


def init_from_system(sysm, **kw) -> Context:
    """cd_ccsd_init from a synth.System (host arrays)."""
    return cd_ccsd_init(sysm.nirrep, sysm.nocc, sysm.nvir, sysm.nchol,
                        sysm.orb_irrep, sysm.eps, sysm.chol_irrep, sysm.L, **kw)


# ------------------------------------------------------------------ serving
class cdcc_job_desc(ctypes.Structure):
    _fields_ = [("nirrep", ctypes.c_int), ("nocc", ctypes.c_int),
                ("nvir", ctypes.c_int), ("nchol", ctypes.c_int),
                ("orb_irrep", ctypes.c_void_p), ("eps", ctypes.c_void_p),
                ("chol_irrep", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("nx", ctypes.c_int), ("x_irrep", ctypes.c_void_p),
                ("dL", ctypes.c_void_p)]


class cdcc_result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int),
                ("nx", ctypes.c_int), ("ladder", ctypes.c_int),
                ("retries", ctypes.c_int), ("e_corr", ctypes.c_double),
                ("err_dE", ctypes.c_double), ("t_wait", ctypes.c_double),
                ("t_run", ctypes.c_double), ("g", ctypes.c_void_p),
                ("message", ctypes.c_char * 160)]


EXECUTOR_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_uint64,
                               ctypes.POINTER(cdcc_job_desc), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double),
                               ctypes.c_void_p)


class cdcc_server_options(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("budget_gb", ctypes.c_double),
                ("reserve_gb", ctypes.c_double),
                ("stored_max_gb", ctypes.c_double),
                ("error_report", ctypes.c_int), ("executor", EXECUTOR_FN),
                ("executor_user", ctypes.c_void_p)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = range(4)


def _server_lib():
    lib = load()
    if not hasattr(lib, "_server_typed"):
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.cdcc_server_default_options.argtypes = [P(cdcc_server_options)]
        lib.cdcc_server_default_options.restype = None
        lib.cdcc_server_create.argtypes = [P(vp), P(cdcc_options),
                                           P(cdcc_server_options)]
        lib.cdcc_server_create.restype = ctypes.c_int
        lib.cdcc_submit.argtypes = [vp, P(cdcc_job_desc),
                                    P(ctypes.c_uint64)]
        lib.cdcc_submit.restype = ctypes.c_int
        lib.cdcc_poll.argtypes = [vp, ctypes.c_uint64, P(cdcc_result)]
        lib.cdcc_poll.restype = ctypes.c_int
        lib.cdcc_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double,
                                  P(cdcc_result)]
        lib.cdcc_wait.restype = ctypes.c_int
        lib.cdcc_server_max_active_seen.argtypes = [vp]
        lib.cdcc_server_max_active_seen.restype = ctypes.c_int
        lib.cdcc_job_footprint.argtypes = [P(cdcc_job_desc), ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double]
        lib.cdcc_job_footprint.restype = ctypes.c_size_t
        lib.cdcc_server_destroy.argtypes = [vp]
        lib.cdcc_server_destroy.restype = None
        lib.cdcc_energy_error.argtypes = [vp, P(ctypes.c_double)]
        lib.cdcc_energy_error.restype = ctypes.c_int
        lib._server_typed = True
    return lib


def cdcc_server_default_options() -> cdcc_server_options:
    o = cdcc_server_options()
    _server_lib().cdcc_server_default_options(ctypes.byref(o))
    return o


def job_desc(nirrep, nocc, nvir, nchol, orb_irrep, eps, chol_irrep, L, dL,
             x_irrep=None):
    """(cdcc_job_desc, keepalive) for host arrays (numpy)."""
    oi, ci = _i32(orb_irrep), _i32(chol_irrep)
    e, Lh = _f64(eps), _f64(L)
    dLh = _f64(dL)
    nx = int(dLh.shape[0]) if dLh.ndim > 1 else (1 if dLh.size else 0)
    xi = _i32(x_irrep) if x_irrep is not None else None
    d = cdcc_job_desc(int(nirrep), int(nocc), int(nvir), int(nchol),
                      oi.ctypes.data, e.ctypes.data, ci.ctypes.data,
                      Lh.ctypes.data, nx,
                      xi.ctypes.data if xi is not None else None,
                      dLh.ctypes.data if dLh.size else None)
    return d, (oi, ci, e, Lh, dLh, xi)


def cdcc_job_footprint(desc, precision, ladder, batch_gb=2.0) -> int:
    return int(_server_lib().cdcc_job_footprint(ctypes.byref(desc),
                                                int(precision), int(ladder),
                                                float(batch_gb)))


def cdcc_energy_error(ctx) -> float:
    """Error report of E_corr (see include/cdcc.h)."""
    dE = ctypes.c_double()
    _check(ctx, _server_lib().cdcc_energy_error(ctx.handle,
                                                ctypes.byref(dE)))
    return dE.value


class Server:
    """Owns a cdcc_server* (include/cdcc.h serving entry points)."""

    def __init__(self, options: cdcc_options | None = None,
                 server_options: cdcc_server_options | None = None):
        lib = _server_lib()
        self.opt = options if options is not None else cdcc_default_options()
        self.sopt = (server_options if server_options is not None
                     else cdcc_server_default_options())
        self.handle = ctypes.c_void_p()
        self._keep = {}
        st = lib.cdcc_server_create(ctypes.byref(self.handle),
                                    ctypes.byref(self.opt),
                                    ctypes.byref(self.sopt))
        if st != CDCC_OK:
            raise CdccError(st, "cdcc_server_create failed")

    def submit(self, desc, keep) -> int:
        t = ctypes.c_uint64()
        st = _server_lib().cdcc_submit(self.handle, ctypes.byref(desc),
                                       ctypes.byref(t))
        if st != CDCC_OK:
            raise CdccError(st, "cdcc_submit failed")
        return int(t.value)

    def poll(self, ticket, nx):
        g = np.zeros(max(nx, 1))
        r = cdcc_result()
        r.g = g.ctypes.data
        st = _server_lib().cdcc_poll(self.handle, ctypes.c_uint64(ticket),
                                     ctypes.byref(r))
        if st != CDCC_OK:
            raise CdccError(st, "cdcc_poll failed")
        return r, g[:nx]

    def wait(self, ticket, nx, timeout_s=-1.0):
        g = np.zeros(max(nx, 1))
        r = cdcc_result()
        r.g = g.ctypes.data
        st = _server_lib().cdcc_wait(self.handle, ctypes.c_uint64(ticket),
                                     float(timeout_s), ctypes.byref(r))
        if st not in (CDCC_OK, CDCC_ETIMEOUT):
            raise CdccError(st, "cdcc_wait failed")
        return r, g[:nx]

    def max_active_seen(self) -> int:
        return int(_server_lib().cdcc_server_max_active_seen(self.handle))

    def close(self):
        if self.handle:
            _server_lib().cdcc_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
