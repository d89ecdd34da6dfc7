"""The symmetry-blocked einsum of oracle/blocked.py equals the dense einsum
on totally symmetric tensors, and the oracle's residual and Lagrangian
evaluated with it equal the dense ones (CPU only; D2h c1 sizes, C2v and a
group with empty irreps).  A planted mistake (wrong irrep labels) is
caught."""
import numpy as np
import pytest
import torch

from synth import make_system, random_system, unpack_dense
from oracle import model, ccsd, lagrangian, blocked

T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa


def _sym_tensor(rng, labs):
    shape = [len(l) for l in labs]
    x = rng.standard_normal(shape)
    mask = np.zeros(shape, dtype=int)
    for ax, l in enumerate(labs):
        sh = [1] * len(labs)
        sh[ax] = len(l)
        mask = mask ^ np.asarray(l).reshape(sh)
    return T(x * (mask == 0))


def test_blocked_einsum_equals_dense():
    rng = np.random.default_rng(0)
    occ = np.repeat(np.arange(4), [3, 2, 0, 2])       # an empty irrep
    vir = np.repeat(np.arange(4), [5, 4, 3, 2])
    chol = np.repeat(np.arange(4), [6, 5, 4, 3])
    ein = blocked.irrep_einsum(occ, vir, chol)
    lab = {"i": occ, "j": occ, "k": occ, "l": occ, "a": vir, "b": vir,
           "c": vir, "d": vir, "P": chol}
    for spec in ["Pia,Pjb->iajb", "ijcd,acbd->ijab", "kicd,Pkc->Pid",
                 "ijcd,kcld->kilj", "iajb,ijab->", "ikac,kc->ia"]:
        lhs = spec.split("->")[0].split(",")
        ops = [_sym_tensor(rng, [lab[c] for c in t]) for t in lhs]
        ref = torch.einsum(spec, *ops)
        got = ein(spec, *ops)
        assert torch.allclose(got, ref, rtol=0, atol=1e-12 * max(
            1.0, float(ref.abs().max()))), spec
    # a sub-range of a letter's space
    ops = [_sym_tensor(rng, [chol, vir[2:7], vir]),
           _sym_tensor(rng, [chol, vir, vir])]
    ref = torch.einsum("Pac,Pbd->acbd", *ops)
    got = ein("Pac,Pbd->acbd", *ops, ranges={"a": (2, 7)})
    assert torch.allclose(got, ref, rtol=0, atol=1e-12)


def _random_amplitudes(s, seed):
    rng = np.random.default_rng(seed)
    irr = np.asarray(s.orb_irrep)
    o = s.nocc
    io, iv = irr[:o], irr[o:]
    m1 = io[:, None] == iv[None, :]
    m2 = ((io[:, None, None, None] ^ io[None, :, None, None]) ==
          (iv[None, None, :, None] ^ iv[None, None, None, :]))
    out = []
    for _ in range(2):
        t1 = 0.02 * rng.standard_normal(m1.shape) * m1
        t2 = 0.02 * rng.standard_normal(m2.shape) * m2
        out += [T(t1), T(0.5 * (t2 + t2.transpose(1, 0, 3, 2)))]
    return out


@pytest.mark.parametrize("which", ["c1", "c2_shape", "empty_irrep"])
def test_blocked_residual_and_lagrangian_equal_dense(which):
    if which == "c1":
        s = make_system(1)
    elif which == "c2_shape":
        s = random_system([4, 3, 2, 1], [12, 10, 8, 6], [20, 16, 14, 12],
                          seed=301, scale=0.3)
    else:
        s = random_system([1, 1, 0, 1, 0, 0, 1, 0], [3, 2, 2, 0, 1, 2, 2, 1],
                          [5, 3, 3, 3, 3, 3, 3, 2], seed=213, scale=0.45)
    o = s.nocc
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    t1, t2, l1, l2 = _random_amplitudes(s, 7)
    ein = blocked.for_system(s)
    with torch.no_grad():
        R1, R2, E = ccsd.residual(t1, t2, h, L, o)
        B1, B2, EB = ccsd.residual(t1, t2, h, L, o, ein)
        scale = float(R2.abs().max())
        assert float((B1 - R1).abs().max()) <= 1e-12 * scale
        assert float((B2 - R2).abs().max()) <= 1e-12 * scale
        assert abs(float(EB - E)) <= 1e-12 * max(1.0, abs(float(E)))
        if which != "c1":
            lag = lagrangian.lagrangian(t1, t2, l1, l2, h, L, o)
            lagb = lagrangian.lagrangian(t1, t2, l1, l2, h, L, o, ein)
            assert abs(float(lagb - lag)) <= 1e-12 * max(1.0,
                                                         abs(float(lag)))


def test_planted_wrong_labels_are_caught():
    s = random_system([4, 3, 2, 1], [12, 10, 8, 6], [20, 16, 14, 12],
                      seed=301, scale=0.3)
    o = s.nocc
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    t1, t2, _, _ = _random_amplitudes(s, 7)
    irr = np.asarray(s.orb_irrep)
    vir = irr[o:].copy()
    vir[11] = 1       # the last virtual of irrep 0 labelled as irrep 1
    bad = blocked.irrep_einsum(irr[:o], vir, np.asarray(s.chol_irrep))
    with torch.no_grad():
        _, R2, _ = ccsd.residual(t1, t2, h, L, o)
        _, B2, _ = ccsd.residual(t1, t2, h, L, o, bad)
    assert float((B2 - R2).abs().max()) > 1e-3 * float(R2.abs().max())
