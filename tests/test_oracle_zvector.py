"""Pins of the orbital-relaxation oracle (oracle/zvector.py; Sec. 2.5,
Eq. z_vector) against what the mathematics fixes (CPU only):

  * the relaxed gradient <Gamma^P + Gamma_Z^P, dL_x> equals a central
    difference (Richardson) of the relaxed energy, i.e. of CCSD re-solved in
    orbitals re-optimised by Newton iterations on the Brillouin condition
    at every displaced L;
  * the Hessian of the Brillouin condition (reverse mode) is the bracket of
    Eq. z_vector read with <pq|rs> = (pr|qs);
  * the orbital gradient written from the densities, 2 [h, D] + 2 sum_P
    [L^P, Gamma^P], equals the reverse-mode derivative of the Lagrangian
    with respect to the rotation;
  * the relaxation density written out equals its reverse-mode definition;
  * the relaxed gradient differs from the unrelaxed one (the test has
    teeth), and a planted mistake (the exchange part of the Hessian
    dropped) breaks the finite-difference pin.
"""
import numpy as np
import pytest
import torch

from synth import make_system, random_system, make_displacements, unpack_dense
from oracle import model, lagrangian, zvector

T = lambda x: torch.as_tensor(np.asarray(x), dtype=torch.float64)  # noqa


def _setup(which):
    if which == "c0":
        s = make_system(0)
    else:
        s = random_system([2, 1, 1, 1], [4, 3, 3, 2], [8, 6, 6, 6],
                          seed=13, scale=0.35)
    o = s.nocc
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    dL = T(np.stack([unpack_dense(s, x) for x in make_displacements(s, 2)]))
    return s, o, L, h, dL


def _fd(h, L, o, d, steps=(1e-3, 5e-4)):
    fd = [(zvector.relaxed_energy(h, L + e * d, o)
           - zvector.relaxed_energy(h, L - e * d, o)) / (2 * e)
          for e in steps]
    return (4.0 * fd[1] - fd[0]) / 3.0


@pytest.mark.parametrize("which", ["c0", "sym"])
def test_relaxed_gradient_matches_finite_difference(which):
    s, o, L, h, dL = _setup(which)
    r = lagrangian.run_all(h, L, o, tol=1e-12, e_tol=1e-13)
    g, Z, _ = zvector.relaxed_gradient(r, h, L, o, dL)
    g0 = lagrangian.gradient_from_density(r["G"], dL)
    for x in range(dL.shape[0]):
        fd = _fd(h, L, o, dL[x])
        assert abs(float(g[x]) - fd) < 1e-8, (x, float(g[x]), fd)
        # relaxation matters at this accuracy
        assert abs(float(g0[x]) - fd) > 1e-6, (x, float(g0[x]), fd)
    assert float(Z.abs().max()) > 1e-6


@pytest.mark.parametrize("which", ["c0", "sym"])
def test_orbital_hessian_is_the_z_vector_bracket(which):
    s, o, L, h, _ = _setup(which)
    A = zvector.orbital_hessian(h, L, o)              # [b, j, a, i]
    H = zvector.orbital_hessian_eq(T(s.eps), L, o)    # [a, i, e, m]
    assert float((A.permute(2, 3, 0, 1) - H).abs().max()) <= 1e-12 * float(
        H.abs().max())


@pytest.mark.parametrize("which", ["c0", "sym"])
def test_orbital_gradient_and_relaxation_density_from_densities(which):
    s, o, L, h, _ = _setup(which)
    r = lagrangian.run_all(h, L, o, tol=1e-12, e_tol=1e-13)
    t1, t2 = r["cc"]["t1"], r["cc"]["t2"]
    l1, l2 = r["lam"]["l1"], r["lam"]["l2"]
    ref = zvector.lagrangian_orbital_gradient(t1, t2, l1, l2, h, L, o)
    got = zvector.orbital_gradient(r["D"], r["G"], h, L, o)
    assert float((got - ref).abs().max()) <= 1e-11 * max(
        1.0, float(ref.abs().max()))
    Z = T(np.random.default_rng(3).standard_normal(ref.shape))
    a = zvector.relaxation_density(Z, h, L, o)
    b = zvector.relaxation_density_eq(Z, L, o)
    assert float((a - b).abs().max()) <= 1e-12 * float(a.abs().max())


def test_planted_hessian_mistake_is_caught(monkeypatch):
    s, o, L, h, dL = _setup("c0")
    r = lagrangian.run_all(h, L, o, tol=1e-12, e_tol=1e-13)
    good = zvector.orbital_hessian_eq(T(s.eps), L, o)
    # the paper's bracket without its exchange parts
    Lvv, Loo, Lvo = L[:, o:, o:], L[:, :o, :o], L[:, o:, :o]
    bad = good + torch.einsum("Pea,Pim->aiem", Lvv, Loo) \
        + torch.einsum("Pei,Pam->aiem", Lvo, Lvo)
    monkeypatch.setattr(zvector, "orbital_hessian",
                        lambda h_, L_, o_: bad.permute(2, 3, 0, 1))
    g, _, _ = zvector.relaxed_gradient(r, h, L, o, dL)
    fd = _fd(h, L, o, dL[0])
    assert abs(float(g[0]) - fd) > 1e-7


def test_stored_relaxed_values_are_the_oracle_s():
    # tests/golden/c0_relaxed.json (make_golden.py relaxed0) against a fresh
    # oracle evaluation, and its unrelaxed part against c0.json
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    gold = json.load(open(os.path.join(here, "c0_relaxed.json")))
    base = json.load(open(os.path.join(here, "c0.json")))
    s = make_system(0)
    o = s.nocc
    L = T(unpack_dense(s, s.L))
    h = model.core_from_eps(T(s.eps), L, o)
    r = lagrangian.run_all(h, L, o, tol=1e-11, e_tol=1e-13)
    dL = T(np.stack([unpack_dense(s, x) for x in make_displacements(s)]))
    g, _, _ = zvector.relaxed_gradient(r, h, L, o, dL)
    assert np.abs(g.numpy() - np.array(gold["gradient"])).max() < 1e-9
    assert np.abs(np.array(gold["gradient_unrelaxed"])
                  - np.array(base["gradient"])).max() < 1e-9
