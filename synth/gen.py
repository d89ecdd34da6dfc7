"""Seeded generators for the synthetic CD-CCSD gradient workloads.

Every workload is a closed-shell system described only by
  * the irrep label of each molecular orbital (occupied orbitals first, each
    space ordered irrep-major),
  * the orbital energies eps_p,
  * MO Cholesky vectors L^P_pq, symmetric in pq and nonzero only where
    irrep(p) x irrep(q) = irrep(P) (the selection rule of Sec. 3.1), and
  * derivative vectors dL^P_pq/dx for a set of displacements x.

Irreps of an Abelian group are numbered 0..h-1 in the Z2^k ordering, so the
direct product is the bitwise XOR of the labels.

Packed ("L-pattern") layout of a Cholesky tensor, used at the library
boundary and in the tests:
    for G_P in 0..h-1:                      (irrep of the Cholesky vector)
      for k in 0..nchol[G_P]-1:             (vector within that irrep)
        for G_p in 0..h-1:                  (irrep of the row orbital)
          G_q = G_p ^ G_P ^ G_x             (G_x = irrep of the displacement;
                                             0 for L itself)
          block[p][q], p over the orbitals of irrep G_p, q over those of
          irrep G_q, both in ascending global order, row-major.

Nothing here computes anything the method computes: the generator draws
uniform / normal deviates and arranges them.  The per-workload scale factor
s_cfg (which multiplies L and dL) is a constant; it was chosen once so that
the MP2 correlation energy is about -0.04 Eh per occupied orbital, by the
script oracle/calibrate_scale.py.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

BASE_SEED = 20251221909

# Workloads.  "split" is either "even" or per-irrep fractions.
CONFIGS = {
    0: dict(name="c0", group="C1", nirrep=1, o=4, v=20, nchol=60, nx=6,
            split="even"),
    1: dict(name="c1", group="D2h", nirrep=8, o=16, v=144, nchol=640, nx=18,
            split="even"),
    2: dict(name="c2", group="C2v", nirrep=4, o=40, v=360, nchol=1600, nx=24,
            split=(0.40, 0.25, 0.20, 0.15)),
    3: dict(name="c3", group="D2h", nirrep=8, o=60, v=540, nchol=2400, nx=36,
            split="even"),
}

# s_cfg per workload (see module docstring); 1.0 reproduces the literal
# distribution L = N(0,1) * 0.3 * exp(-3P/nL).
SCALES = {0: 0.2561805150834829, 1: 0.10978620925793245,
          2: 0.03160092428148088, 3: 0.02984614109045192}


@dataclass
class System:
    name: str
    nirrep: int
    occ: list
    vir: list
    chol: list
    orb_irrep: np.ndarray
    eps: np.ndarray
    chol_irrep: np.ndarray
    L: np.ndarray
    scale: float = 1.0
    seed: int = 0
    cfg_index: int = -1
    extra: dict = field(default_factory=dict)

    @property
    def nocc(self):
        return int(sum(self.occ))

    @property
    def nvir(self):
        return int(sum(self.vir))

    @property
    def n(self):
        return self.nocc + self.nvir

    @property
    def nchol(self):
        return int(sum(self.chol))

    def norb_irrep(self):
        return [self.occ[g] + self.vir[g] for g in range(self.nirrep)]

    def nnz(self, gx: int = 0) -> int:
        return packed_size(self.nirrep, self.norb_irrep(), self.chol, gx)


def irrep_split(total: int, nirrep: int, split) -> list:
    """Split `total` over irreps: floor + largest remainder, ties to the
    lower irrep."""
    if split == "even":
        frac = np.full(nirrep, 1.0 / nirrep)
    else:
        frac = np.asarray(split, dtype=np.float64)
        assert len(frac) == nirrep
    exact = frac * total
    base = np.floor(exact + 1e-12).astype(int)
    rem = exact - base
    left = total - int(base.sum())
    order = sorted(range(nirrep), key=lambda g: (-round(rem[g], 12), g))
    for g in order[:left]:
        base[g] += 1
    return [int(x) for x in base]


def pair_count(nirrep: int, norb: list, gamma: int) -> int:
    return int(sum(norb[g] * norb[g ^ gamma] for g in range(nirrep)))


def chol_split(total: int, nirrep: int, norb: list) -> list:
    """Cholesky vectors per irrep, proportional to the number of orbital
    pairs of that irrep (floor + largest remainder)."""
    npp = np.array([pair_count(nirrep, norb, g) for g in range(nirrep)],
                   dtype=np.float64)
    return irrep_split(total, nirrep, tuple(npp / npp.sum()))


def packed_size(nirrep, norb, chol, gx=0) -> int:
    return int(sum(chol[gP] * sum(norb[gp] * norb[gp ^ gP ^ gx]
                                  for gp in range(nirrep))
                   for gP in range(nirrep)))


def _orbital_labels(nirrep, occ, vir):
    lab = []
    for g in range(nirrep):
        lab += [g] * occ[g]
    for g in range(nirrep):
        lab += [g] * vir[g]
    return np.asarray(lab, dtype=np.int32)


def _irrep_members(orb_irrep, nirrep):
    return [np.nonzero(orb_irrep == g)[0] for g in range(nirrep)]


def _draw_symmetric_pattern(rng, nirrep, norb, chol, amp_of, gx=0):
    """Draw one packed Cholesky-pattern tensor.  For each irrep G_P and each
    row irrep G_p a block of standard normals X[G_p] (nchol_GP, n_Gp, n_Gq)
    is drawn; the stored block is amp * (X[G_p] + X[G_q]^T) / 2, i.e. the
    (X + X^T)/2 symmetrisation of the full matrix restricted to the pattern."""
    out = []
    for gP in range(nirrep):
        nP = chol[gP]
        X = []
        for gp in range(nirrep):
            gq = gp ^ gP ^ gx
            X.append(rng.standard_normal((nP, norb[gp], norb[gq])))
        amp = amp_of(gP, nP)[:, None, None]
        for gp in range(nirrep):
            gq = gp ^ gP ^ gx
            blk = 0.5 * (X[gp] + X[gq].transpose(0, 2, 1))
            out.append((amp * blk).reshape(nP, norb[gp] * norb[gq]))
    # reorder to G_P, k, G_p: the blocks above are grouped per G_P as
    # [G_p=0 (nP x ...), G_p=1 ...]; interleave per vector k
    flat = []
    i = 0
    for gP in range(nirrep):
        blocks = out[i:i + nirrep]
        i += nirrep
        if chol[gP] == 0:
            continue
        flat.append(np.concatenate(blocks, axis=1).reshape(-1))
    if not flat:
        return np.zeros(0)
    return np.concatenate(flat)


def make_system(cfg_index: int, scale: float | None = None) -> System:
    cfg = CONFIGS[cfg_index]
    h = cfg["nirrep"]
    occ = irrep_split(cfg["o"], h, cfg["split"])
    vir = irrep_split(cfg["v"], h, cfg["split"])
    norb = [occ[g] + vir[g] for g in range(h)]
    chol = chol_split(cfg["nchol"], h, norb)
    s = SCALES[cfg_index] if scale is None else scale
    seed = BASE_SEED + cfg_index
    sysm = random_system(occ, vir, chol, seed=seed, scale=s,
                         name=cfg["name"])
    sysm.cfg_index = cfg_index
    return sysm


def random_system(occ, vir, chol, seed, scale=1.0, name="custom",
                  eps_occ=(-1.5, -0.3), eps_vir=(0.1, 3.0)) -> System:
    h = len(occ)
    assert len(vir) == h and len(chol) == h and h in (1, 2, 4, 8)
    rng = np.random.Generator(np.random.PCG64(seed))
    orb_irrep = _orbital_labels(h, occ, vir)
    o, v = int(sum(occ)), int(sum(vir))
    e_o = rng.uniform(eps_occ[0], eps_occ[1], o)
    e_v = rng.uniform(eps_vir[0], eps_vir[1], v)
    eps = np.concatenate([e_o, e_v])
    # sort ascending inside each (space, irrep) segment
    start = 0
    for counts in (occ, vir):
        for g in range(h):
            seg = slice(start, start + counts[g])
            eps[seg] = np.sort(eps[seg])
            start += counts[g]
    norb = [occ[g] + vir[g] for g in range(h)]

    def amp_of(gP, nP):
        k = np.arange(nP, dtype=np.float64)
        return scale * 0.3 * np.exp(-3.0 * k / max(nP, 1))

    L = _draw_symmetric_pattern(rng, h, norb, chol, amp_of)
    chol_irrep = np.concatenate([np.full(chol[g], g, dtype=np.int32)
                                 for g in range(h)]) if sum(chol) else \
        np.zeros(0, np.int32)
    return System(name=name, nirrep=h, occ=list(occ), vir=list(vir),
                  chol=list(chol), orb_irrep=orb_irrep, eps=eps,
                  chol_irrep=chol_irrep, L=L, scale=scale, seed=seed)


def make_displacements(sysm: System, nx: int | None = None,
                       sigma: float = 0.05) -> np.ndarray:
    """Totally symmetric displacement derivatives dL/dx, shape (nx, nnz),
    drawn N(0, sigma) * s_cfg with L's block pattern and symmetrisation."""
    if nx is None:
        nx = CONFIGS[sysm.cfg_index]["nx"] if sysm.cfg_index >= 0 else 6
    rng = np.random.Generator(np.random.PCG64(sysm.seed + 7919))
    norb = sysm.norb_irrep()
    out = np.empty((nx, sysm.nnz()))

    def amp_of(gP, nP):
        return np.full(nP, sigma * sysm.scale)

    for x in range(nx):
        out[x] = _draw_symmetric_pattern(rng, sysm.nirrep, norb, sysm.chol,
                                         amp_of)
    return out


def make_displacement_nontotsym(sysm: System, gx: int, seed_offset=1,
                                sigma: float = 0.05) -> np.ndarray:
    """One displacement of irrep gx != 0: dL^P_pq nonzero only where
    irrep(p) x irrep(q) x irrep(P) = gx.  Packed with the same loop order
    as L (G_q = G_p ^ G_P ^ gx)."""
    rng = np.random.Generator(np.random.PCG64(sysm.seed + 104729 +
                                              seed_offset))
    norb = sysm.norb_irrep()

    def amp_of(gP, nP):
        return np.full(nP, sigma * sysm.scale)

    return _draw_symmetric_pattern(rng, sysm.nirrep, norb, sysm.chol, amp_of,
                                   gx=gx)


def unpack_dense(sysm: System, packed: np.ndarray, gx: int = 0) -> np.ndarray:
    """Packed pattern -> dense (nchol, n, n) array (zeros off-pattern)."""
    h = sysm.nirrep
    mem = _irrep_members(sysm.orb_irrep, h)
    n = sysm.n
    dense = np.zeros((sysm.nchol, n, n))
    pos = 0
    P0 = 0
    for gP in range(h):
        nP = sysm.chol[gP]
        for k in range(nP):
            for gp in range(h):
                gq = gp ^ gP ^ gx
                rp, rq = mem[gp], mem[gq]
                sz = len(rp) * len(rq)
                dense[P0 + k][np.ix_(rp, rq)] = \
                    packed[pos:pos + sz].reshape(len(rp), len(rq))
                pos += sz
        P0 += nP
    assert pos == packed.size
    return dense


def pack_dense(sysm: System, dense: np.ndarray, gx: int = 0) -> np.ndarray:
    h = sysm.nirrep
    mem = _irrep_members(sysm.orb_irrep, h)
    out = []
    P0 = 0
    for gP in range(h):
        nP = sysm.chol[gP]
        for k in range(nP):
            for gp in range(h):
                gq = gp ^ gP ^ gx
                out.append(dense[P0 + k][np.ix_(mem[gp], mem[gq])].reshape(-1))
        P0 += nP
    return np.concatenate(out) if out else np.zeros(0)


def as_c1(sysm: System, packed_extra=()):
    """The same data with every irrep label set to 0 (symmetry ignored).
    Returns the C1 system and the C1-packed versions of `packed_extra`
    (each a packed array of the symmetric system, totally symmetric)."""
    dense = unpack_dense(sysm, sysm.L)
    c1 = System(name=sysm.name + "-C1", nirrep=1, occ=[sysm.nocc],
                vir=[sysm.nvir], chol=[sysm.nchol],
                orb_irrep=np.zeros(sysm.n, np.int32), eps=sysm.eps.copy(),
                chol_irrep=np.zeros(sysm.nchol, np.int32),
                L=dense.reshape(-1).copy(), scale=sysm.scale, seed=sysm.seed,
                cfg_index=sysm.cfg_index)
    extra = [unpack_dense(sysm, p).reshape(-1) for p in packed_extra]
    return c1, extra
