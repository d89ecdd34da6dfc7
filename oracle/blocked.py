"""Einstein summation restricted to the symmetry-allowed irrep blocks
(oracle helper; Abelian point groups, Sec. 3.1).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
CPU baseline may import this module; the library never does.

Every tensor of the closed-shell CCSD equations with Cholesky vectors is
totally symmetric: an element vanishes unless the irreps of its indices
multiply (XOR, irreps 0..h-1 as Z2^k) to the totally symmetric irrep -- for
L^P_pq the Cholesky index P carries the irrep of the pair pq.  A product of
such tensors therefore only needs the index blocks whose irreps make every
operand totally symmetric; all other blocks multiply zeros.  `irrep_einsum`
runs torch.einsum on exactly those blocks and adds them into a zero output,
so it equals the dense einsum for totally symmetric operands (pinned in
tests/test_oracle_blocked.py against the dense evaluation).  The dense
oracle stays the definition; this form only makes the Lagrangian affordable
at sizes where the dense one takes hours.

The index letters name spaces: i j k l m n occupied, a b c d e f virtual,
P Cholesky vectors.  Each space's indices must be sorted by irrep, so that
an irrep is one contiguous range.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

OCC, VIR = "ijklmn", "abcdef"


def _ranges(lab):
    out = {}
    for g in np.unique(lab):
        idx = np.nonzero(lab == g)[0]
        if idx[-1] - idx[0] + 1 != idx.size:
            raise ValueError("indices of a space must be sorted by irrep")
        out[int(g)] = (int(idx[0]), int(idx[-1]) + 1)
    return out


def irrep_einsum(occ_irrep, vir_irrep, chol_irrep):
    """An einsum-compatible function over the allowed blocks; the keyword
    `ranges` = {letter: (start, stop)} says that an operand holds only that
    sub-range of the letter's space (a block of virtuals, say)."""
    labels = {}
    for c in OCC:
        labels[c] = np.asarray(occ_irrep)
    for c in VIR:
        labels[c] = np.asarray(vir_irrep)
    labels["P"] = np.asarray(chol_irrep)

    def ein(spec, *ops, ranges=None):
        lhs, out = spec.replace(" ", "").split("->")
        terms = lhs.split(",")
        letters = sorted(set("".join(terms)))
        rng = {}
        for c in letters:
            lab = labels[c]
            if ranges and c in ranges:
                lab = lab[ranges[c][0]:ranges[c][1]]
            rng[c] = _ranges(lab)
        size = {}
        for op, term in zip(ops, terms):
            for ax, c in enumerate(term):
                size[c] = op.shape[ax]
        res = torch.zeros([size[c] for c in out], dtype=ops[0].dtype)
        for combo in itertools.product(*(sorted(rng[c]) for c in letters)):
            g = dict(zip(letters, combo))
            ok = True
            for term in terms:
                x = 0
                for c in term:
                    x ^= g[c]
                if x:
                    ok = False
                    break
            if not ok:
                continue
            blocks = [op[tuple(slice(*rng[c][g[c]]) for c in term)]
                      for op, term in zip(ops, terms)]
            res[tuple(slice(*rng[c][g[c]]) for c in out)] += torch.einsum(
                spec, *blocks)
        return res

    return ein


def for_system(s):
    """irrep_einsum for a synth System (orbitals: occupied, then virtual)."""
    irr = np.asarray(s.orb_irrep)
    return irrep_einsum(irr[:s.nocc], irr[s.nocc:], np.asarray(s.chol_irrep))
