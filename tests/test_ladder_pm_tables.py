"""Index tables of the +/- packed ladder, as the library builds them
(cdcc_ladder_pm_tables: host code, no GPU), against the DPD block layout
of the doubles (rows (i,j) in sub-blocks by irrep(i), columns (c,d) by
irrep(c)) and the pair symmetry of Sec. 2.3:

  * canonical pairs only (irrep(p) > irrep(q), or the same irrep and
    p >= q), each once; the second table entry is the swapped pair;
  * the unpack writes every element of every block exactly once
    (rows (i,j), (j,i) x columns (a,b), (b,a)), all offsets in bounds;
  * the A+- gather reads every column once as (c,d) or (d,c);
  * batches cover each canonical (a,b) once, with rows inside the batch.
Shapes: D2h with ragged and empty irreps, C2v, C1, one-row batches.
"""
import numpy as np
import pytest

from paper_2512_21909_gb300 import cdcc


def _sub(n, h, G):
    """first offset of each sub-block (irrep of the first index) in G."""
    off, t = [], 0
    for g in range(h):
        off.append(t)
        t += n[g] * n[g ^ G]
    return off, t


def _decode(off, n, h, G, x):
    """(irrep, p, q) of the pair stored at offset x of block G."""
    for g in range(h - 1, -1, -1):
        if n[g] * n[g ^ G] and x >= off[g]:
            r = x - off[g]
            m = n[g ^ G]
            return g, r // m, r % m
    raise AssertionError(x)


SHAPES = [
    ([8, 7, 8, 7, 8, 7, 8, 7], [12, 11, 12, 11, 12, 11, 12, 11], 2.0),
    ([3, 2, 0, 1, 2, 0, 1, 1], [5, 4, 3, 0, 2, 3, 4, 1], 2.0),
    ([4, 3, 2, 1], [12, 10, 8, 6], 2.0),
    ([4, 3, 2, 1], [12, 10, 8, 6], 1e-9),       # one a per batch
    ([5], [9], 2.5e-6),
]


@pytest.mark.parametrize("occ,vir,gb", SHAPES)
def test_pm_tables_cover_every_element_once(occ, vir, gb):
    h = len(occ)
    tabs = cdcc.ladder_pm_tables(occ, vir, gb)
    for G in range(h):
        ooff, nrow = _sub(occ, h, G)
        voff, ncol = _sub(vir, h, G)
        if nrow == 0 or ncol == 0:
            assert G not in tabs
            continue
        t = tabs[G]
        assert (t["nrow"], t["ncol"]) == (nrow, ncol)
        # canonical occupied pairs and their swaps
        seen = set()
        for x1, x2 in zip(t["r1"], t["r2"]):
            gi, i, j = _decode(ooff, occ, h, G, int(x1))
            gj, j2, i2 = _decode(ooff, occ, h, G, int(x2))
            assert gj == gi ^ G and (i2, j2) == (i, j)
            assert gi > gj or (gi == gj and i >= j)
            seen.add((gi, i, j))
        assert len(seen) == len(t["r1"])
        # the A+- gather reads each column once
        cov = np.zeros(ncol, int)
        np.add.at(cov, t["c1"], 1)
        np.add.at(cov, t["c2"][t["c1"] != t["c2"]], 1)
        assert (cov == 1).all()
        for x1, x2 in zip(t["c1"], t["c2"]):
            gc, c, d = _decode(voff, vir, h, G, int(x1))
            gd, d2, c2 = _decode(voff, vir, h, G, int(x2))
            assert gd == gc ^ G and (c2, d2) == (c, d)
            assert gc > gd or (gc == gd and c >= d)
        # the unpack writes each element of the block exactly once
        cnt = np.zeros((nrow, ncol), np.int32)
        r1, r2 = t["r1"], t["r2"]
        off_diag = r1 != r2
        for b in t["batches"]:
            ga, gbb = b["ga"], b["ga"] ^ G
            assert ga >= gbb
            nb = vir[gbb]
            rows = (b["a1"] - b["a0"]) * nb
            assert ((b["lr"] >= 0) & (b["lr"] < rows)).all()
            for lr, y1, y2 in zip(b["lr"], b["y1"], b["y2"]):
                a, bb = b["a0"] + lr // nb, lr % nb
                assert y1 == voff[ga] + a * nb + bb
                if ga == gbb:
                    assert bb <= a and (y2 == -1) == (a == bb)
                if y2 >= 0:
                    assert y2 == voff[gbb] + bb * vir[ga] + a
            m = b["y2"] >= 0
            np.add.at(cnt, (r1[:, None], b["y1"][None, :]), 1)
            np.add.at(cnt, (r1[:, None], b["y2"][None, m]), 1)
            np.add.at(cnt, (r2[off_diag][:, None], b["y1"][None, :]), 1)
            np.add.at(cnt, (r2[off_diag][:, None], b["y2"][None, m]), 1)
        assert (cnt == 1).all(), (G, np.unique(cnt, return_counts=True))


def test_pm_tables_reject_bad_arguments():
    with pytest.raises(cdcc.CdccError):
        cdcc.ladder_pm_tables([1, 2, 3], [4, 5, 6])      # 3 irreps
    with pytest.raises(cdcc.CdccError):
        cdcc.ladder_pm_tables([1, -2], [4, 5])
    with pytest.raises(cdcc.CdccError):
        cdcc.ladder_pm_tables([1, 2], [4, 5], batch_gb=0.0)
