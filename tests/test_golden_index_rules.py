"""The oracle's per-sample index rules against rows worked by hand (tests/golden/index_rules.txt):
pixel of the first tap, oversampling offset, signed w-plane, and the keep/drop decision, including
the ties and the first and last kept positions.  The inputs are dyadic, so every intermediate value
of the rules is exact in FP64 and the rows follow from the rules alone."""
import os

import numpy as np

from oracle import cf as ocf
from oracle import index as oindex

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "index_rules.txt")


def load_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        f = line.split()
        uvw = tuple(float(t) for t in f[:3])
        kept = f[3] == "1"
        rest = tuple(int(t) for t in f[4:9]) if kept else None
        rows.append((uvw, kept, rest))
    return rows


def test_index_rules_match_the_hand_worked_rows():
    rows = load_rows()
    assert len(rows) == 14
    p = ocf.CFParams(grid_n=64, cell_rad=1.0 / 512.0, oversampling=20, ps_support=7, use_w=True, n_wplanes=5,
                     w_max_lambda=8.0, max_support=8)
    assert set(ocf.supports(p).tolist()) == {8}
    uvw = np.array([r[0] for r in rows], dtype=np.float64)
    idx = oindex.sample_index(p, uvw, np.array([oindex.C_LIGHT]))
    for i, (uvw_i, kept, rest) in enumerate(rows):
        assert bool(idx.valid[i]) == kept, (i, uvw_i)
        if kept:
            ks, p0x, p0y, ox, oy = rest
            got = (int(idx.cf[i]), int(idx.p0x[i]), int(idx.p0y[i]), int(idx.ox[i]), int(idx.oy[i]))
            assert got == (ks, p0x, p0y, ox, oy), (i, uvw_i, got)
            assert int(idx.support[i]) == 8
