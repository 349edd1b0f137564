"""Pins of the oracle's tiling arithmetic (Sec. 3.2, Eqs. 20-21, Table 1)."""
import os

import numpy as np
import pytest

from oracle import tiling

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_setups.txt")


def _table1_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _table1_rows())
def test_table1_setups(row):
    L, Np, N, Ntiles, Ntile, Ltile, Nbuf, Lbuf, Ng, r_pub, p_pub = row
    Np, Ntiles, Ntile, Nbuf, Ng = int(Np), int(Ntiles), int(Ntile), int(Nbuf), int(Ng)
    assert Np % Ntiles == 0 and Np // Ntiles == Ntile
    assert abs(L * Ntile / Np - Ltile) <= 0.05 + 1e-9          # printed to 0.1
    assert abs(L * Nbuf / Np - Lbuf) <= 0.05 + 1e-9
    r, p = tiling.oversimulation(Np, Ntiles, Nbuf)
    # printed to two decimals (integers when exact)
    assert abs(r - r_pub) <= 0.005 + 1e-9
    assert abs(p - p_pub) <= 0.005 + 1e-9
    # every setup of Table 1 uses Ng = Np,sCOLA + 1 (even Ng + 1, Sec. 4.4)
    assert Ng == Ntile + 2 * Nbuf + 1


@pytest.mark.parametrize("Np,Ntiles,Nbuf", [(12, 3, 2), (16, 2, 5), (8, 4, 1)])
def test_tile_interiors_partition_the_lattice(Np, Ntiles, Nbuf):
    seen = np.zeros(Np**3, dtype=np.int64)
    keep = tiling.tile_interior_mask(Np, Ntiles, Nbuf)
    for t in tiling.tile_coords(Ntiles):
        ids = tiling.box_global_ids(Np, Ntiles, t, Nbuf)
        np.add.at(seen, ids[keep], 1)
    assert np.all(seen == 1)


def test_box_membership_brute_force():
    # a box holds the lattice sites within Nbuf (periodic lattice distance, per axis) of its tile
    Np, Ntiles, Nbuf = 10, 2, 2
    Ntile = Np // Ntiles
    for t in tiling.tile_coords(Ntiles):
        ids = tiling.box_global_ids(Np, Ntiles, t, Nbuf)
        expected = set()
        for i in range(Np):
            for j in range(Np):
                for k in range(Np):
                    ok = True
                    for ax, v in enumerate((i, j, k)):
                        lo = t[ax] * Ntile - Nbuf
                        ok &= ((v - lo) % Np) < Ntile + 2 * Nbuf
                    if ok:
                        expected.add((i * Np + j) * Np + k)
        assert set(ids.tolist()) == expected
        assert len(ids) == (Ntile + 2 * Nbuf) ** 3


def test_uneven_buffers_oversimulation():
    Np, Ntiles = 16, 2
    bufs = [1, 2, 3, 4, 1, 2, 3, 4]
    r, p = tiling.oversimulation(Np, Ntiles, bufs)
    assert abs(r - sum((8 + 2 * b) ** 3 for b in bufs) / 16**3) < 1e-15
    assert abs(p - 8 / r) < 1e-12
