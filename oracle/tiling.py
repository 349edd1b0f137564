"""Tiling of the Lagrangian lattice, buffer regions and sCOLA boxes (Sec. 3.2).

Test infrastructure (see ``oracle/__init__``).

Step B.1: the Np^3 lattice is split into Ntiles^3 cubic tiles of
Np,tile = Np / Ntiles particles per side (Np must be a multiple of Ntiles).
Each tile is surrounded by Np,buffer particles on every side; its sCOLA box
holds Np,sCOLA = Np,tile + 2 Np,buffer particles per side (wrapped periodically
on the lattice).  Over-simulation r and parallelisation potential p follow
Eqs. 20-21 (for uneven buffers r sums the box volumes).  Step B.2 keeps only
tile particles at the end.

Index conventions (a reading; the paper does not fix an order):
  * particle (i, j, k), k fastest, has global id (i Np + j) Np + k and sits at
    q = ((i + 1/2), (j + 1/2), (k + 1/2)) dq, dq = L / Np;
  * tile (tx, ty, tz) has box id (tx Ntiles + ty) Ntiles + tz and owns lattice
    indices [t Np,tile, (t+1) Np,tile) per axis;
  * box-local lattice index b in [0, Np,sCOLA) maps to the global index
    (t Np,tile - Np,buffer + b) mod Np; box-local ids are (bi Nsc + bj) Nsc + bk;
  * the box-local frame has its origin at (t Np,tile - Np,buffer) dq, so the
    box particle b sits at q_loc = (b + 1/2) dq and the box spans [0, L_sCOLA).

Pins (tests/test_oracle_tiling.py): the 16 rows of Table 1 (r, p, L_tile,
L_buffer and Ng = Np,sCOLA + 1) from tests/golden/table1_setups.txt; every
global particle belongs to exactly one tile interior; box membership equals a
brute-force periodic-distance definition.
"""
import numpy as np


def tile_coords(Ntiles):
    """Tile coordinates (tx, ty, tz) in box-id order (tz fastest)."""
    r = np.arange(Ntiles)
    tx, ty, tz = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([tx.ravel(), ty.ravel(), tz.ravel()], axis=1)


def box_axis_indices(Np, Ntiles, t_axis, Nbuf):
    """Global lattice indices along one axis covered by a box (Sec. 3.2)."""
    Ntile = Np // Ntiles
    Nsc = Ntile + 2 * Nbuf
    return (t_axis * Ntile - Nbuf + np.arange(Nsc)) % Np


def box_global_ids(Np, Ntiles, t, Nbuf):
    """Global particle ids of a box's particles in box-local order."""
    ix = box_axis_indices(Np, Ntiles, t[0], Nbuf)
    iy = box_axis_indices(Np, Ntiles, t[1], Nbuf)
    iz = box_axis_indices(Np, Ntiles, t[2], Nbuf)
    return ((ix[:, None, None] * Np + iy[None, :, None]) * Np + iz[None, None, :]).ravel().astype(np.int64)


def box_local_lattice(Nsc):
    """Box-local lattice indices (bi, bj, bk) of every box particle, shape (Nsc^3, 3)."""
    r = np.arange(Nsc)
    bi, bj, bk = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([bi.ravel(), bj.ravel(), bk.ravel()], axis=1)


def tile_interior_mask(Np, Ntiles, Nbuf):
    """Boolean mask over box-local ids: True for tile particles (kept at B.2)."""
    Ntile = Np // Ntiles
    b = box_local_lattice(Ntile + 2 * Nbuf)
    inside = (b >= Nbuf) & (b < Nbuf + Ntile)
    return inside.all(axis=1)


def box_origin(Np, Ntiles, t, Nbuf, L):
    """Origin of the box-local frame in full-box coordinates (may be negative)."""
    Ntile = Np // Ntiles
    dq = L / Np
    return (np.asarray(t, dtype=np.float64) * Ntile - Nbuf) * dq


def oversimulation(Np, Ntiles, Nbufs):
    """Over-simulation factor r (Eq. 20) and parallelisation potential p (Eq. 21).

    ``Nbufs`` is a scalar (same buffer for every tile) or one buffer per tile.
    p is Ntiles^3 / r, which equals Np^3 / Np,sCOLA^3 for uniform buffers.
    """
    Ntile = Np // Ntiles
    nb = np.broadcast_to(np.asarray(Nbufs, dtype=np.int64), (Ntiles**3,))
    Nsc = Ntile + 2 * nb
    r = float(np.sum(Nsc.astype(np.float64) ** 3)) / float(Np) ** 3
    return r, Ntiles**3 / r


def lpt_grid_portion(Np, N, Ntile_p, Nbuf_p):
    """N_tile and N_sCOLA, the LPT-grid portions covering a tile and a box (Eq. 22)."""
    Ntile = int(np.ceil(Ntile_p * N / Np))
    return Ntile, Ntile + 2 * int(np.ceil(Nbuf_p * N / Np))
