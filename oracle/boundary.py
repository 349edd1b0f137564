"""Dirichlet boundary potential on the padded PM grid (Sec. 3.3 C.3, Sec. 3.4 D.2, Eq. 23).

Test infrastructure (see ``oracle/__init__``).

The PM grid of a box has Ng^3 interior cells of size dg = L_sCOLA / Ng with
centres at (c + 1/2) dg in the box-local frame, padded by 2 Nghost = 2 cells on
every side (FDA order 2), i.e. padded indices c in [-2, Ng + 2) stored at array
index c + 2.  The Dirichlet planes of the DST-I solve are the first ghost
layers c = -1 and c = Ng (indices 0 and Ng + 1 of App. C).

C.3 interpolates the full-box phi1 (LPT grid nodes at (i + 1/2) d, periodic)
trilinearly (the CIC interpolation operator) to the centre of every padded cell
outside the interior.  The LEP approximation (Eq. 23) then gives
Phi_BCs(a_K) = D1(a_K) * shell at every force evaluation.  Interior cells of
the returned array are zero, matching App. C's Phi_BCs, which is non-zero only
outside the active domain.

Pins (tests/test_oracle_boundary.py): a constant phi1 is reproduced exactly;
the interpolation equals a brute-force sum of tent weights; a single smooth
Fourier mode is reproduced to the trilinear error bound.
"""
import numpy as np


def padded_cell_index(Ng, order=2):
    """Padded cell indices c = -P .. Ng + P - 1 along one axis, P = 2 N_ghost = order."""
    return np.arange(-order, Ng + order)


def interior_mask(Ng, order=2):
    """True on the Ng^3 interior cells of the padded (Ng + 2 order)^3 grid."""
    c = padded_cell_index(Ng, order)
    m = (c >= 0) & (c < Ng)
    return m[:, None, None] & m[None, :, None] & m[None, None, :]


def trilinear_periodic(field, L, X):
    """Trilinear interpolation of a periodic grid field (nodes at (i + 1/2) d) at points X (M, 3)."""
    N = field.shape[0]
    d = L / N
    u = X / d - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    out = np.zeros(X.shape[0])
    for dx in (0, 1):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dz in (0, 1):
                wz = f[:, 2] if dz else 1.0 - f[:, 2]
                out += wx * wy * wz * field[(i0[:, 0] + dx) % N, (i0[:, 1] + dy) % N,
                                            (i0[:, 2] + dz) % N]
    return out


def bc_shell(phi1, L, origin, dg, Ng, order=2):
    """phi1 interpolated to every padded PM cell outside the interior (C.3).

    ``origin`` is the box-local frame origin in full-box coordinates.  Returns
    an (Ng + 2 order)^3 array (order = FDA order: 2 N_ghost ghost layers per side),
    zero on the interior.  Multiply by D1(a_K) for Phi_BCs at a force evaluation
    (Eq. 23).
    """
    c = padded_cell_index(Ng, order).astype(np.float64)
    cx, cy, cz = np.meshgrid(c, c, c, indexing="ij")
    X = np.stack([origin[0] + (cx.ravel() + 0.5) * dg,
                  origin[1] + (cy.ravel() + 0.5) * dg,
                  origin[2] + (cz.ravel() + 0.5) * dg], axis=1)
    shell = trilinear_periodic(phi1, L, X).reshape((Ng + 2 * order,) * 3)
    shell[interior_mask(Ng, order)] = 0.0
    return shell
