"""Particle-mesh force in one sCOLA box (Sec. 2.2, Sec. 3.4, App. C).

Test infrastructure (see ``oracle/__init__``).

Mesh conventions (readings of the paper, which leaves them open): box-local
coordinate x_loc in [0, L_sCOLA); PM cells of size dg = L_sCOLA / Ng with
centres at (c + 1/2) dg; the mesh coordinate of a particle is u = x_loc/dg - 1/2,
so cell c sits at u = c.  CIC weights use i0 = floor(u), f = u - i0.

D.1 density assignment B^sCOLA (Sec. 3.4.1): CIC of the box particles onto the
Ng^3 interior cells, discarding the weight that would land on cells outside.
The mean is the cosmic one, nbar = (Np,sCOLA / Ng)^3 particles per cell, so
delta = n / nbar - 1 in every interior cell.

D.2 Poisson solve (Sec. 3.4.2 and App. C): with Phi_BCs non-zero only outside
the interior, delta' = delta - Lap Phi_BCs (Eq. 62); the zero-boundary problem
Lap Phi~ = delta' is solved with the DST-I (Eqs. 63-67): forward transform,
division by lambda_l + lambda_m + lambda_n with the FDA-2 eigenvalues
lambda_l = -(4/dg^2) sin^2(pi l / (2 (Ng + 1)))  (Eq. 68 with
k_l dx/4 * Nx/(Nx+1) = pi l / (2 (Nx + 1)), Eq. 71), and the inverse transform
= DST-I times 8 / (Ng + 1)^3.  The transform here is the dense definition,
three tensor contractions with S_li = sin(pi l i / (Ng + 1)); no fast algorithm.
The solution is padded with Phi_BCs in the 2 ghost layers on every side.

Accelerations (Sec. 3.4.2): FDA-2 central gradient of the padded potential at
the 8 CIC corners of each particle, interpolated with the CIC weights.  The
padded potential supports gradients on cells [-1, Ng]; a particle whose mesh
coordinate leaves [-1, Ng] is clamped to that range (a reading: the paper is
silent) and its corner index i0 is capped at Ng - 1 so that both corners stay in
[-1, Ng].

Pins (tests/test_oracle_pm.py): the DST-I matrix against scipy's DST-I and the
orthogonality S S = (Ng + 1)/2 I; the eigenvalues against the stencil; the
Dirichlet solve against a dense 7-point-Laplacian linear solve with the
boundary terms; the restriction of a periodic solution; mass conservation and a
brute-force tent-weight deposit; zero force on a uniform lattice; exact
gradients of linear and quadratic potentials; deposit/interpolation adjointness.
"""
import numpy as np


def mesh_coordinate(xloc, dg):
    """u = x_loc / dg - 1/2: cell c centred at u = c."""
    return np.asarray(xloc, dtype=np.float64) / dg - 0.5


def cic_deposit_box(xloc, dg, Ng, Nsc):
    """B^sCOLA (Sec. 3.4.1).  Returns (delta, deposited_count).

    ``deposited_count`` is the total CIC weight that landed inside; the rest
    (Nsc^3 - deposited) was discarded at the box boundary.
    """
    u = mesh_coordinate(xloc, dg)
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    rho = np.zeros(Ng**3)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                cell = i0 + np.array([dx, dy, dz])
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                inside = np.all((cell >= 0) & (cell < Ng), axis=1)
                flat = (cell[inside, 0] * Ng + cell[inside, 1]) * Ng + cell[inside, 2]
                rho += np.bincount(flat, weights=w[inside], minlength=Ng**3)
    rho = rho.reshape(Ng, Ng, Ng)
    nbar = (Nsc / Ng) ** 3
    return rho / nbar - 1.0, float(rho.sum())


def laplacian_on_interior(padded, dg):
    """FDA-2 Laplacian of a padded (Ng + 4)^3 field evaluated on its Ng^3 interior."""
    Ng = padded.shape[0] - 4
    c = padded[2:Ng + 2, 2:Ng + 2, 2:Ng + 2]
    lap = -6.0 * c
    lap = lap + padded[3:Ng + 3, 2:Ng + 2, 2:Ng + 2] + padded[1:Ng + 1, 2:Ng + 2, 2:Ng + 2]
    lap = lap + padded[2:Ng + 2, 3:Ng + 3, 2:Ng + 2] + padded[2:Ng + 2, 1:Ng + 1, 2:Ng + 2]
    lap = lap + padded[2:Ng + 2, 2:Ng + 2, 3:Ng + 3] + padded[2:Ng + 2, 2:Ng + 2, 1:Ng + 1]
    return lap / dg**2


def modified_density(delta, phi_bc_padded, dg):
    """delta' = delta - Lap Phi_BCs on the interior (App. C, Eq. 62).

    ``phi_bc_padded`` is Phi_BCs on the padded grid, zero on the interior, so
    only ghost neighbours of the boundary cells contribute.
    """
    return delta - laplacian_on_interior(phi_bc_padded, dg)


def dst1_matrix(N):
    """S[l-1, i-1] = sin(pi l i / (N + 1)), l, i = 1..N (Eq. 64)."""
    idx = np.arange(1, N + 1, dtype=np.float64)
    return np.sin(np.pi * np.outer(idx, idx) / (N + 1))


def dst1_3d(field):
    """Three-dimensional DST-I, the dense definition of Eq. 63."""
    S = dst1_matrix(field.shape[0])
    out = np.tensordot(S, field, axes=([1], [0]))                          # x
    out = np.tensordot(S, out, axes=([1], [1])).transpose(1, 0, 2)          # y
    out = np.tensordot(out, S, axes=([2], [1]))                             # z
    return out


def dirichlet_eigenvalues(N, dg):
    """FDA-2 eigenvalues lambda_l, l = 1..N, of the 1D second difference with zero ends (Eq. 68)."""
    l = np.arange(1, N + 1, dtype=np.float64)
    return -(4.0 / dg**2) * np.sin(np.pi * l / (2.0 * (N + 1))) ** 2


def zero_bc_poisson(source, dg):
    """Solve Lap Phi~ = source with Phi~ = 0 on the Dirichlet planes (App. C.2, Eqs. 63-71)."""
    N = source.shape[0]
    lam = dirichlet_eigenvalues(N, dg)
    hat = dst1_3d(source)
    hat = hat / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :])
    return dst1_3d(hat) * (8.0 / (N + 1) ** 3)


def pad_potential(phi_interior, phi_bc_padded):
    """Phi on the padded grid: the solve inside, Phi_BCs in the ghost layers (Sec. 3.4.2)."""
    Ng = phi_interior.shape[0]
    out = np.array(phi_bc_padded, dtype=np.float64, copy=True)
    out[2:Ng + 2, 2:Ng + 2, 2:Ng + 2] = phi_interior
    return out


def dirichlet_potential(delta, phi_bc_padded, dg):
    """Padded Phi^sCOLA from the interior density and Phi_BCs (App. C.1-C.2)."""
    src = modified_density(delta, phi_bc_padded, dg)
    return pad_potential(zero_bc_poisson(src, dg), phi_bc_padded)


def interpolate_gradient(phi_padded, xloc, dg):
    """grad Phi at the particles: FDA-2 central gradient at the CIC corners, CIC-interpolated.

    Returns (F, clamped) with F of shape (P, 3) and ``clamped`` a boolean mask
    of particles whose mesh coordinate was moved back into [-1, Ng].
    """
    Ng = phi_padded.shape[0] - 4
    u_raw = mesh_coordinate(xloc, dg)
    u = np.clip(u_raw, -1.0, float(Ng))
    clamped = np.any(u != u_raw, axis=1)
    i0 = np.minimum(np.floor(u).astype(np.int64), Ng - 1)
    f = u - i0
    F = np.zeros_like(u)
    P = phi_padded
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                cx = i0[:, 0] + dx + 2
                cy = i0[:, 1] + dy + 2
                cz = i0[:, 2] + dz + 2
                F[:, 0] += w * (P[cx + 1, cy, cz] - P[cx - 1, cy, cz]) / (2.0 * dg)
                F[:, 1] += w * (P[cx, cy + 1, cz] - P[cx, cy - 1, cz]) / (2.0 * dg)
                F[:, 2] += w * (P[cx, cy, cz + 1] - P[cx, cy, cz - 1]) / (2.0 * dg)
    return F, clamped


def box_force(xloc, dg, Ng, Nsc, phi_bc_padded, delta_override=None):
    """One PM force evaluation in a box: deposit, Dirichlet solve, gradient, interpolation.

    ``phi_bc_padded`` is Phi_BCs at this force time (already scaled by D1).
    ``delta_override`` replaces B^sCOLA by a given interior density (used only
    by the consistency pin of Sec. 4.3, which feeds the true density).
    Returns a dict with F, delta, phi (padded), deposited and clamped.
    """
    if delta_override is None:
        delta, deposited = cic_deposit_box(xloc, dg, Ng, Nsc)
    else:
        delta, deposited = delta_override, float("nan")
    phi = dirichlet_potential(delta, phi_bc_padded, dg)
    F, clamped = interpolate_gradient(phi, xloc, dg)
    return {"F": F, "delta": delta, "phi": phi, "deposited": deposited, "clamped": clamped}
