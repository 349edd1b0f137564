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

FDA order 4 and 6 (Sec. 3.1, App. C; ``order`` argument, default 2): the padding is
2 N_ghost = order cells per side, Phi_BCs fills the N_ghost layers next to the
interior, the source correction of Eq. 62 uses the order-n Laplacian (it reaches
N_ghost cells inside), the eigenvalues are App. C's order-n ones (``fda``), and the
gradient at the CIC corners is the order-n central difference.  Particles are clamped
to [-N_ghost, Ng + N_ghost - 1] (the accelerations exist on the grid padded by N_ghost,
Sec. 3.4.2) with i0 capped at Ng + N_ghost - 2.  The DST-I treats the potential as odd
across each Dirichlet plane; for order > 2 the stencil reaches past the first ghost
layer, where the paper's solve (App. C) thus sees the odd continuation of Phi~.

Pins (tests/test_oracle_pm.py): the DST-I matrix against scipy's DST-I and the
orthogonality S S = (Ng + 1)/2 I; the eigenvalues against the stencil; the
Dirichlet solve against a dense 7-point-Laplacian linear solve with the
boundary terms; the restriction of a periodic solution; mass conservation and a
brute-force tent-weight deposit; zero force on a uniform lattice; exact
gradients of linear and quadratic potentials; deposit/interpolation adjointness.
"""
import numpy as np

from . import fda


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


def laplacian_on_interior(padded, dg, order=2):
    """Order-n FDA Laplacian of a padded (Ng + 2 order)^3 field evaluated on its Ng^3 interior."""
    P = order
    Ng = padded.shape[0] - 2 * P
    s = fda.second_derivative_coefficients(order)
    inner = slice(P, Ng + P)
    lap = 3.0 * s[0] * padded[inner, inner, inner]
    for m in range(1, len(s)):
        lo, hi = slice(P - m, Ng + P - m), slice(P + m, Ng + P + m)
        lap = lap + s[m] * (padded[hi, inner, inner] + padded[lo, inner, inner])
        lap = lap + s[m] * (padded[inner, hi, inner] + padded[inner, lo, inner])
        lap = lap + s[m] * (padded[inner, inner, hi] + padded[inner, inner, lo])
    return lap / dg**2


def modified_density(delta, phi_bc_padded, dg, order=2):
    """delta' = delta - Lap Phi_BCs on the interior (App. C, Eq. 62).

    ``phi_bc_padded`` is Phi_BCs on the padded grid, zero on the interior, so
    only ghost neighbours of the boundary cells contribute.
    """
    return delta - laplacian_on_interior(phi_bc_padded, dg, order)


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


def zero_bc_poisson(source, dg, order=2):
    """Solve Lap Phi~ = source with Phi~ = 0 on the Dirichlet planes (App. C.2, Eqs. 63-71)."""
    N = source.shape[0]
    lam = dirichlet_eigenvalues(N, dg) if order == 2 else fda.dst_eigenvalues(N, dg, order)
    hat = dst1_3d(source)
    hat = hat / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :])
    return dst1_3d(hat) * (8.0 / (N + 1) ** 3)


def pad_potential(phi_interior, phi_bc_padded):
    """Phi on the padded grid: the solve inside, Phi_BCs in the ghost layers (Sec. 3.4.2)."""
    Ng = phi_interior.shape[0]
    P = (phi_bc_padded.shape[0] - Ng) // 2
    out = np.array(phi_bc_padded, dtype=np.float64, copy=True)
    out[P:Ng + P, P:Ng + P, P:Ng + P] = phi_interior
    return out


def dirichlet_potential(delta, phi_bc_padded, dg, order=2):
    """Padded Phi^sCOLA from the interior density and Phi_BCs (App. C.1-C.2)."""
    src = modified_density(delta, phi_bc_padded, dg, order)
    return pad_potential(zero_bc_poisson(src, dg, order), phi_bc_padded)


def interpolate_gradient(phi_padded, xloc, dg, order=2):
    """grad Phi at the particles: central gradient (FDA order n) at the CIC corners,
    CIC-interpolated.

    Returns (F, clamped) with F of shape (P, 3) and ``clamped`` a boolean mask
    of particles whose mesh coordinate was moved back into [-N_ghost, Ng + N_ghost - 1].
    """
    pad = order
    ng = fda.n_ghost(order)
    Ng = phi_padded.shape[0] - 2 * pad
    u_raw = mesh_coordinate(xloc, dg)
    u = np.clip(u_raw, -float(ng), float(Ng + ng - 1))
    clamped = np.any(u != u_raw, axis=1)
    i0 = np.minimum(np.floor(u).astype(np.int64), Ng + ng - 2)
    f = u - i0
    F = np.zeros_like(u)
    P = phi_padded
    g = fda.gradient_coefficients(order)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                cx = i0[:, 0] + dx + pad
                cy = i0[:, 1] + dy + pad
                cz = i0[:, 2] + dz + pad
                for m, gm in enumerate(g, start=1):
                    F[:, 0] += w * gm * (P[cx + m, cy, cz] - P[cx - m, cy, cz]) / dg
                    F[:, 1] += w * gm * (P[cx, cy + m, cz] - P[cx, cy - m, cz]) / dg
                    F[:, 2] += w * gm * (P[cx, cy, cz + m] - P[cx, cy, cz - m]) / dg
    return F, clamped


def box_force(xloc, dg, Ng, Nsc, phi_bc_padded, delta_override=None, order=2):
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
    phi = dirichlet_potential(delta, phi_bc_padded, dg, order)
    F, clamped = interpolate_gradient(phi, xloc, dg, order)
    return {"F": F, "delta": delta, "phi": phi, "deposited": deposited, "clamped": clamped}
