"""Lagrangian potentials and 2LPT displacements (Sec. 2.1, Sec. 3.1 A.2, Sec. 3.3 C.2).

Test infrastructure (see ``oracle/__init__``).

All operators are FDA at order 2 on the periodic N^3 LPT grid (the paper's runs
use order 2, Sec. 4), spacing d = L/N, nodes at the particle sites:
  * Laplacian symbol      Lambda(k) = -(4/d^2) sum_i sin^2(k_i d / 2)
  * central difference    d_i  <->  i sin(k_i d)/d
  * second derivatives    phi_,ij = d_i d_j phi  (central difference applied
    twice, for i = j too), which is what "nine one-dimensional gradient
    operations" in configuration space computes (Sec. 3.1); the Fourier and
    configuration-space routes are then the same operator.
Potentials (Eqs. 5-6):
    Lap phi1 = delta_i,
    Lap phi2 = sum_{i>j} [phi1_,ii phi1_,jj - (phi1_,ij)^2],
with the k = 0 mode of both set to zero.  Displacement vectors (App. A, below
Eq. 39): Psi1 = grad phi1, Psi2 = grad phi2, with the central difference at the
grid nodes; the LPT trajectory is x_LPT = q - D1 Psi1 + D2 Psi2 (Eq. 39).

Pins (tests/test_oracle_lpt.py): a single plane wave has a vanishing
second-order source; two orthogonal plane waves give the closed-form source and
phi2; the Fourier-space second derivatives equal central differences applied
twice in configuration space; the Laplacian of phi1 returns delta exactly.
"""
import numpy as np

from . import fda
from .ics import fourier_wavenumbers


def laplacian_symbol(N, L, order=2):
    """Laplacian eigenvalues on the rfftn grid (FDA-2: -(4/d^2) sum sin^2(k d/2); order
    4 and 6: the sum of the order-n second-derivative symbols, ``fda``)."""
    d = L / N
    kx, ky, kz = fourier_wavenumbers(N, L)
    if order != 2:
        return sum(fda.second_derivative_symbol(k, d, order) for k in (kx, ky, kz))
    return -(4.0 / d**2) * (np.sin(kx * d / 2) ** 2 + np.sin(ky * d / 2) ** 2
                            + np.sin(kz * d / 2) ** 2)


def _inverse_laplacian(field_k, lam):
    """field / Lambda with the k = 0 mode set to zero (Eqs. 5-6)."""
    out = np.zeros_like(field_k)
    nz = lam != 0
    nz[0, 0, 0] = False
    out[nz] = field_k[nz] / lam[nz]
    return out


def lpt_potentials(delta, L, order=2):
    """phi1, phi2 and the second-order source on the LPT grid (Eqs. 5-6)."""
    delta = np.asarray(delta, dtype=np.float64)
    N = delta.shape[0]
    d = L / N
    lam = laplacian_symbol(N, L, order)
    phi1_k = _inverse_laplacian(np.fft.rfftn(delta), lam)
    phi1 = np.fft.irfftn(phi1_k, s=delta.shape, axes=(0, 1, 2))
    kx, ky, kz = fourier_wavenumbers(N, L)
    if order == 2:
        D = [np.sin(kx * d) / d, np.sin(ky * d) / d, np.sin(kz * d) / d]
    else:
        D = [fda.gradient_symbol(k, d, order) for k in (kx, ky, kz)]

    def second(i, j):
        return np.fft.irfftn(-D[i] * D[j] * phi1_k, s=delta.shape, axes=(0, 1, 2))

    xx, yy, zz = second(0, 0), second(1, 1), second(2, 2)
    xy, xz, yz = second(0, 1), second(0, 2), second(1, 2)
    source = xx * yy + xx * zz + yy * zz - xy**2 - xz**2 - yz**2
    phi2 = np.fft.irfftn(_inverse_laplacian(np.fft.rfftn(source), lam), s=delta.shape, axes=(0, 1, 2))
    return phi1, phi2, source


def central_gradient(phi, L, order=2):
    """Periodic central gradient at the grid nodes (FDA-2: (phi[i+1] - phi[i-1]) / (2d);
    order 4, 6: the ``fda`` stencils).

    Returns an array of shape (3, N, N, N).
    """
    N = phi.shape[0]
    d = L / N
    if order == 2:
        return np.stack([(np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)) / (2.0 * d)
                         for ax in range(3)])
    g = fda.gradient_coefficients(order)
    return np.stack([sum(gm * (np.roll(phi, -m, axis=ax) - np.roll(phi, m, axis=ax)) for m, gm in
                         enumerate(g, start=1)) / d for ax in range(3)])


def lpt_fields(delta, L, order=2):
    """phi1, phi2, Psi1 = grad phi1, Psi2 = grad phi2 on the LPT grid."""
    phi1, phi2, _ = lpt_potentials(delta, L, order)
    return phi1, phi2, central_gradient(phi1, L, order), central_gradient(phi2, L, order)
