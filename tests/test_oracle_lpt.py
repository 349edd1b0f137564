"""Pins of the oracle's 2LPT potentials and displacements (Sec. 2.1, A.2, C.2)."""
import numpy as np

import synth_inputs
from oracle import lpt


def _grid(N):
    x = np.arange(N)
    return np.meshgrid(x, x, x, indexing="ij")


def test_plane_wave_has_no_second_order_source():
    # A single plane wave: phi_,ii phi_,jj - phi_,ij^2 vanishes for every pair (Eq. 6).
    N, L = 16, 64.0
    X, Y, Z = _grid(N)
    delta = 0.3 * np.cos(2 * np.pi * (2 * X + Y + 3 * Z) / N)
    phi1, phi2, src = lpt.lpt_potentials(delta, L)
    assert np.abs(src).max() < 1e-14 * np.abs(phi1).max() ** 2 * (N / L) ** 4
    assert np.abs(phi2).max() < 1e-12 * np.abs(phi1).max()


def test_two_orthogonal_waves_closed_form():
    # delta = A cos(k1 x) + B cos(k2 y): phi1 = A cos/Lam1 + B cos/Lam2; the only
    # non-zero pair is phi_,xx phi_,yy; cos(k1 x) cos(k2 y) has Laplacian eigenvalue Lam1 + Lam2.
    N, L = 16, 50.0
    d = L / N
    X, Y, _ = _grid(N)
    A, B, m1, m2 = 0.7, -0.4, 2, 3
    k1, k2 = 2 * np.pi * m1 / L, 2 * np.pi * m2 / L
    lam1 = -(4 / d**2) * np.sin(k1 * d / 2) ** 2
    lam2 = -(4 / d**2) * np.sin(k2 * d / 2) ** 2
    c1, c2 = np.cos(k1 * X * d), np.cos(k2 * Y * d)
    delta = A * c1 + B * c2
    phi1, phi2, src = lpt.lpt_potentials(delta, L)
    np.testing.assert_allclose(phi1, A * c1 / lam1 + B * c2 / lam2, rtol=1e-12, atol=1e-13)
    s1, s2 = (np.sin(k1 * d) / d) ** 2, (np.sin(k2 * d) / d) ** 2
    src_exact = s1 * s2 * A * B / (lam1 * lam2) * c1 * c2
    np.testing.assert_allclose(src, src_exact, atol=1e-12 * np.abs(src_exact).max())
    np.testing.assert_allclose(phi2, src_exact / (lam1 + lam2), atol=1e-12 * np.abs(src_exact).max() / abs(lam1 + lam2))
    # Psi1 = central gradient of phi1: the x component is -A sin(k1 x) sin(k1 d)/d / lam1
    _, _, psi1, _ = lpt.lpt_fields(delta, L)
    np.testing.assert_allclose(psi1[0], -A * np.sin(k1 * X * d) * np.sin(k1 * d) / d / lam1,
                               atol=1e-12 * np.abs(phi1).max() / d)


def test_fourier_second_derivatives_equal_central_difference_twice():
    # phi_,ij in Fourier space (-D_i D_j) is the configuration-space central difference applied twice.
    N, L = 12, 30.0
    delta = synth_inputs.random_field((N, N, N), 3)
    delta -= delta.mean()
    phi1, _, src = lpt.lpt_potentials(delta, L)
    g = lpt.central_gradient(phi1, L)
    gg = [lpt.central_gradient(g[i], L) for i in range(3)]
    xx, yy, zz = gg[0][0], gg[1][1], gg[2][2]
    xy, xz, yz = gg[0][1], gg[0][2], gg[1][2]
    np.testing.assert_allclose(gg[0][1], gg[1][0], atol=1e-12)
    ref = xx * yy + xx * zz + yy * zz - xy**2 - xz**2 - yz**2
    np.testing.assert_allclose(src, ref, atol=1e-10 * np.abs(ref).max())


def test_laplacian_of_phi1_returns_delta():
    N, L = 12, 30.0
    d = L / N
    delta = synth_inputs.random_field((N, N, N), 4)
    delta -= delta.mean()
    phi1, _, _ = lpt.lpt_potentials(delta, L)
    lap = sum(np.roll(phi1, 1, ax) + np.roll(phi1, -1, ax) for ax in range(3)) - 6 * phi1
    np.testing.assert_allclose(lap / d**2, delta, atol=1e-11)
