"""Pins of the oracle's Dirichlet boundary shell (Sec. 3.3 C.3, Eq. 23)."""
import numpy as np

import synth_inputs
from oracle import boundary


def test_constant_potential_is_reproduced():
    N, L, Ng = 8, 40.0, 6
    phi = np.full((N, N, N), 2.5)
    sh = boundary.bc_shell(phi, L, np.array([-3.0, 1.0, 7.5]), 2.1, Ng)
    inside = boundary.interior_mask(Ng)
    assert np.all(sh[inside] == 0.0)
    np.testing.assert_allclose(sh[~inside], 2.5, rtol=1e-15)


def test_trilinear_equals_brute_force_tent_weights():
    # phi(X) = sum_i phi_i prod_axes max(0, 1 - |u - i|) with periodic images, u = X/d - 1/2.
    N, L = 6, 12.0
    d = L / N
    phi = synth_inputs.random_field((N, N, N), 11)
    X = synth_inputs.random_positions(20, -15.0, 30.0, 12)
    got = boundary.trilinear_periodic(phi, L, X)
    for m in range(len(X)):
        u = X[m] / d - 0.5
        ref = 0.0
        for i in range(-3 * N, 4 * N):
            wx = max(0.0, 1 - abs(u[0] - i))
            if wx == 0:
                continue
            for j in range(-3 * N, 4 * N):
                wy = max(0.0, 1 - abs(u[1] - j))
                if wy == 0:
                    continue
                for k in range(-3 * N, 4 * N):
                    wz = max(0.0, 1 - abs(u[2] - k))
                    if wz:
                        ref += wx * wy * wz * phi[i % N, j % N, k % N]
        assert abs(got[m] - ref) < 1e-12


def test_smooth_mode_within_trilinear_error_bound():
    # interpolating cos(k x) with nodes spacing d has error <= (k d)^2 / 8 per axis.
    N, L, Ng = 32, 100.0, 10
    d = L / N
    x = (np.arange(N) + 0.5) * d
    k = 2 * np.pi / L
    phi = np.cos(k * x)[:, None, None] * np.ones((1, N, N))
    origin = np.array([13.0, -4.0, 50.0])
    dg = 3.3
    sh = boundary.bc_shell(phi, L, origin, dg, Ng)
    c = np.arange(-2, Ng + 2)
    exact = np.cos(k * (origin[0] + (c + 0.5) * dg))[:, None, None] * np.ones((1, Ng + 4, Ng + 4))
    out = ~boundary.interior_mask(Ng)
    assert np.abs(sh[out] - exact[out]).max() <= (k * d) ** 2 / 8 + 1e-14
