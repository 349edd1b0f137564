"""Pins of the oracle's box PM force: deposit, Dirichlet DST-I solve, gradient, interpolation
(Sec. 3.4, App. C)."""
import numpy as np
import pytest
from scipy import fft as sfft

import synth_inputs
from oracle import lpt, pm, tiling


@pytest.mark.parametrize("N", [1, 5, 24, 97])
def test_dst1_matrix_matches_library_dst(N):
    # scipy's DST-I is y_l = 2 sum_i x_i sin(pi (l+1)(i+1)/(N+1)) (Eq. 63 up to the factor 2).
    x = synth_inputs.random_field((N,), N)
    np.testing.assert_allclose(pm.dst1_matrix(N) @ x, sfft.dst(x, type=1) / 2, atol=1e-12 * max(1, N))


@pytest.mark.parametrize("N", [4, 24, 96])
def test_dst1_orthogonality(N):
    # (2/(N+1)) S S = I (Eq. 65): the inverse 3D transform is DST-I times 8/(N+1)^3 (Eq. 66).
    S = pm.dst1_matrix(N)
    np.testing.assert_allclose(S @ S, (N + 1) / 2 * np.eye(N), atol=1e-11 * N)
    f = synth_inputs.random_field((N % 13 + 3,) * 3, 5)
    n = f.shape[0]
    np.testing.assert_allclose(pm.dst1_3d(pm.dst1_3d(f)) * 8 / (n + 1) ** 3, f, atol=1e-12)


@pytest.mark.parametrize("N", [3, 10, 33])
def test_eigenvalues_of_second_difference(N):
    # the FDA-2 second difference with zero ends maps basis column l to lambda_l times it (Eq. 68).
    dg = 0.7
    S = pm.dst1_matrix(N)
    lam = pm.dirichlet_eigenvalues(N, dg)
    T = (np.diag(-2.0 * np.ones(N)) + np.diag(np.ones(N - 1), 1) + np.diag(np.ones(N - 1), -1)) / dg**2
    np.testing.assert_allclose(T @ S, S * lam[None, :], atol=1e-11 / dg**2)


def _dense_dirichlet_solve(delta, bc_pad, dg):
    """Assemble the 7-point Laplacian on the interior with Dirichlet ghosts and solve densely."""
    Ng = delta.shape[0]
    n = Ng**3
    A = np.zeros((n, n))
    b = delta.ravel().copy()
    idx = lambda i, j, k: (i * Ng + j) * Ng + k
    for i in range(Ng):
        for j in range(Ng):
            for k in range(Ng):
                r = idx(i, j, k)
                A[r, r] = -6.0 / dg**2
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < Ng and 0 <= jj < Ng and 0 <= kk < Ng:
                        A[r, idx(ii, jj, kk)] = 1.0 / dg**2
                    else:
                        b[r] -= bc_pad[ii + 2, jj + 2, kk + 2] / dg**2
    return np.linalg.solve(A, b).reshape(Ng, Ng, Ng)


@pytest.mark.parametrize("Ng", [1, 4, 7])
def test_dirichlet_solve_matches_dense_linear_solve(Ng):
    dg = 1.3
    delta = synth_inputs.random_field((Ng,) * 3, 20 + Ng)
    bc = synth_inputs.random_field((Ng + 4,) * 3, 40 + Ng)
    c = np.arange(-2, Ng + 2)
    m = (c >= 0) & (c < Ng)
    bc[m[:, None, None] & m[None, :, None] & m[None, None, :]] = 0.0
    phi = pm.dirichlet_potential(delta, bc, dg)
    ref = _dense_dirichlet_solve(delta, bc, dg)
    np.testing.assert_allclose(phi[2:Ng + 2, 2:Ng + 2, 2:Ng + 2], ref, atol=1e-11 * np.abs(ref).max())
    out = ~(m[:, None, None] & m[None, :, None] & m[None, None, :])
    assert np.all(phi[out] == bc[out])


def test_restriction_of_periodic_solution():
    # The periodic FDA-2 solution, restricted to a sub-box with its own ghost values as
    # Phi_BCs, is the unique Dirichlet solution there (basis of the Sec. 4.3 consistency test).
    N, L = 16, 32.0
    d = L / N
    delta = synth_inputs.random_field((N, N, N), 7)
    delta -= delta.mean()
    lam = lpt.laplacian_symbol(N, L)
    dk = np.fft.rfftn(delta)
    dk[lam != 0] /= lam[lam != 0]
    dk[lam == 0] = 0
    phi_per = np.fft.irfftn(dk, s=delta.shape, axes=(0, 1, 2))
    Ng, start = 6, np.array([13, 2, 5])
    idx = [(start[a] + np.arange(-2, Ng + 2)) % N for a in range(3)]
    padded = phi_per[np.ix_(*idx)]
    bc = padded.copy()
    bc[2:Ng + 2, 2:Ng + 2, 2:Ng + 2] = 0.0
    delta_box = delta[np.ix_(*[i[2:Ng + 2] for i in idx])]
    phi = pm.dirichlet_potential(delta_box, bc, d)
    np.testing.assert_allclose(phi, padded, atol=1e-12 * np.abs(padded).max())


def test_cic_mass_conservation_with_drop():
    Ng, Nsc, dg = 6, 6, 1.0
    xloc = synth_inputs.random_positions(300, -1.5, 7.5, 8)
    delta, deposited = pm.cic_deposit_box(xloc, dg, Ng, Nsc)
    nbar = (Nsc / Ng) ** 3
    assert abs((delta + 1).sum() * nbar - deposited) < 1e-10
    # independent: the kept fraction of a particle is the product of its per-axis kept 1D weights
    u = xloc / dg - 0.5
    i0 = np.floor(u)
    f = u - i0
    keep = np.ones(len(u))
    for ax in range(3):
        lo_in = (i0[:, ax] >= 0) & (i0[:, ax] < Ng)
        hi_in = (i0[:, ax] + 1 >= 0) & (i0[:, ax] + 1 < Ng)
        keep *= np.where(lo_in, 1 - f[:, ax], 0) + np.where(hi_in, f[:, ax], 0)
    assert abs(keep.sum() - deposited) < 1e-10
    assert deposited < 300


def test_cic_deposit_brute_force():
    Ng, Nsc, dg = 5, 4, 1.7
    xloc = synth_inputs.random_positions(40, -2.0, Ng * dg + 2.0, 9)
    delta, _ = pm.cic_deposit_box(xloc, dg, Ng, Nsc)
    u = xloc / dg - 0.5
    ref = np.zeros((Ng,) * 3)
    for i in range(Ng):
        for j in range(Ng):
            for k in range(Ng):
                w = (np.maximum(0, 1 - np.abs(u[:, 0] - i)) * np.maximum(0, 1 - np.abs(u[:, 1] - j))
                     * np.maximum(0, 1 - np.abs(u[:, 2] - k)))
                ref[i, j, k] = w.sum()
    np.testing.assert_allclose(delta, ref / (Nsc / Ng) ** 3 - 1, atol=1e-12)


@pytest.mark.parametrize("ratio", [1, 2])
def test_uniform_lattice_feels_no_force(ratio):
    Nsc, L_sc = 8, 16.0
    dq = L_sc / Nsc
    Ng = ratio * Nsc
    dg = L_sc / Ng
    q = (tiling.box_local_lattice(Nsc) + 0.5) * dq
    delta, deposited = pm.cic_deposit_box(q, dg, Ng, Nsc)
    assert np.abs(delta).max() < 1e-13 and abs(deposited - Nsc**3) < 1e-9
    r = pm.box_force(q, dg, Ng, Nsc, np.zeros((Ng + 4,) * 3))
    assert np.abs(r["F"]).max() < 1e-13


def test_gradient_of_linear_and_quadratic_potentials_is_exact():
    Ng, dg = 7, 0.9
    c = (np.arange(-2, Ng + 2) + 0.5) * dg
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    x = synth_inputs.random_positions(200, -0.5 * dg, (Ng + 0.5) * dg, 3)   # u in [-1, Ng]
    F, clamped = pm.interpolate_gradient(0.3 * X - 1.1 * Y + 2.0 * Z, x, dg)
    assert not clamped.any()
    np.testing.assert_allclose(F, np.tile([0.3, -1.1, 2.0], (200, 1)), atol=1e-12)
    # central differences are exact on quadratics, and trilinear interpolation is exact on
    # the resulting linear gradient:  grad (x^2 + 2 y z) = (2x, 2z, 2y)
    F, _ = pm.interpolate_gradient(X**2 + 2 * Y * Z, x, dg)
    np.testing.assert_allclose(F, np.stack([2 * x[:, 0], 2 * x[:, 2], 2 * x[:, 1]], 1), atol=1e-11)


def test_deposit_interpolation_adjointness():
    # sum_p F_x(p) = sum_c rho_c G_x(c) for particles whose CIC corners are all interior.
    Ng, Nsc, dg = 6, 6, 1.0
    x = synth_inputs.random_positions(100, 0.5 * dg + 1e-9, (Ng - 0.5) * dg - 1e-9, 4)
    phi = synth_inputs.random_field((Ng + 4,) * 3, 6)
    F, _ = pm.interpolate_gradient(phi, x, dg)
    delta, _ = pm.cic_deposit_box(x, dg, Ng, Nsc)
    rho = (delta + 1) * (Nsc / Ng) ** 3
    Gx = (phi[3:Ng + 3, 2:Ng + 2, 2:Ng + 2] - phi[1:Ng + 1, 2:Ng + 2, 2:Ng + 2]) / (2 * dg)
    assert abs(F[:, 0].sum() - (rho * Gx).sum()) < 1e-10


def test_clamped_particles_use_edge_position():
    Ng, dg = 5, 1.0
    phi = synth_inputs.random_field((Ng + 4,) * 3, 2)
    far = np.array([[-7.0, 2.2, 3.1], [2.0, 40.0, 1.0]])
    edge = np.array([[-0.5, 2.2, 3.1], [2.0, (Ng + 0.5) * dg, 1.0]])
    F1, cl = pm.interpolate_gradient(phi, far, dg)
    F2, _ = pm.interpolate_gradient(phi, edge, dg)
    assert cl.all()
    np.testing.assert_allclose(F1, F2, atol=1e-14)
