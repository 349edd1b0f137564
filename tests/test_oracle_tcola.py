"""Pins of the oracle's periodic tCOLA pieces (Sec. 2.2): the full-box deposit, Poisson solve
and force interpolation that the study modes of Sec. 4.3 take their true fields from."""
import numpy as np

import synth_inputs
from oracle import tcola


def _periodic_laplacian_1d(N, d):
    A = -2.0 * np.eye(N)
    for i in range(N):
        A[i, (i + 1) % N] += 1.0
        A[i, (i - 1) % N] += 1.0
    return A / d**2


def test_periodic_potential_equals_a_dense_solve_of_the_7_point_laplacian():
    # FDA-2 periodic Laplacian on a 6^3 grid as a dense matrix; its null space is the
    # constant, so the zero-mean least-squares solution is the potential of the source.
    N, L = 6, 9.0
    d = L / N
    A1 = _periodic_laplacian_1d(N, d)
    I = np.eye(N)
    A = np.kron(np.kron(A1, I), I) + np.kron(np.kron(I, A1), I) + np.kron(np.kron(I, I), A1)
    src = synth_inputs.random_field((N, N, N), 61)
    src -= src.mean()
    ref, *_ = np.linalg.lstsq(A, src.ravel(), rcond=None)
    ref -= ref.mean()
    phi = tcola.periodic_potential(src, L)
    np.testing.assert_allclose(phi.ravel(), ref, atol=1e-10 * np.abs(ref).max())
    assert abs(phi.mean()) < 1e-12 * np.abs(phi).max()


def test_periodic_deposit_conserves_mass_and_matches_brute_force():
    Np, Ng, L = 4, 8, 10.0
    rng = np.random.default_rng(62)
    x = rng.uniform(0.0, L, size=(Np**3, 3))
    x[0] = [L - 1e-3, 0.2, L - 0.3]            # stencils that wrap across the faces
    x[1] = [0.05, L - 0.01, 0.05]
    delta = tcola.periodic_deposit(x, L, Ng, Np)
    nbar = Np**3 / Ng**3
    assert abs(((delta + 1.0) * nbar).sum() - Np**3) < 1e-9
    dg = L / Ng
    rho = np.zeros((Ng, Ng, Ng))
    for p in x:
        u = p / dg - 0.5
        i0 = np.floor(u).astype(int)
        f = u - i0
        for c in np.ndindex(2, 2, 2):
            w = np.prod([f[a] if c[a] else 1.0 - f[a] for a in range(3)])
            rho[tuple((i0[a] + c[a]) % Ng for a in range(3))] += w
    np.testing.assert_allclose(delta, rho / nbar - 1.0, atol=1e-12)


def test_periodic_force_of_a_single_mode():
    # Phi = cos(2 pi (m . x) / L) at the cell centres: the FDA-2 central gradient along axis a
    # is -sin(2 pi (m . x)/L) sin(2 pi m_a dg / L) / dg exactly; a particle at a cell centre
    # receives that value, and elsewhere the trilinear blend of the eight corner values.
    Ng, L = 12, 30.0
    dg = L / Ng
    m = np.array([1, -2, 3])
    c = (np.arange(Ng) + 0.5) * dg
    X = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1)
    ph = 2 * np.pi * (X @ m) / L
    phi = np.cos(ph)
    g_nodes = np.stack([-np.sin(ph) * np.sin(2 * np.pi * m[a] * dg / L) / dg for a in range(3)])
    nodes = np.array([[0.5, 0.5, 0.5], [3.5, 7.5, 11.5], [11.5, 0.5, 6.5]]) * dg
    F = tcola.periodic_interpolate_gradient(phi, nodes, L)
    for k, q in enumerate(np.round(nodes / dg - 0.5).astype(int)):
        np.testing.assert_allclose(F[k], g_nodes[:, q[0], q[1], q[2]], atol=1e-12)
    pts = synth_inputs.random_positions(20, 0.0, L, 63)
    F = tcola.periodic_interpolate_gradient(phi, pts, L)
    for k, p in enumerate(pts):
        u = p / dg - 0.5
        i0 = np.floor(u).astype(int)
        f = u - i0
        want = np.zeros(3)
        for cc in np.ndindex(2, 2, 2):
            w = np.prod([f[a] if cc[a] else 1.0 - f[a] for a in range(3)])
            idx = tuple((i0[a] + cc[a]) % Ng for a in range(3))
            want += w * g_nodes[(slice(None),) + idx]
        np.testing.assert_allclose(F[k], want, atol=1e-12)
