"""Oracle pins for the FDA orders 4 and 6 (Sec. 3.1, App. C)."""
import numpy as np
import pytest

import synth_inputs
from oracle import fda, lpt, pm

ORDERS = (2, 4, 6)


@pytest.mark.parametrize("order", ORDERS)
def test_stencils_are_exact_on_polynomials(order):
    # A central stencil of order n reproduces the first derivative of every polynomial of
    # degree <= n and the second derivative of every polynomial of degree <= n + 1.
    x0, d = 0.37, 0.21
    g = fda.gradient_coefficients(order)
    s = fda.second_derivative_coefficients(order)
    for p in range(order + 2):
        f = lambda x: x**p
        d1 = sum(gm * (f(x0 + m * d) - f(x0 - m * d)) for m, gm in enumerate(g, start=1)) / d
        d2 = (s[0] * f(x0) + sum(sm * (f(x0 + m * d) + f(x0 - m * d)) for m, sm in enumerate(s) if m)) / d**2
        ex1 = p * x0 ** (p - 1) if p else 0.0
        ex2 = p * (p - 1) * x0 ** (p - 2) if p > 1 else 0.0
        if p <= order:
            assert abs(d1 - ex1) < 1e-10 * max(1.0, abs(ex1))
        if p <= order + 1:
            assert abs(d2 - ex2) < 1e-9 * max(1.0, abs(ex2))
    # and not beyond: the next odd power shows the truncation error of the gradient
    p = order + 1
    d1 = sum(gm * ((x0 + m * d) ** p - (x0 - m * d) ** p) for m, gm in enumerate(g, start=1)) / d
    assert abs(d1 - p * x0 ** (p - 1)) > 1e-8


@pytest.mark.parametrize("order", ORDERS)
def test_printed_dst_eigenvalues_equal_the_stencil_symbol(order):
    # App. C prints the eigenvalues as sums of sin^2; they must be the second-derivative
    # symbol of the stencil at k d = pi l / (N + 1).
    for N in (7, 24, 97):
        d = 0.9
        l = np.arange(1, N + 1)
        sym = fda.second_derivative_symbol(np.pi * l / ((N + 1) * d), d, order)
        np.testing.assert_allclose(fda.dst_eigenvalues(N, d, order), sym, rtol=1e-12, atol=1e-12 / d**2)


@pytest.mark.parametrize("order", ORDERS)
def test_second_derivative_symbol_matches_the_stencil_sum_and_vanishes_at_zero(order):
    # The cancellation-free form equals s_0 + 2 sum_m s_m cos(m k d) and is exactly 0 at k = 0.
    d = 0.8
    s = fda.second_derivative_coefficients(order)
    assert abs(s[0] + 2 * sum(s[1:])) < 1e-15
    k = np.linspace(0.0, np.pi / d, 17)
    direct = (s[0] + 2.0 * sum(sm * np.cos(m * k * d) for m, sm in enumerate(s) if m)) / d**2
    np.testing.assert_allclose(fda.second_derivative_symbol(k, d, order), direct, atol=1e-13 / d**2)
    assert fda.second_derivative_symbol(np.zeros(1), d, order)[0] == 0.0


@pytest.mark.parametrize("order", ORDERS)
def test_dst_basis_is_eigenvector_with_odd_continuation(order):
    # The DST-I basis vectors sin(pi l i/(N+1)) vanish at i = 0 and N + 1 and are odd across
    # both planes; the order-n stencil applied to that continuation returns lambda_l times
    # the vector (the relation the App. C solve relies on).
    N, d = 11, 1.3
    s = fda.second_derivative_coefficients(order)
    lam = fda.dst_eigenvalues(N, d, order)
    for l in (1, 4, 11):
        ext = np.sin(np.pi * l * np.arange(-N - 1, 2 * N + 3) / (N + 1))    # odd continuation
        off = N + 1
        v = ext[off + 1:off + N + 1]
        out = np.array([(s[0] * ext[off + i] + sum(s[m] * (ext[off + i + m] + ext[off + i - m])
                                                   for m in range(1, len(s)))) / d**2 for i in range(1, N + 1)])
        np.testing.assert_allclose(out, lam[l - 1] * v, atol=1e-11)


def _odd_operator_1d(N, d, order):
    """The order-n second difference on N points with odd continuation across both planes."""
    s = fda.second_derivative_coefficients(order)
    A = np.zeros((N, N))
    for i in range(N):                      # point i + 1 in 1-based DST indexing
        A[i, i] += s[0]
        for m in range(1, len(s)):
            for j, sign in ((i + 1 + m, 1.0), (i + 1 - m, 1.0)):
                if 1 <= j <= N:
                    A[i, j - 1] += sign * s[m]
                elif j < 0:                  # reflected across plane 0: value -v_{-j}
                    A[i, -j - 1] -= s[m]
                elif j > N + 1:              # reflected across plane N + 1
                    A[i, 2 * (N + 1) - j - 1] -= s[m]
    return A / d**2


@pytest.mark.parametrize("order", (4, 6))
def test_dirichlet_solve_equals_dense_solve_of_the_order_n_operator(order):
    N, d = 6, 0.7
    A1 = _odd_operator_1d(N, d, order)
    I = np.eye(N)
    A = np.kron(np.kron(A1, I), I) + np.kron(np.kron(I, A1), I) + np.kron(np.kron(I, I), A1)
    src = synth_inputs.random_field((N, N, N), 41)
    phi = pm.zero_bc_poisson(src, d, order)
    ref = np.linalg.solve(A, src.ravel()).reshape(N, N, N)
    np.testing.assert_allclose(phi, ref, atol=1e-11 * np.abs(ref).max())


@pytest.mark.parametrize("order", (4, 6))
def test_boundary_source_uses_every_ghost_layer_in_reach(order):
    # delta' - delta = -Lap Phi_BCs: with Phi_BCs = 1 in ghost layer m (counted outward from
    # the x- face) only, the cells at distance r < ... inside get -s_q / dg^2 with
    # q = m + r (the stencil offset reaching that layer), nothing else.
    Ng, dg = 8, 0.5
    P = order
    s = fda.second_derivative_coefficients(order)
    for m in range(1, order // 2 + 1):
        bc = np.zeros((Ng + 2 * P,) * 3)
        bc[P - m, P:P + Ng, P:P + Ng] = 1.0
        diff = pm.modified_density(np.zeros((Ng,) * 3), bc, dg, order)
        for r in range(Ng):
            q = m + r
            want = -s[q] / dg**2 if q < len(s) else 0.0
            np.testing.assert_allclose(diff[r], want, atol=1e-12)


@pytest.mark.parametrize("order", (4, 6))
def test_lpt_symbols_equal_configuration_space_stencils(order):
    # The Fourier-space Laplacian and gradient of order n equal the stencils applied in
    # configuration space on a periodic random field.
    N, L = 16, 40.0
    d = L / N
    f = synth_inputs.random_field((N, N, N), 43)
    s = fda.second_derivative_coefficients(order)
    lap_conf = 3 * s[0] * f + sum(s[m] * (np.roll(f, m, a) + np.roll(f, -m, a)) for m in range(1, len(s))
                                  for a in range(3))
    lap_conf = lap_conf / d**2
    lap_four = np.fft.irfftn(lpt.laplacian_symbol(N, L, order) * np.fft.rfftn(f), s=f.shape, axes=(0, 1, 2))
    np.testing.assert_allclose(lap_four, lap_conf, atol=1e-10 * np.abs(lap_conf).max())
    from oracle.ics import fourier_wavenumbers
    kx, _, _ = fourier_wavenumbers(N, L)
    gx_four = np.fft.irfftn(1j * fda.gradient_symbol(kx, d, order) * np.fft.rfftn(f), s=f.shape, axes=(0, 1, 2))
    np.testing.assert_allclose(lpt.central_gradient(f, L, order)[0], gx_four, atol=1e-10 * np.abs(gx_four).max())


@pytest.mark.parametrize("order", (4, 6))
def test_uniform_lattice_feels_no_force(order):
    # P6 at orders 4 and 6: a lattice at 1:1 and 2:1 with zero boundary potential.
    for ratio in (1, 2):
        Nsc, dq = 8, 1.0
        Ng = ratio * Nsc
        dg = Nsc * dq / Ng
        q = (np.stack(np.meshgrid(*(np.arange(Nsc),) * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) * dq
        r = pm.box_force(q, dg, Ng, Nsc, np.zeros((Ng + 2 * order,) * 3), order=order)
        assert np.abs(r["delta"]).max() < 1e-12
        assert np.abs(r["F"]).max() < 1e-12


def test_order_4_gradient_is_exact_on_a_cubic_potential_where_order_2_is_not():
    Ng, dg = 10, 0.4
    for order, exact in ((2, False), (4, True), (6, True)):
        P = order
        c = (np.arange(-P, Ng + P) + 0.5) * dg
        X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
        phi = X**3 - 2 * Y**2 * Z + Z
        pts = synth_inputs.random_positions(50, 1.0 * dg, (Ng - 1) * dg, 44)
        F, _ = pm.interpolate_gradient(phi, pts, dg, order)
        # CIC interpolation of the exact corner gradients
        u = pts / dg - 0.5
        i0 = np.floor(u).astype(int)
        f = u - i0
        Fref = np.zeros_like(F)
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1])
                         * (f[:, 2] if dz else 1 - f[:, 2]))
                    x, y, z = ((i0 + np.array([dx, dy, dz])) + 0.5).T * dg
                    Fref += w[:, None] * np.stack([3 * x**2, -4 * y * z, 1 - 2 * y**2], 1)
        err = np.abs(F - Fref).max()
        assert (err < 1e-10) == exact, (order, err)
