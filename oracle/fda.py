"""Finite-difference approximations (FDA) at order 2, 4 and 6 (Sec. 3.1, App. C).

Test infrastructure (see ``oracle/__init__``).

The paper takes the gradient and Laplacian stencils at order 2, 4 or 6 and writes
N_ghost = 1, 2, 3 for them (Sec. 3.1); the PM grid is padded by 2 N_ghost cells on
every side and the Dirichlet values fill the N_ghost layers next to the interior
(App. C).  The stencils are the standard central ones, written here with their
coefficients for offsets m = 0 .. N_ghost:

  gradient           f'(x)  = (1/d)   sum_m  g_m (f(x + m d) - f(x - m d))
  second derivative  f''(x) = (1/d^2) [s_0 f(x) + sum_m s_m (f(x + m d) + f(x - m d))]

and their Fourier symbols on a mode exp(i k x): i (2/d) sum_m g_m sin(m k d) and
(1/d^2) (s_0 + 2 sum_m s_m cos(m k d)).  The DST-I eigenvalues of App. C are the
second-derivative symbol at k d = pi l / (N + 1); the paper prints them as sin^2
sums (``dst_eigenvalues`` follows that printed form, and a pin checks it against
the symbol of the stencil).

Pins (tests/test_oracle_fda.py): each stencil is exact on polynomials up to its
order; the printed eigenvalues equal the stencil symbol; DST-I basis vectors are
eigenvectors of the stencil applied with odd continuation across the Dirichlet
planes.
"""
import numpy as np


def n_ghost(order):
    """N_ghost = 1, 2, 3 for FDA order 2, 4, 6."""
    if order not in (2, 4, 6):
        raise ValueError("FDA order must be 2, 4 or 6")
    return order // 2


def gradient_coefficients(order):
    """g_m, m = 1 .. N_ghost, of the central first derivative."""
    return {2: [1.0 / 2.0],
            4: [2.0 / 3.0, -1.0 / 12.0],
            6: [3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0]}[order]


def second_derivative_coefficients(order):
    """s_m, m = 0 .. N_ghost, of the central second derivative."""
    return {2: [-2.0, 1.0],
            4: [-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0],
            6: [-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0]}[order]


def gradient_symbol(k, d, order):
    """Real factor G(k) of the gradient's Fourier symbol i G(k)."""
    g = gradient_coefficients(order)
    return (2.0 / d) * sum(gm * np.sin((m + 1) * k * d) for m, gm in enumerate(g))


def second_derivative_symbol(k, d, order):
    """Fourier symbol of the second derivative (real, <= 0), written as
    (2/d^2) sum_m s_m (cos(m k d) - 1): the central stencils have s_0 = -2 sum_m s_m, and
    this form vanishes exactly at k = 0 (no cancellation of s_0 against the sum)."""
    s = second_derivative_coefficients(order)
    return 2.0 * sum(sm * (np.cos(m * k * d) - 1.0) for m, sm in enumerate(s) if m > 0) / d**2


def dst_eigenvalues(N, d, order):
    """lambda_l, l = 1..N, as printed in App. C for FDA order 2, 4, 6 (with
    k_l d / 4 * N / (N + 1) = pi l / (2 (N + 1)) =: t)."""
    t = np.pi * np.arange(1, N + 1, dtype=np.float64) / (2.0 * (N + 1))
    if order == 2:
        return -(4.0 / d**2) * np.sin(t) ** 2
    if order == 4:
        return (np.sin(2 * t) ** 2 - 16.0 * np.sin(t) ** 2) / (3.0 * d**2)
    if order == 6:
        return -(2.0 * np.sin(3 * t) ** 2 - 27.0 * np.sin(2 * t) ** 2 + 270.0 * np.sin(t) ** 2) / (45.0 * d**2)
    raise ValueError("FDA order must be 2, 4 or 6")
