"""Pins of the oracle's final density and P(k) estimator (Sec. 4.1-4.2, Eq. 24)."""
import numpy as np

from oracle import scola, stats


def test_uniform_lattice_has_zero_density_contrast():
    Np, L = 8, 20.0
    q = scola.lattice_positions(Np, L)
    assert np.abs(stats.cic_density_periodic(q, L, Np, Np)).max() < 1e-13
    assert np.abs(stats.cic_density_periodic(q + 100 * L, L, Np, Np)).max() < 1e-9


def test_single_cosine_power():
    # delta = A cos(2 pi x / L): |DFT|^2 = A^2 N^6 / 4 at +-k, so the fundamental bin
    # (6 modes of |k| = 2 pi / L) averages 2 * A^2 L^3 / 4 / 6.
    N, L, A = 16, 50.0, 0.3
    x = np.arange(N)[:, None, None] * np.ones((1, N, N))
    delta = A * np.cos(2 * np.pi * x / N)
    kf = 2 * np.pi / L
    k, P, n = stats.power_spectrum(delta, L, np.array([0.5 * kf, 1.2 * kf, 1.5 * kf]))
    assert n[0] == 6 and abs(P[0] - A**2 * L**3 / 12) < 1e-12 * A**2 * L**3
    assert abs(P[1]) < 1e-20 + 1e-12 * P[0]


def test_density_mass_conservation():
    Np, N, L = 8, 4, 10.0
    rng = np.random.default_rng(0)
    x = rng.uniform(-L, 2 * L, size=(Np**3, 3))
    d = stats.cic_density_periodic(x, L, N, Np)
    assert abs(d.mean()) < 1e-12
